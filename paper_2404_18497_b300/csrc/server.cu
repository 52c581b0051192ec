// Serving loop: built MPHFs stay resident on the device and requests of three
// kinds arrive at any time from any host thread.
//   build   (keys on the device, parameters)  -> a resident MPHF id
//   query   (resident id, keys, output)       -> positions written to output
//   release (resident id)                     -> its memory returned
// The paper has no counterpart; this is a deployment layer around the
// construction and query of the paper, whose arithmetic it does not touch.
//
// Continuous mode (the default):
//   * Builds are admitted in arrival order while at most `build_slots` run and
//     the bytes of resident MPHFs plus the estimated peak of admitted builds
//     stay within the HBM budget.  A build that does not fit waits (and those
//     behind it) until releases or finished builds free memory.  Each build
//     slot has a host worker thread and its own stream; the builds' kernels
//     overlap on the device with each other and with queries.
//   * Pending query requests, against any resident MPHFs, are coalesced into
//     one kernel launch on a high-priority stream (up to max_batch_requests
//     requests and max_batch_keys keys) while builds run.  Up to `launch_slots`
//     coalesced launches are in flight; requests that arrive meanwhile form the
//     next launch.  An event recorded after each launch marks its completion;
//     the scheduler thread polls the events of the launches in flight, in
//     launch order, and completes their requests (no host callbacks: a
//     callback thread taking the server's lock for every launch competed with
//     the submitting threads).
//   * A release waits until no queued or in-flight query reads the MPHF, then
//     returns its memory in stream order (no device synchronisation).
// Serial mode: one request at a time in arrival order, each as its own launch
// sequence waited for to completion (the plain path to compare with).
//
// The scheduler never holds its mutex across a CUDA call.  Submissions wake it
// only while it sleeps; while launches are in flight it polls their events.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/phobic.h"
#include "phobic_dev.cuh"
#include "phobic_kernels.cuh"

namespace {

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

// Peak device bytes of a build of n keys beyond its input: hashed and sorted
// keys (ping-pong, 16 B/key), bucket-sorted keys (8 B/key), the pilot matrix
// (4/lambda B/key) and smaller per-partition arrays; 32 B/key + 64 MiB bounds
// them for lambda >= 1.
uint64_t build_estimate(uint64_t n) { return 32ull * n + (64ull << 20); }

struct Req {
    uint64_t id = 0;
    uint32_t kind = 0;
    const uint64_t* keys = nullptr;
    uint64_t* out = nullptr;
    uint64_t n = 0;
    phobic_params prm{};
    uint64_t handle = 0;
    phobic_handle* h = nullptr;  // query: the MPHF it reads
    cudaEvent_t ready = nullptr;
    uint64_t est = 0;
    bool waited = false;
    int64_t t_submit = 0, t_start = 0, t_done = 0;
    uint32_t batch_requests = 0;
    uint64_t batch_id = 0;
};

struct Resident {
    phobic_handle* h = nullptr;
    uint64_t bytes = 0;
    uint32_t refs = 0;  // submitted queries not yet completed
    bool releasing = false;
};

struct Slot;

}  // namespace

struct phobic_server {
    phobic_server_config cfg{};
    std::mutex mu;
    std::condition_variable cv;       // scheduler
    std::condition_variable cv_work;  // build workers
    std::condition_variable cv_idle;  // drain
    std::deque<Req*> q_builds;        // waiting for admission
    std::deque<Req*> q_admitted;      // admitted, waiting for a worker
    std::deque<Req*> q_queries;
    std::deque<Req*> q_releases;
    std::deque<Req*> q_serial;  // serial mode: every request, in arrival order
    std::deque<phobic_completion> done;
    std::unordered_map<uint64_t, Resident> res;
    std::vector<Slot*> slots;
    std::vector<std::thread> workers;
    std::thread sched;
    cudaStream_t qstream = nullptr;
    std::vector<cudaStream_t> bstreams;
    int device = 0;
    bool stop = false;
    bool sched_waiting = false;  // the scheduler sleeps on cv (submissions must wake it)
    std::atomic<uint64_t> work_seq{0};  // bumped by every submission and finished build
    uint64_t next_id = 1, next_handle = 1, next_batch = 1;
    uint64_t pending = 0;
    uint32_t active_builds = 0;
    phobic_server_stats st{};
};

namespace {

// one coalesced query launch in flight
struct Slot {
    phobic_server* srv = nullptr;
    phobic::MultiQuery* h_desc = nullptr;  // pinned
    phobic::MultiQuery* d_desc = nullptr;
    cudaEvent_t done = nullptr;            // recorded after the launch
    std::vector<Req*> reqs;
    bool busy = false;
};

void complete_locked(phobic_server* s, Req* r, phobic_status status) {
    phobic_completion c{};
    c.request_id = r->id;
    c.kind = r->kind;
    c.status = (int32_t)status;
    c.handle_id = r->handle;
    c.keys = r->n;
    c.t_submit_ns = r->t_submit;
    c.t_start_ns = r->t_start;
    c.t_done_ns = r->t_done ? r->t_done : now_ns();
    c.batch_requests = r->batch_requests;
    c.batch_id = r->batch_id;
    s->done.push_back(c);
    if (r->kind == PHOBIC_REQ_BUILD) s->st.builds_done++;
    if (r->kind == PHOBIC_REQ_QUERY) {
        s->st.queries_done++;
        auto it = s->res.find(r->handle);
        if (it != s->res.end()) it->second.refs--;
    }
    if (r->kind == PHOBIC_REQ_RELEASE) s->st.releases_done++;
    s->pending--;
    delete r;
    if (s->pending == 0) s->cv_idle.notify_all();
}

// a launch's requests are done (caller holds the lock)
void finish_slot_locked(phobic_server* s, Slot* slot, phobic_status status, int64_t t) {
    for (Req* r : slot->reqs) {
        r->t_done = t;
        complete_locked(s, r, status);
    }
    slot->reqs.clear();
    slot->busy = false;
}

void account_peak(phobic_server* s) {
    const uint64_t a = s->st.resident_bytes + s->st.reserved_bytes;
    if (a > s->st.peak_accounted_bytes) s->st.peak_accounted_bytes = a;
}

// a finished build: register the MPHF (caller holds the lock)
void finish_build_locked(phobic_server* s, Req* r, phobic_status status, phobic_handle* h) {
    if (status == PHOBIC_OK) {
        phobic_info info{};
        phobic_get_info(h, &info);
        const uint64_t id = s->next_handle++;
        s->res[id] = Resident{h, info.device_bytes, 0, false};
        s->st.resident_bytes += info.device_bytes;
        s->st.resident_handles++;
        r->handle = id;
        account_peak(s);
    }
    complete_locked(s, r, status);
}

phobic_status run_build(Req* r, cudaStream_t bs, phobic_handle** h) {
    r->t_start = now_ns();
    phobic_status status = PHOBIC_OK;
    if (r->ready && cudaStreamWaitEvent(bs, r->ready, 0) != cudaSuccess) status = PHOBIC_ERR_CUDA;
    if (status == PHOBIC_OK) status = phobic_build_ex(r->keys, r->n, &r->prm, (phobic_stream_t)bs, h);
    r->t_done = now_ns();
    return status;
}

void build_worker(phobic_server* s, uint32_t w) {
    cudaSetDevice(s->device);
    phobic::warm_build_thread();  // no pinned allocation inside the first request's build
    for (;;) {
        Req* r = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || !s->q_admitted.empty(); });
            if (s->q_admitted.empty()) return;  // stopping
            r = s->q_admitted.front();
            s->q_admitted.pop_front();
        }
        phobic_handle* h = nullptr;
        const phobic_status status = run_build(r, s->bstreams[w], &h);
        std::lock_guard<std::mutex> lk(s->mu);
        s->st.reserved_bytes -= r->est;
        s->active_builds--;
        finish_build_locked(s, r, status, h);
        s->work_seq.fetch_add(1, std::memory_order_release);
        s->cv.notify_all();
    }
}

// admission of waiting builds in arrival order (caller holds the lock)
void admit_locked(phobic_server* s) {
    while (!s->q_builds.empty() && s->active_builds < s->cfg.build_slots) {
        Req* r = s->q_builds.front();
        const uint64_t budget = s->cfg.hbm_budget_bytes;
        const uint64_t committed = s->st.resident_bytes + s->st.reserved_bytes;
        // a build larger than the whole budget runs alone, once nothing else is committed
        const bool fits = budget == 0 || committed + r->est <= budget || (committed == 0 && s->active_builds == 0);
        if (!fits) {
            if (!r->waited) {
                r->waited = true;
                s->st.builds_waited_for_memory++;
            }
            return;
        }
        s->q_builds.pop_front();
        s->st.reserved_bytes += r->est;
        s->active_builds++;
        account_peak(s);
        s->q_admitted.push_back(r);
        s->cv_work.notify_one();
    }
}

// releases whose MPHF no query reads any more (caller holds the lock); the
// handles are freed after the lock is dropped
void take_releases_locked(phobic_server* s, std::vector<std::pair<Req*, phobic_handle*>>& out) {
    for (size_t i = 0; i < s->q_releases.size();) {
        Req* r = s->q_releases[i];
        auto it = s->res.find(r->handle);
        if (it->second.refs == 0) {
            out.emplace_back(r, it->second.h);
            s->st.resident_bytes -= it->second.bytes;
            s->st.resident_handles--;
            s->res.erase(it);
            s->q_releases.erase(s->q_releases.begin() + (long)i);
        } else {
            i++;
        }
    }
}

// pending queries into a free launch slot (caller holds the lock)
Slot* take_queries_locked(phobic_server* s) {
    if (s->q_queries.empty()) return nullptr;
    Slot* sl = nullptr;
    for (Slot* x : s->slots)
        if (!x->busy) {
            sl = x;
            break;
        }
    if (!sl) return nullptr;
    uint64_t keys = 0;
    const int64_t t = now_ns();
    while (!s->q_queries.empty() && sl->reqs.size() < s->cfg.max_batch_requests) {
        Req* r = s->q_queries.front();
        if (!sl->reqs.empty() && keys + r->n > s->cfg.max_batch_keys) break;
        s->q_queries.pop_front();
        r->t_start = t;
        keys += r->n;
        sl->reqs.push_back(r);
    }
    sl->busy = true;
    const uint64_t bid = s->next_batch++;
    for (Req* r : sl->reqs) {
        r->batch_requests = (uint32_t)sl->reqs.size();
        r->batch_id = bid;
    }
    s->st.query_launches++;
    s->st.max_batch_requests_seen = std::max<uint64_t>(s->st.max_batch_requests_seen, sl->reqs.size());
    return sl;
}

// descriptors, waits on the requests' ready events, one launch and the
// completion host function, all on the query stream (no lock held)
cudaError_t launch_slot(phobic_server* s, Slot* sl) {
    uint64_t begin = 0;
    uint32_t k = 0;
    cudaError_t e = cudaSuccess;
    for (Req* r : sl->reqs) {
        if (r->ready && (e = cudaStreamWaitEvent(s->qstream, r->ready, 0)) != cudaSuccess) return e;
        if (r->n == 0) continue;
        sl->h_desc[k++] = phobic::MultiQuery{*phobic::handle_view(r->h), r->keys, r->out, begin};
        begin += r->n;
    }
    if (k) {
        e = cudaMemcpyAsync(sl->d_desc, sl->h_desc, k * sizeof(phobic::MultiQuery), cudaMemcpyHostToDevice,
                            s->qstream);
        if (e == cudaSuccess) e = phobic::launch_query_multi(sl->d_desc, k, begin, s->qstream);
        if (e != cudaSuccess) return e;
    }
    return cudaEventRecord(sl->done, s->qstream);
}

// pause of about a microsecond between two polls, without a system call
inline void poll_pause() {
    for (int i = 0; i < 64; i++) {
#if defined(__x86_64__) || defined(__i386__)
        __builtin_ia32_pause();
#else
        std::atomic_signal_fence(std::memory_order_seq_cst);
#endif
    }
}

void scheduler_continuous(phobic_server* s) {
    cudaSetDevice(s->device);
    std::vector<std::pair<Req*, phobic_handle*>> rel;
    std::deque<Slot*> inflight;  // launched, in launch order (they finish in order on the query stream)
    std::vector<std::pair<Slot*, phobic_status>> finished;
    for (;;) {
        // launches that have finished, oldest first (polled without the lock)
        while (!inflight.empty()) {
            const cudaError_t q = cudaEventQuery(inflight.front()->done);
            if (q == cudaErrorNotReady) break;
            finished.emplace_back(inflight.front(), q == cudaSuccess ? PHOBIC_OK : PHOBIC_ERR_CUDA);
            inflight.pop_front();
        }
        Slot* sl = nullptr;
        bool idle = false;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (!finished.empty()) {
                const int64_t t = now_ns();
                for (auto& f : finished) finish_slot_locked(s, f.first, f.second, t);
                finished.clear();
            }
            take_releases_locked(s, rel);
            admit_locked(s);
            if (rel.empty()) sl = take_queries_locked(s);
            if (rel.empty() && !sl) {
                if (s->stop && s->pending == 0 && inflight.empty()) return;
                if (inflight.empty()) {
                    s->sched_waiting = true;
                    s->cv.wait_for(lk, std::chrono::milliseconds(2));
                    s->sched_waiting = false;
                    continue;
                }
                idle = true;
            }
        }
        if (idle) {  // launches in flight, nothing new: poll, without the lock, until one finishes or work arrives
            const uint64_t seen = s->work_seq.load(std::memory_order_acquire);
            while (cudaEventQuery(inflight.front()->done) == cudaErrorNotReady &&
                   s->work_seq.load(std::memory_order_acquire) == seen)
                poll_pause();
            continue;
        }
        for (auto& pr : rel) {
            pr.first->t_start = now_ns();
            phobic::handle_free_idle(pr.second, s->qstream);
            pr.first->t_done = now_ns();
            std::lock_guard<std::mutex> lk(s->mu);
            complete_locked(s, pr.first, PHOBIC_OK);
        }
        rel.clear();
        if (sl) {
            const cudaError_t e = launch_slot(s, sl);
            if (e != cudaSuccess) {
                std::lock_guard<std::mutex> lk(s->mu);
                finish_slot_locked(s, sl, PHOBIC_ERR_CUDA, now_ns());
            } else {
                inflight.push_back(sl);
            }
        }
    }
}

void scheduler_serial(phobic_server* s) {
    cudaSetDevice(s->device);
    phobic::warm_build_thread();
    for (;;) {
        Req* r = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] { return s->stop || !s->q_serial.empty(); });
            if (s->q_serial.empty()) return;  // stopping, nothing left
            r = s->q_serial.front();
            s->q_serial.pop_front();
        }
        if (r->kind == PHOBIC_REQ_BUILD) {
            phobic_handle* h = nullptr;
            const phobic_status status = run_build(r, s->qstream, &h);
            std::lock_guard<std::mutex> lk(s->mu);
            finish_build_locked(s, r, status, h);
        } else if (r->kind == PHOBIC_REQ_QUERY) {
            r->t_start = now_ns();
            phobic_status status = PHOBIC_OK;
            if (r->ready && cudaStreamWaitEvent(s->qstream, r->ready, 0) != cudaSuccess) status = PHOBIC_ERR_CUDA;
            if (status == PHOBIC_OK) status = phobic_query(r->h, r->keys, r->out, r->n, (phobic_stream_t)s->qstream);
            if (status == PHOBIC_OK && cudaStreamSynchronize(s->qstream) != cudaSuccess) status = PHOBIC_ERR_CUDA;
            r->t_done = now_ns();
            r->batch_requests = 1;
            std::lock_guard<std::mutex> lk(s->mu);
            r->batch_id = s->next_batch++;
            s->st.query_launches++;
            s->st.max_batch_requests_seen = std::max<uint64_t>(s->st.max_batch_requests_seen, 1);
            complete_locked(s, r, status);
        } else {
            r->t_start = now_ns();
            phobic_handle* h = nullptr;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                auto it = s->res.find(r->handle);
                h = it->second.h;
                s->st.resident_bytes -= it->second.bytes;
                s->st.resident_handles--;
                s->res.erase(it);
            }
            phobic::handle_free_idle(h, s->qstream);
            r->t_done = now_ns();
            std::lock_guard<std::mutex> lk(s->mu);
            complete_locked(s, r, PHOBIC_OK);
        }
    }
}

phobic_status submit(phobic_server* s, Req* r, uint64_t* request_id) {
    r->t_submit = now_ns();
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
        delete r;
        return PHOBIC_ERR_INVALID_ARG;
    }
    r->id = s->next_id++;
    if (request_id) *request_id = r->id;
    s->pending++;
    if (s->cfg.serial) {
        s->q_serial.push_back(r);
    } else if (r->kind == PHOBIC_REQ_BUILD) {
        s->q_builds.push_back(r);
        admit_locked(s);
    } else if (r->kind == PHOBIC_REQ_QUERY) {
        s->q_queries.push_back(r);
    } else {
        s->q_releases.push_back(r);
    }
    // the serial scheduler waits on cv for every request; the continuous one
    // polls while launches are in flight and needs waking only when it sleeps
    s->work_seq.fetch_add(1, std::memory_order_release);
    if (s->cfg.serial || s->sched_waiting) s->cv.notify_all();
    return PHOBIC_OK;
}

}  // namespace

extern "C" {

void phobic_server_config_init(phobic_server_config* c) {
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->build_slots = 2;
    c->max_batch_requests = 1024;
    c->max_batch_keys = 1ull << 24;
    c->launch_slots = 4;
}

phobic_status phobic_server_create(const phobic_server_config* cfg, phobic_server** out) {
    if (!out) return PHOBIC_ERR_INVALID_ARG;
    *out = nullptr;
    phobic_server_config c;
    phobic_server_config_init(&c);
    if (cfg) c = *cfg;
    if (c.build_slots == 0) c.build_slots = 2;
    if (c.max_batch_requests == 0) c.max_batch_requests = 1024;
    if (c.max_batch_keys == 0) c.max_batch_keys = 1ull << 24;
    if (c.launch_slots == 0) c.launch_slots = 4;
    if (c.build_slots > 64 || c.launch_slots > 64 || c.max_batch_requests > (1u << 20)) return PHOBIC_ERR_INVALID_ARG;
    phobic_server* s = new (std::nothrow) phobic_server();
    if (!s) return PHOBIC_ERR_OOM;
    s->cfg = c;
    auto fail = [&](phobic_status st) {
        for (Slot* sl : s->slots) {
            if (sl->h_desc) cudaFreeHost(sl->h_desc);
            if (sl->d_desc) cudaFree(sl->d_desc);
            if (sl->done) cudaEventDestroy(sl->done);
            delete sl;
        }
        for (cudaStream_t b : s->bstreams) cudaStreamDestroy(b);
        if (s->qstream) cudaStreamDestroy(s->qstream);
        delete s;
        return st;
    };
    if (cudaGetDevice(&s->device) != cudaSuccess) return fail(PHOBIC_ERR_CUDA);
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) return fail(PHOBIC_ERR_CUDA);
    if (cudaStreamCreateWithPriority(&s->qstream, cudaStreamNonBlocking, greatest) != cudaSuccess)
        return fail(PHOBIC_ERR_CUDA);
    if (!c.serial) {
        for (uint32_t w = 0; w < c.build_slots; w++) {
            cudaStream_t b = nullptr;
            if (cudaStreamCreateWithPriority(&b, cudaStreamNonBlocking, least) != cudaSuccess)
                return fail(PHOBIC_ERR_CUDA);
            s->bstreams.push_back(b);
        }
        for (uint32_t i = 0; i < c.launch_slots; i++) {
            Slot* sl = new (std::nothrow) Slot();
            if (!sl) return fail(PHOBIC_ERR_OOM);
            s->slots.push_back(sl);
            sl->srv = s;
            const size_t bytes = (size_t)c.max_batch_requests * sizeof(phobic::MultiQuery);
            if (cudaMallocHost(&sl->h_desc, bytes) != cudaSuccess || cudaMalloc(&sl->d_desc, bytes) != cudaSuccess)
                return fail(PHOBIC_ERR_OOM);
            if (cudaEventCreateWithFlags(&sl->done, cudaEventDisableTiming) != cudaSuccess)
                return fail(PHOBIC_ERR_CUDA);
            sl->reqs.reserve(c.max_batch_requests);
        }
    }
    if (c.serial) {
        s->sched = std::thread(scheduler_serial, s);
    } else {
        s->sched = std::thread(scheduler_continuous, s);
        for (uint32_t w = 0; w < c.build_slots; w++) s->workers.emplace_back(build_worker, s, w);
    }
    *out = s;
    return PHOBIC_OK;
}

phobic_status phobic_server_submit_build(phobic_server* s, const uint64_t* d_keys, uint64_t n,
                                         const phobic_params* params, phobic_event_t ready, uint64_t* request_id) {
    if (!s || !d_keys || n == 0 || !params) return PHOBIC_ERR_INVALID_ARG;
    Req* r = new (std::nothrow) Req();
    if (!r) return PHOBIC_ERR_OOM;
    r->kind = PHOBIC_REQ_BUILD;
    r->keys = d_keys;
    r->n = n;
    r->prm = *params;
    r->ready = (cudaEvent_t)ready;
    r->est = build_estimate(n);
    return submit(s, r, request_id);
}

phobic_status phobic_server_submit_query(phobic_server* s, uint64_t handle_id, const uint64_t* d_keys,
                                         uint64_t* d_out, uint64_t m, phobic_event_t ready, uint64_t* request_id) {
    if (!s || (m && (!d_keys || !d_out))) return PHOBIC_ERR_INVALID_ARG;
    Req* r = new (std::nothrow) Req();
    if (!r) return PHOBIC_ERR_OOM;
    r->kind = PHOBIC_REQ_QUERY;
    r->keys = d_keys;
    r->out = d_out;
    r->n = m;
    r->handle = handle_id;
    r->ready = (cudaEvent_t)ready;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->res.find(handle_id);
        if (it == s->res.end() || it->second.releasing || phobic::handle_view(it->second.h)->key_kind != 0) {
            delete r;
            return PHOBIC_ERR_INVALID_ARG;
        }
        r->h = it->second.h;
        it->second.refs++;  // the MPHF stays until this request completes
    }
    return submit(s, r, request_id);
}

phobic_status phobic_server_submit_release(phobic_server* s, uint64_t handle_id, uint64_t* request_id) {
    if (!s) return PHOBIC_ERR_INVALID_ARG;
    Req* r = new (std::nothrow) Req();
    if (!r) return PHOBIC_ERR_OOM;
    r->kind = PHOBIC_REQ_RELEASE;
    r->handle = handle_id;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->res.find(handle_id);
        if (it == s->res.end() || it->second.releasing) {
            delete r;
            return PHOBIC_ERR_INVALID_ARG;
        }
        it->second.releasing = true;
    }
    return submit(s, r, request_id);
}

phobic_status phobic_server_poll(phobic_server* s, phobic_completion* out, uint32_t cap, uint32_t* count) {
    if (!s || !count || (cap && !out)) return PHOBIC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    uint32_t k = 0;
    while (k < cap && !s->done.empty()) {
        out[k++] = s->done.front();
        s->done.pop_front();
    }
    *count = k;
    return PHOBIC_OK;
}

phobic_status phobic_server_drain(phobic_server* s, double timeout_s) {
    if (!s) return PHOBIC_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    const bool ok = s->cv_idle.wait_for(lk, std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0.0),
                                        [&] { return s->pending == 0; });
    return ok ? PHOBIC_OK : PHOBIC_ERR_TIMEOUT;
}

phobic_status phobic_server_handle(phobic_server* s, uint64_t handle_id, const phobic_handle** out) {
    if (!s || !out) return PHOBIC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->res.find(handle_id);
    if (it == s->res.end()) return PHOBIC_ERR_INVALID_ARG;
    *out = it->second.h;
    return PHOBIC_OK;
}

phobic_status phobic_server_get_stats(phobic_server* s, phobic_server_stats* out) {
    if (!s || !out) return PHOBIC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    out->pending = s->pending;
    return PHOBIC_OK;
}

void phobic_server_destroy(phobic_server* s) {
    if (!s) return;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        s->cv_idle.wait(lk, [&] { return s->pending == 0; });
        s->stop = true;
    }
    s->cv.notify_all();
    s->cv_work.notify_all();
    if (s->sched.joinable()) s->sched.join();
    for (auto& t : s->workers) t.join();
    cudaStreamSynchronize(s->qstream);
    for (auto& kv : s->res) phobic::handle_free_idle(kv.second.h, s->qstream);
    cudaStreamSynchronize(s->qstream);
    for (Slot* sl : s->slots) {
        cudaFreeHost(sl->h_desc);
        cudaFree(sl->d_desc);
        cudaEventDestroy(sl->done);
        delete sl;
    }
    for (cudaStream_t b : s->bstreams) cudaStreamDestroy(b);
    cudaStreamDestroy(s->qstream);
    delete s;
}

}  // extern "C"
