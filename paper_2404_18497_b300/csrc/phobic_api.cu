// libphobic C ABI: argument checks, build orchestration, the handle,
// serialization and space accounting.  Every step of construction and query
// runs in the kernels of k_*.cu; this file only sequences them, sizes buffers
// from the few scalars the device reports, and owns memory.
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "../../include/phobic.h"
#include "phobic_dev.cuh"
#include "phobic_kernels.cuh"

using namespace phobic;

namespace phobic {
static std::atomic<uint64_t> g_launches{0};
void note_launches(uint64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
}  // namespace phobic

namespace {

constexpr uint64_t kMagic = 0x31304349424F4850ull;  // "PHOBIC01"
constexpr uint64_t kFormatVersion = 1;

// ---------------------------------------------------------------- table ---
// Appendix C: gamma tabulated at 2048 points, as 32-bit fixed point.
//   eps = lambda / (5 sqrt P) (clamped to 1), beta_*(x) = x + (1-x) ln(1-x),
//   gamma(x) = eps x + (1 - eps) beta_*(x), gamma(1) = 1;
//   alpha < 1 (Appendix B): gamma_alpha(x) = gamma(alpha x) / gamma(alpha).
// Compiled with -ffp-contract=off: every operation rounds separately.
double eps_of(double lambda, uint32_t P) {
    double e = lambda / (5.0 * std::sqrt((double)P));
    return e > 1.0 ? 1.0 : e;
}

double beta_star(double x) { return x >= 1.0 ? 1.0 : x + (1.0 - x) * std::log1p(-x); }

// gamma before the alpha rescaling: beta_eps (Theorem 2), beta_* (eps = 0),
// PTHash's skewed split (hash < 0.6 -> first 30 % of the buckets) or uniform
double gamma_base(double x, double eps, uint32_t fn) {
    if (x >= 1.0) return 1.0;
    switch (fn) {
        case PHOBIC_BUCKET_BETA_STAR: return beta_star(x);
        case PHOBIC_BUCKET_SKEWED: return x < 0.6 ? 0.5 * x : 0.3 + 1.75 * (x - 0.6);
        case PHOBIC_BUCKET_UNIFORM: return x;
        default: return eps * x + (1.0 - eps) * beta_star(x);
    }
}

void make_table(double lambda, double alpha, uint32_t P, uint64_t* t, uint32_t fn = PHOBIC_BUCKET_OPTIMIZED) {
    const double eps = eps_of(lambda, P);
    for (int k = 0; k <= kTablePoints; k++) {
        const double x = (double)k / (double)kTablePoints;
        double g;
        if (alpha == 1.0) {
            g = gamma_base(x, eps, fn);
        } else if (fn == PHOBIC_BUCKET_OPTIMIZED) {
            const double ax = alpha * x;
            g = (eps * ax + (1.0 - eps) * beta_star(ax)) / (eps * alpha + (1.0 - eps) * beta_star(alpha));
        } else {
            g = gamma_base(alpha * x, eps, fn) / gamma_base(alpha, eps, fn);  // Appendix B
        }
        long long r = std::llround(g * 4294967296.0);
        if (r < 0) r = 0;
        if (r > 4294967296LL) r = 4294967296LL;
        t[k] = (uint64_t)r;
    }
}

// The table of a parameter set, computed once per process (2049 evaluations of
// gamma take tens of microseconds, and builds repeat their parameters)
void cached_table(double lambda, double alpha, uint32_t P, uint32_t fn, uint64_t* t) {
    static std::mutex mu;
    static std::map<std::tuple<double, double, uint32_t, uint32_t>, std::vector<uint64_t>> cache;
    const auto key = std::make_tuple(lambda, alpha, P, fn);
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            std::memcpy(t, it->second.data(), it->second.size() * 8);
            return;
        }
    }
    std::vector<uint64_t> v(kTablePoints + 1);
    make_table(lambda, alpha, P, v.data(), fn);
    std::memcpy(t, v.data(), v.size() * 8);
    std::lock_guard<std::mutex> lock(mu);
    if (cache.size() < 4096) cache.emplace(key, std::move(v));
}

uint32_t num_buckets(double lambda, uint32_t P) {
    double b = std::ceil((double)P / lambda);
    return b < 1.0 ? 1u : (uint32_t)b;
}

// Golomb-Rice parameter of an IC-R column with `count` pilots summing to `sum`:
// Kiely's choice for a geometric source with the column's mean mu,
// max(0, 1 + floor(log2(log(phi - 1) / log(theta)))), theta = mu / (mu + 1),
// phi the golden ratio; at most 31.  Computed on the host in double.
uint32_t rice_param(uint64_t sum, uint64_t count) {
    if (sum == 0 || count == 0) return 0;
    const double mu = (double)sum / (double)count;
    const double theta = mu / (mu + 1.0);
    const double ratio = std::log((std::sqrt(5.0) - 1.0) / 2.0) / std::log(theta);
    const double k = 1.0 + std::floor(std::log2(ratio));
    if (!(k > 0.0)) return 0;
    if (k > 31.0) return 31;
    return (uint32_t)k;
}

uint64_t num_partitions(uint64_t n, uint32_t P) {
    uint64_t np = (n + P - 1) / P;
    return np ? np : 1;
}
uint64_t num_partitions_of(uint64_t n, uint32_t P) { return num_partitions(n, P); }

phobic_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return PHOBIC_OK;
    if (e == cudaErrorMemoryAllocation) return PHOBIC_ERR_OOM;
    return PHOBIC_ERR_CUDA;
}

// keep freed stream-ordered allocations cached in the pool between builds
void ensure_pool() {
    static std::once_flag once;
    std::call_once(once, [] {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return;
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return;
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    });
}

// stream-ordered allocations released together unless ownership is taken
struct Arena {
    cudaStream_t st;
    std::vector<void*> ptrs;
    explicit Arena(cudaStream_t s) : st(s) {}
    ~Arena() {
        for (void* p : ptrs) cudaFreeAsync(p, st);
    }
    template <class T>
    cudaError_t alloc(T** out, size_t bytes) {
        void* p = nullptr;
        cudaError_t e = cudaMallocAsync(&p, bytes ? bytes : 16, st);
        if (e != cudaSuccess) return e;
        ptrs.push_back(p);
        *out = static_cast<T*>(p);
        return cudaSuccess;
    }
    void release(void* p) {
        for (auto& q : ptrs)
            if (q == p) {
                cudaFreeAsync(q, st);
                q = ptrs.back();
                ptrs.pop_back();
                return;
            }
    }
};

// CUDA events around the build phases (only when requested)
struct PhaseEvents {
    bool on = false;
    cudaEvent_t ev[8] = {};
    int used = 0;
    ~PhaseEvents() {
        for (int i = 0; i < used; i++) cudaEventDestroy(ev[i]);
    }
    cudaError_t init(bool enable) {
        on = enable;
        if (!on) return cudaSuccess;
        for (int i = 0; i < 8; i++) {
            cudaError_t e = cudaEventCreate(&ev[i]);
            if (e != cudaSuccess) return e;
            used = i + 1;
        }
        return cudaSuccess;
    }
    cudaError_t mark(int i, cudaStream_t st) { return on ? cudaEventRecord(ev[i], st) : cudaSuccess; }
    float between(int a, int b) const {
        float ms = 0.f;
        if (on) cudaEventElapsedTime(&ms, ev[a], ev[b]);
        return ms;
    }
};

// Small pinned host buffer for the scalars a build reads back, kept per host
// thread and grown on demand (pinned allocation is slow; builds are frequent).
struct PinnedBuf {
    void* p = nullptr;
    cudaError_t alloc(size_t bytes) {
        thread_local void* buf = nullptr;
        thread_local size_t cap = 0;
        if (cap < bytes) {
            // grow in whole 64 KB steps: a pinned allocation (and its release)
            // is slow and can stall other threads' CUDA calls
            const size_t want = (bytes + 65535) & ~(size_t)65535;
            if (buf) cudaFreeHost(buf);
            buf = nullptr;
            cap = 0;
            cudaError_t e = cudaMallocHost(&buf, want);
            if (e != cudaSuccess) return e;
            cap = want;
        }
        p = buf;
        return cudaSuccess;
    }
};

}  // namespace

// Device memory shared by the handles of one build (or one import): freed when
// the last handle that refers to it is freed.
struct SharedMem {
    void* ptr = nullptr;
    std::atomic<int> refs{0};
    size_t bytes = 0;
    bool pooled = false;  // from the stream-ordered pool (builds) rather than cudaMalloc (imports)
};

struct phobic_handle {
    phobic_params prm;
    phobic_info info;
    QueryView view;
    SharedMem* mem = nullptr;  // owns every device array below
    uint64_t* table = nullptr;
    uint64_t* off_words = nullptr;
    uint64_t* col_meta = nullptr;
    uint64_t* pil_words = nullptr;
    uint64_t* dict_words = nullptr;
    uint64_t* ef_low = nullptr;
    uint64_t* ef_high = nullptr;
    uint64_t* ef_samples = nullptr;
    uint32_t* pilots = nullptr;  // only with keep_pilots
    bool has_timings = false;
    phobic_timings timings;
    uint64_t n_off_words = 0, n_col_meta = 0, n_pil_words = 0, n_dict_words = 0;
    uint64_t n_ef_low = 0, n_ef_high = 0, n_ef_samples = 0;
};

namespace {

void release_mem(SharedMem* m) {
    if (m && m->refs.fetch_sub(1) == 1) {
        cudaDeviceSynchronize();
        cudaFree(m->ptr);
        delete m;
    }
}

void handle_destroy(phobic_handle* h) {
    if (!h) return;
    release_mem(h->mem);
    delete h;
}

}  // namespace

namespace phobic {
// Allocates the calling thread's pinned read-back buffer ahead of its first
// build (a server's build workers call it when they start).
cudaError_t warm_build_thread() {
    PinnedBuf pin;
    return pin.alloc(65536);
}

// Frees a handle without synchronising the device: the caller guarantees that
// no work that reads the handle is in flight.  Pool memory goes back to the
// pool in stream order on `st`; cudaMalloc'ed memory is freed directly.
void handle_free_idle(phobic_handle* h, cudaStream_t st) {
    if (!h) return;
    SharedMem* m = h->mem;
    if (m && m->refs.fetch_sub(1) == 1) {
        if (m->pooled)
            cudaFreeAsync(m->ptr, st);
        else
            cudaFree(m->ptr);
        delete m;
    }
    delete h;
}
}  // namespace phobic

namespace {

phobic_status check_params(uint64_t n, const phobic_params& p) {
    if (n == 0) return PHOBIC_ERR_INVALID_ARG;
    if (!(p.lambda > 0.0) || !std::isfinite(p.lambda)) return PHOBIC_ERR_INVALID_ARG;
    if (!(p.alpha > 0.0) || p.alpha > 1.0) return PHOBIC_ERR_INVALID_ARG;
    if (p.partition_size == 0 || p.partition_size > kMaxPartitionSize) return PHOBIC_ERR_INVALID_ARG;
    if ((double)p.partition_size < p.lambda) return PHOBIC_ERR_INVALID_ARG;  // fewer keys than one bucket
    if (p.encoder > PHOBIC_ENC_MONO_EF || p.pilot_mode > PHOBIC_PILOT_XOR) return PHOBIC_ERR_INVALID_ARG;
    if (p.compact_columns >= (1u << 24)) return PHOBIC_ERR_INVALID_ARG;
    if (p.warps_per_partition != 0 && p.warps_per_partition != 1 && p.warps_per_partition != 2 &&
        p.warps_per_partition != 4 && p.warps_per_partition != 8)
        return PHOBIC_ERR_INVALID_ARG;
    if (p.candidate_width != 0 && p.candidate_width != 32 && p.candidate_width != 64) return PHOBIC_ERR_INVALID_ARG;
    if (p.search_schedule > 2) return PHOBIC_ERR_INVALID_ARG;
    if (p.bucket_function > PHOBIC_BUCKET_UNIFORM) return PHOBIC_ERR_INVALID_ARG;
    return PHOBIC_OK;
}

template <class T>
cudaError_t d2h(T* host, const T* dev, size_t count, cudaStream_t st) {
    return cudaMemcpyAsync(host, dev, count * sizeof(T), cudaMemcpyDeviceToHost, st);
}
template <class T>
cudaError_t h2d(T* dev, const T* host, size_t count, cudaStream_t st) {
    return cudaMemcpyAsync(dev, host, count * sizeof(T), cudaMemcpyHostToDevice, st);
}

#define CK(x)                                         \
    do {                                              \
        cudaError_t _e = (x);                         \
        if (_e != cudaSuccess) return from_cuda(_e);  \
    } while (0)

// One key set of a build: keys [key_base, key_base + n) of the input.
struct SetIn {
    uint64_t key_base, n;
    uint32_t P;
};

// Per-set plan and layout, filled in as the build proceeds.
struct SetPlan {
    uint64_t key_base, n, NP, part_base, first_tile, pilot_base, col_base, M, g0;
    uint32_t P, B, table_idx;
    double eps;
    uint64_t Q;
    int64_t dmin;
    uint32_t off_w;
    // arena word offsets and sizes
    uint64_t a_off, n_off, a_meta, n_meta, a_pil, n_pil, a_dict, n_dict, a_low, n_low, a_high, n_high, a_samp,
        n_samp, a_pilots, samp_words;
    uint32_t mix_c;
    uint32_t ef_l;
    uint64_t bits_header, bits_offsets, bits_pilots, bits_remap, bits_total;
};

// Builds the MPHFs of every set of `sets` from one input array.  `in` holds raw
// 64-bit keys (hash_input = 1) or master hashes (hash_input = 0).  One handle per
// set is returned in `out`; all of them share one device arena.
// Waits for the work enqueued on st so far.  A build reads device results on
// the host several times; polling an event returns as soon as they are ready,
// where a blocking wait can add a scheduler round trip (measured: 0.3 ms per
// 1e8-key build while an NVML client such as nvidia-smi is attached, and no
// difference without one).  After kSpinWaitUs of polling it blocks instead, so
// that long builds do not keep a core busy.  Between two polls the thread
// pauses for about a microsecond without a system call: every poll is a driver
// call, and back-to-back polls from several building threads (a server's build
// slots) contend with the other threads' launches for the driver.
constexpr double kSpinWaitUs = 50000.0;
inline void pause_briefly() {
    for (int i = 0; i < 64; i++) {
#if defined(__x86_64__) || defined(__i386__)
        __builtin_ia32_pause();
#else
        std::atomic_signal_fence(std::memory_order_seq_cst);
#endif
    }
}
cudaError_t wait_stream(cudaStream_t st) {
    cudaEvent_t e;
    cudaError_t r = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    if (r != cudaSuccess) return r;
    r = cudaEventRecord(e, st);
    if (r == cudaSuccess) {
        const auto t0 = std::chrono::steady_clock::now();
        while ((r = cudaEventQuery(e)) == cudaErrorNotReady) {
            if (std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count() >
                kSpinWaitUs) {
                r = cudaEventSynchronize(e);
                break;
            }
            pause_briefly();
        }
    }
    cudaEventDestroy(e);
    return r;
}

// One shard's part of a partition-sharded build (Section 4: partitions are
// independent, so a build can be split by partition ranges across devices).
//   kShardSearch: bucketing and pilot search of partitions [j0, j1) only.  The
//     master hashes of exactly those partitions are given grouped by partition
//     (sorted, n_local of them; start: N_P + 1 entries indexing `sorted`, of
//     which j0..j1 are read), with the build's global slot offsets T.  Pilots
//     go to the global [B x N_P] matrix `pilots`, taken slots are ORed into the
//     global occupancy bitmap `taken` (may be null); no handle is made.
//   kShardAssemble: the rest of a build from the global partition starts
//     (start, N_P + 1), the full pilot matrix and (M > n) the full occupancy
//     bitmap: table sizes and offsets, encoding, remap, handle.  The result is
//     the structure a single build of the same keys makes.
// Either mode builds one set of sets[0].n keys (the whole build's n).
enum { kShardNone = 0, kShardSearch = 1, kShardAssemble = 2 };
struct ShardCtl {
    int mode;
    const uint64_t* sorted;
    uint64_t n_local;
    const uint64_t* start;
    const uint64_t* T;
    uint64_t j0, j1;
    uint32_t* pilots;
    uint32_t* taken;
};

phobic_status build_sets(const uint64_t* in, int hash_input, const std::vector<SetIn>& sets, const phobic_params& prm,
                         cudaStream_t st, uint32_t key_kind, std::vector<phobic_handle*>* out,
                         const ShardCtl* sc = nullptr) {
    const int smode = sc ? sc->mode : kShardNone;
    ensure_pool();
    const uint32_t S = (uint32_t)sets.size();
    const uint64_t kseed = key_seed(prm.seed);
    Arena tmp(st);
    PhaseEvents ev;
    CK(ev.init(prm.record_timings != 0));

    // ---- host plan
    std::vector<SetPlan> pl(S);
    std::vector<uint32_t> table_P;
    uint64_t n_total = 0, NPT = 0, tiles = 0, pilots_total = 0, cols_total = 0, max_np = 1;
    uint32_t cap_B = 1;
    for (uint32_t s = 0; s < S; s++) {
        SetPlan& p = pl[s];
        std::memset(&p, 0, sizeof(p));
        p.key_base = sets[s].key_base;
        p.n = sets[s].n;
        p.P = sets[s].P;
        p.NP = num_partitions(p.n, p.P);
        p.B = num_buckets(prm.lambda, p.P);
        p.eps = eps_of(prm.lambda, p.P);
        uint32_t ti = 0;
        while (ti < table_P.size() && table_P[ti] != p.P) ti++;
        if (ti == table_P.size()) table_P.push_back(p.P);
        p.table_idx = ti;
        p.part_base = NPT;
        p.first_tile = tiles;
        p.pilot_base = pilots_total;
        p.col_base = cols_total;
        NPT += p.NP;
        tiles += sort_tiles(p.n);
        pilots_total += (uint64_t)p.B * p.NP;
        cols_total += p.B;
        n_total += p.n;
        if (p.NP > max_np) max_np = p.NP;
        if (p.B > cap_B) cap_B = p.B;
    }
    const uint32_t ntab = (uint32_t)table_P.size();
    // the device holds each table packed (kTablePoints words, bucket_of)
    std::vector<uint64_t> tables((size_t)ntab * kTablePoints);
    {
        std::vector<uint64_t> t1(kTablePoints + 1);
        for (uint32_t t = 0; t < ntab; t++) {
            cached_table(prm.lambda, prm.alpha, table_P[t], prm.bucket_function, t1.data());
            pack_bucket_table(t1.data(), tables.data() + (size_t)t * kTablePoints);
        }
    }

    PinnedBuf pin;
    CK(pin.alloc(4096 + (size_t)S * 48 + (size_t)cols_total * 12));
    uint64_t* hst = static_cast<uint64_t*>(pin.p);
    uint64_t* hTb = hst + 32;                                       // [S + 1] set slot bases
    long long* hmm = reinterpret_cast<long long*>(hTb + S + 1);     // [2 S]
    uint32_t* hcolmax = reinterpret_cast<uint32_t*>(hmm + 2 * S);   // [cols_total]
    uint64_t* hK = reinterpret_cast<uint64_t*>(hcolmax + cols_total + (cols_total & 1));  // [cols_total]
    uint32_t* hstatus = reinterpret_cast<uint32_t*>(hst + 4);

    // ---- K1 + K2: hash, segmented partition sort, partition starts
    std::vector<SortSeg> segs(S);
    for (uint32_t s = 0; s < S; s++) segs[s] = SortSeg{pl[s].key_base, pl[s].n, pl[s].NP, pl[s].part_base, pl[s].first_tile};
    SortSeg* d_segs;
    uint64_t *d_tables, *sorted = nullptr, *start = nullptr, *T = nullptr, *stats;
    uint32_t* status;
    void *sort_scratch, *sizes_scratch;
    CK(tmp.alloc(&d_segs, (size_t)S * sizeof(SortSeg)));
    CK(tmp.alloc(&d_tables, tables.size() * 8));
    if (smode == kShardNone) {
        CK(tmp.alloc(&sorted, n_total * 8));
        CK(tmp.alloc(&start, (NPT + 1) * 8));
    } else {
        sorted = const_cast<uint64_t*>(sc->sorted);
        start = const_cast<uint64_t*>(sc->start);
    }
    if (smode == kShardSearch)
        T = const_cast<uint64_t*>(sc->T);
    else
        CK(tmp.alloc(&T, (NPT + 1) * 8));
    CK(tmp.alloc(&stats, 64));
    CK(tmp.alloc(&status, 64));
    CK(cudaMemsetAsync(status, 0, 64, st));
    CK(h2d(d_segs, segs.data(), S, st));
    CK(h2d(d_tables, tables.data(), tables.size(), st));
    CK(ev.mark(0, st));
    if (smode == kShardNone) {
        CK(tmp.alloc(&sort_scratch, sort_seg_scratch_bytes(n_total, tiles, S, max_np)));
        CK(launch_partition_sort_segs(in, hash_input, kseed, d_segs, S, n_total, tiles, max_np, NPT, sorted, start,
                                      sort_scratch, status, st));
        tmp.release(sort_scratch);
    }
    CK(ev.mark(1, st));
    if (smode == kShardSearch) {
        // the shard's largest n_j and m_j (stats[1], stats[2]) from its own partitions;
        // M from the global offsets
        uint64_t* Tloc;
        const uint64_t np_loc = sc->j1 - sc->j0;
        CK(tmp.alloc(&Tloc, (np_loc + 1) * 8));
        CK(tmp.alloc(&sizes_scratch, sizes_scratch_bytes(np_loc)));
        CK(launch_sizes(start + sc->j0, np_loc, prm.alpha, Tloc, stats, sizes_scratch, st));
        CK(cudaMemcpyAsync(stats, T + NPT, sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
    } else {
        CK(tmp.alloc(&sizes_scratch, sizes_scratch_bytes(NPT)));
        CK(launch_sizes(start, NPT, prm.alpha, T, stats, sizes_scratch, st));
    }
    CK(ev.mark(2, st));
    {  // slot base of every set: T[part_base_s], s = 0..S
        std::vector<uint64_t> idx(S + 1);
        for (uint32_t s = 0; s < S; s++) idx[s] = pl[s].part_base;
        idx[S] = NPT;
        uint64_t *d_idx, *d_out;
        CK(tmp.alloc(&d_idx, (S + 1) * 8));
        CK(tmp.alloc(&d_out, (S + 1) * 8));
        CK(h2d(d_idx, idx.data(), S + 1, st));
        CK(launch_gather_u64(T, d_idx, d_out, S + 1, st));
        CK(d2h(hTb, d_out, S + 1, st));
    }
    CK(d2h(hst, stats, 3, st));
    CK(d2h(hstatus, status, 1, st));
    if (smode == kShardAssemble) CK(d2h(hst + 16, start + NPT, 1, st));
    CK(wait_stream(st));
    if (hstatus[0] == kDevTimeout) return PHOBIC_ERR_TIMEOUT;
    if (smode == kShardAssemble && hst[16] != n_total) return PHOBIC_ERR_INVALID_ARG;  // starts must end at n
    const uint64_t M_total = hst[0], max_n = hst[1], max_m = hst[2];
    if (smode == kShardAssemble && M_total > n_total && !sc->taken) return PHOBIC_ERR_INVALID_ARG;
    for (uint32_t s = 0; s < S; s++) {
        pl[s].g0 = hTb[s];
        pl[s].M = hTb[s + 1] - hTb[s];
    }
    const char* ks = std::getenv("PHOBIC_KEYS_IN_SMEM");
    const bool keys_in_smem = ks && ks[0] == '1';
    // warps per partition: as asked, or (0) chosen from the partition count and
    // lambda.  The build ends with its slowest partitions, and the spread of
    // per-partition search work grows like e^lambda, so 4 warps (testing
    // consecutive candidate ranges of a bucket at once) pay off while there are
    // few waves of partitions per resident one-warp CTA slot (32 per SM), the
    // more so at large lambda; with more waves one warp per partition wastes
    // the fewest issue slots.  Measured (search ms, 1 / 2 / 4 warps): lambda 7,
    // alpha 0.99: 0.084 waves 0.84 / 0.76 / 0.67, 0.15 waves 0.83 / 0.79 / 0.80,
    // 0.25 waves 0.82 / 0.81 / 1.03, 0.5 waves 1.15 / 1.28 / 1.86; lambda 9,
    // alpha 1: 0.3 waves 2.81 / 2.41 / 2.38, 0.84 waves 4.87 / 5.61 / 5.29;
    // lambda 11: 0.84 waves 27.8 / 27.8 / 23.4.  Two warps never win by more
    // than a few percent, so the choice is between one and four.
    uint32_t wpp = prm.warps_per_partition;
    if (wpp == 0) {
        int dev = 0, sms = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const double waves = (double)(smode == kShardSearch ? sc->j1 - sc->j0 : NPT) / ((double)sms * 32.0);
        const double t = 0.15 * std::exp(0.6 * (prm.lambda - 7.0));
        wpp = waves <= t ? 4 : 1;
        // Eight warps from lambda 12, while the partitions fill at most one wave:
        // a bucket then tries so many seeds that eight at a time pay for the
        // CTAs they take.  Measured (search ms, 4 / 8 warps, IC-R, alpha 1):
        // 1e7 keys (0.84 waves) lambda 11: 23.2 / 24.0, 12: 62.3 / 60.9,
        // 13: 169.1 / 157.5, 14: 486 / 437; 1e8 keys (8.4 waves) lambda 14:
        // 3502 / 3684; lambda 7, 1e6 keys: 0.62 / 0.74.
        if (wpp == 4 && prm.lambda >= 12.0 && waves <= 1.0) wpp = 8;
        while (wpp > 1 && search_smem_bytes((uint32_t)max_n, (uint32_t)max_m, cap_B, keys_in_smem, wpp) >
                              search_smem_limit())
            wpp /= 2;
    }
    if (max_m >= 65536 || max_n >= (1u << 31) ||
        search_smem_bytes((uint32_t)max_n, (uint32_t)max_m, cap_B, keys_in_smem, wpp) > search_smem_limit())
        return PHOBIC_ERR_PARTITION_TOO_LARGE;
    // 0: no limit beyond the 32-bit pilot, which the search applies per partition
    const uint32_t s_max = prm.s_max ? prm.s_max : 0xFFFFFFFFu;

    // ---- K3 + K4: bucketing and pilot search, one persistent launch over all sets
    std::vector<SearchSet> ss(S);
    for (uint32_t s = 0; s < S; s++)
        ss[s] = SearchSet{pl[s].part_base, pl[s].NP, pl[s].pilot_base,
                          d_tables + (size_t)pl[s].table_idx * kTablePoints, pl[s].B, 0};
    SearchSet* d_ss;
    uint32_t* pilots;
    uint32_t* taken = nullptr;
    uint64_t* bkeys = nullptr;
    unsigned long long *queue, *work = nullptr;
    if (smode == kShardSearch) {  // partitions j0..j1-1: pilots at column offset j0, starts and offsets from j0
        ss[0].pilot_base = sc->j0;
        pilots = sc->pilots;
        taken = sc->taken;
    } else if (smode == kShardAssemble) {
        pilots = sc->pilots;
        taken = sc->taken;
    } else {
        CK(tmp.alloc(&pilots, pilots_total * 4));
        CK(cudaMemsetAsync(pilots, 0, pilots_total * 4, st));
        if (M_total > n_total) {
            CK(tmp.alloc(&taken, ((M_total + 31) / 32 + 1) * 4));
            CK(cudaMemsetAsync(taken, 0, ((M_total + 31) / 32 + 1) * 4, st));
        }
    }
    CK(tmp.alloc(&d_ss, (size_t)S * sizeof(SearchSet)));
    CK(h2d(d_ss, ss.data(), S, st));
    if (!keys_in_smem && smode != kShardAssemble)
        CK(tmp.alloc(&bkeys, (smode == kShardSearch ? sc->n_local : n_total) * 8));
    CK(tmp.alloc(&queue, 16));
    if (prm.record_timings) {
        CK(tmp.alloc(&work, 16));
        CK(cudaMemsetAsync(work, 0, 16, st));
    }
    SearchLaunch sl;
    sl.sorted = sorted;
    sl.start = smode == kShardSearch ? start + sc->j0 : start;
    sl.T = smode == kShardSearch ? T + sc->j0 : T;
    sl.sets = d_ss;
    sl.nsets = S;
    sl.total_parts = smode == kShardSearch ? sc->j1 - sc->j0 : NPT;
    sl.cap_B = cap_B;
    sl.mode = prm.pilot_mode;
    sl.s_max = s_max;
    sl.s_fast = max_m > 0 ? (uint32_t)std::min<uint64_t>(s_max, 0xFFFFFFFFull / max_m) : s_max;
    sl.cap_n = (uint32_t)max_n;
    sl.cap_m = (uint32_t)max_m;
    sl.bkeys = bkeys;
    sl.keys_in_smem = keys_in_smem ? 1 : 0;
    sl.window_bits = prm.candidate_width == 32 ? 32 : 64;
    sl.warps = wpp;
    sl.pilots = pilots;
    sl.taken_bits = taken;
    sl.status = status;
    sl.work = work;
    sl.queue = queue;
    // schedule: 1 = one CTA per partition, 2 = persistent CTAs over the work queue;
    // 0 (auto) = one CTA per partition, which measured faster for single builds
    // and for batches (the block scheduler balances uneven partitions for free)
    sl.use_queue = prm.search_schedule == 2 ? 1 : 0;
    CK(ev.mark(3, st));
    if (smode != kShardAssemble) CK(launch_search(sl, st));
    CK(ev.mark(4, st));
    if (smode == kShardNone) tmp.release(sorted);
    if (bkeys) tmp.release(bkeys);
    if (smode == kShardSearch) {
        CK(d2h(hstatus, status, 1, st));
        CK(wait_stream(st));
        switch (hstatus[0]) {
            case kDevOk: return PHOBIC_OK;
            case kDevDupHash: return PHOBIC_ERR_DUP_HASH;
            case kDevSearchLimit: return PHOBIC_ERR_SEARCH_LIMIT;
            default: return PHOBIC_ERR_TIMEOUT;
        }
    }

    // ---- K5: offset differences; K6: column maxima (all sets)
    std::vector<OffDesc> od(S);
    for (uint32_t s = 0; s < S; s++) {
        pl[s].Q = (uint64_t)((((unsigned __int128)pl[s].M) << 32) / pl[s].NP);
        od[s] = OffDesc{pl[s].part_base, pl[s].NP, pl[s].Q, 0, 0, 0, 0};
    }
    std::vector<ColDesc> cd(cols_total);
    for (uint32_t s = 0; s < S; s++)
        for (uint32_t b = 0; b < pl[s].B; b++) {
            ColDesc& c = cd[pl[s].col_base + b];
            std::memset(&c, 0, sizeof(c));
            c.src = pl[s].pilot_base + (uint64_t)b * pl[s].NP;
            c.count = pl[s].NP;
        }
    OffDesc* d_od;
    ColDesc* d_cd;
    long long* mm;
    uint32_t* colmax;
    CK(tmp.alloc(&d_od, (size_t)S * sizeof(OffDesc)));
    CK(tmp.alloc(&d_cd, (size_t)cols_total * sizeof(ColDesc)));
    CK(tmp.alloc(&mm, (size_t)S * 16));
    CK(tmp.alloc(&colmax, (size_t)cols_total * 4));
    CK(h2d(d_od, od.data(), S, st));
    CK(h2d(d_cd, cd.data(), cols_total, st));
    CK(ev.mark(5, st));
    CK(launch_offset_minmax(T, d_od, S, mm, st));
    // a mono encoder runs its column encoder over one column per set: the set's
    // physical columns keep their work items and continue one sequence
    const bool mono = prm.encoder >= PHOBIC_ENC_MONO_C;
    const uint32_t enc = mono ? prm.encoder - PHOBIC_ENC_MONO_C : prm.encoder;
    const bool icr = enc == PHOBIC_ENC_IC_R;
    const bool icef = enc == PHOBIC_ENC_IC_EF;
    const bool icmix = enc == PHOBIC_ENC_IC_CR;
    const bool icd = enc == PHOBIC_ENC_IC_D;
    const bool unary = icr || icef || icmix;  // column layouts with a select-sampled unary part
    uint64_t* colsum = nullptr;
    if (unary) CK(tmp.alloc(&colsum, (size_t)cols_total * 8));
    CK(launch_column_max(pilots, d_cd, (uint32_t)cols_total, max_np, colmax, colsum, st));
    CK(d2h(hmm, mm, 2 * (size_t)S, st));
    CK(d2h(hcolmax, colmax, cols_total, st));
    if (unary) CK(d2h(hK, colsum, cols_total, st));
    CK(d2h(hstatus, status, 1, st));
    if (work) CK(d2h(hst + 12, reinterpret_cast<uint64_t*>(work), 2, st));
    CK(wait_stream(st));
    switch (hstatus[0]) {
        case kDevOk: break;
        case kDevDupHash: return PHOBIC_ERR_DUP_HASH;
        case kDevSearchLimit: return PHOBIC_ERR_SEARCH_LIMIT;
        default: return PHOBIC_ERR_TIMEOUT;
    }

    // largest pilot and (Rice, Elias-Fano) pilot sum of each set, for the mono encoders
    std::vector<uint32_t> set_max(S, 0);
    std::vector<uint64_t> set_sum(S, 0);
    if (mono)
        for (uint32_t s = 0; s < S; s++)
            for (uint32_t b = 0; b < pl[s].B; b++) {
                set_max[s] = std::max(set_max[s], hcolmax[pl[s].col_base + b]);
                if (unary) set_sum[s] += hK[pl[s].col_base + b];
            }

    // ---- IC-D: presence bitmaps, ranks, dictionary sizes; one dictionary per
    // column, or (mono-D) one per set whose bitmap all the set's columns mark
    uint64_t *bitmaps = nullptr, *brank = nullptr;
    const uint64_t ndict = icd ? (mono ? S : cols_total) : 0;
    std::vector<uint64_t> bm_begin(ndict + 1, 0);
    std::vector<ColDesc> dd(mono && icd ? S : 0);
    ColDesc* d_dd = nullptr;
    if (icd) {
        if (mono) {
            for (uint32_t s = 0; s < S; s++) {
                std::memset(&dd[s], 0, sizeof(ColDesc));
                dd[s].bm_base = bm_begin[s];
                dd[s].bm_words = ((uint64_t)set_max[s] + 64) / 64;
                bm_begin[s + 1] = bm_begin[s] + dd[s].bm_words;
                for (uint32_t b = 0; b < pl[s].B; b++) {
                    cd[pl[s].col_base + b].bm_base = dd[s].bm_base;
                    cd[pl[s].col_base + b].bm_words = dd[s].bm_words;
                }
            }
            CK(tmp.alloc(&d_dd, (size_t)S * sizeof(ColDesc)));
            CK(h2d(d_dd, dd.data(), S, st));
        } else {
            for (uint64_t c = 0; c < cols_total; c++) {
                cd[c].bm_base = bm_begin[c];
                cd[c].bm_words = ((uint64_t)hcolmax[c] + 64) / 64;
                bm_begin[c + 1] = bm_begin[c] + cd[c].bm_words;
            }
        }
        uint64_t* dK;
        CK(tmp.alloc(&bitmaps, bm_begin[ndict] * 8));
        CK(tmp.alloc(&brank, bm_begin[ndict] * 8));
        CK(tmp.alloc(&dK, ndict * 8));
        CK(h2d(d_cd, cd.data(), cols_total, st));
        CK(cudaMemsetAsync(bitmaps, 0, bm_begin[ndict] * 8, st));
        CK(launch_dict_mark(pilots, d_cd, (uint32_t)cols_total, bitmaps, st));
        CK(launch_dict_rank(mono ? d_dd : d_cd, (uint32_t)ndict, brank, bitmaps, dK, st));
        CK(d2h(hK, dK, ndict, st));
        CK(wait_stream(st));
    }

    // ---- IC-EF: low bits from the column sums (the unary lengths follow from
    // them); mono-EF: one universe per set, the column sums carried as sum0
    if (icef)
        for (uint32_t s = 0; s < S; s++) {
            uint64_t carry = 0;
            for (uint32_t b = 0; b < pl[s].B; b++) {
                ColDesc& c = cd[pl[s].col_base + b];
                const uint64_t N = mono ? (uint64_t)pl[s].B * pl[s].NP : c.count;
                const uint64_t U = (mono ? set_sum[s] : hK[pl[s].col_base + b]) + 1;
                c.width = U >= N ? bitlen64(U / N) - 1 : 0;
                if (mono) {
                    c.idx0 = (uint64_t)b * pl[s].NP;
                    c.sum0 = carry;
                    carry += hK[pl[s].col_base + b];
                }
            }
        }
    // ---- IC-R (and the Rice columns of IC-CR): Rice parameters from the column
    // sums (mono-R: from the set's sum), then the unary lengths; IC-CR's Compact
    // columns take the bit length of their largest pilot
    if (icr || icmix) {
        for (uint32_t s = 0; s < S; s++)
            for (uint32_t b = 0; b < pl[s].B; b++) {
                const uint64_t c = pl[s].col_base + b;
                const bool compact = icmix && b < std::min<uint32_t>(prm.compact_columns, pl[s].B);
                cd[c].width = compact ? bitlen64(hcolmax[c])
                              : mono  ? rice_param(set_sum[s], (uint64_t)pl[s].B * pl[s].NP)
                                      : rice_param(hK[c], cd[c].count);
            }
        uint64_t* dH;
        CK(tmp.alloc(&dH, cols_total * 8));
        CK(h2d(d_cd, cd.data(), cols_total, st));
        CK(launch_rice_unary_len(pilots, d_cd, (uint32_t)cols_total, dH, st));
        CK(d2h(hK, dH, cols_total, st));
        CK(wait_stream(st));
    }

    // ---- layouts and the arena
    uint64_t aw = (uint64_t)ntab * kTablePoints;  // packed tables first
    std::vector<uint64_t> off_begin(S + 1, 0), col_begin(cols_total + 1, 0), remap_sets;
    std::vector<std::vector<uint64_t>> metas(S);
    for (uint32_t s = 0; s < S; s++) {
        SetPlan& p = pl[s];
        p.dmin = hmm[2 * s];
        p.off_w = bitlen64((uint64_t)(hmm[2 * s + 1] - hmm[2 * s]));
        p.n_off = packed_words((p.NP + 1) * (uint64_t)p.off_w);
        p.a_off = aw;
        aw += p.n_off;
        off_begin[s + 1] = off_begin[s] + p.n_off;
        p.n_meta = ((icd || unary) ? 2 : 1) * (mono ? 1 : (uint64_t)p.B);
        p.a_meta = aw;
        aw += p.n_meta;
        metas[s].resize(p.n_meta);
        uint64_t rbase = 0, dbase = 0, bp = icmix ? 32 : 0;  // IC-CR records its c
        const uint64_t ns = (p.NP + 63) / 64;  // IC-R select samples per column
        const uint32_t cmix = icmix ? std::min<uint32_t>(prm.compact_columns, p.B) : 0;
        const uint64_t Nm = (uint64_t)p.B * p.NP;  // a mono encoder's values
        if (mono) {
            // one encoder: column b's values continue at index b N_P, every column
            // with the set's width (Compact), rank width (Dictionary) or parameter
            uint32_t w = 0, dw = 0;
            uint64_t K = 0, Hc = 0;
            if (unary) {
                w = cd[p.col_base].width;
            } else if (icd) {
                K = hK[s];
                w = bitlen64(K - 1);
                dw = bitlen64(set_max[s]);
            } else {
                w = bitlen64(set_max[s]);
            }
            for (uint32_t b = 0; b < p.B; b++) {
                ColDesc& c = cd[p.col_base + b];
                c.width = w;
                c.base = (uint64_t)b * p.NP * w;
                if (unary) {
                    c.hi_base = 0;
                    c.samp_base = 0;
                    c.idx0 = (uint64_t)b * p.NP;
                    if (icr) {  // Rice: sum of pilot >> l over the columns before
                        c.sum0 = Hc;
                        Hc += hK[p.col_base + b];
                    }
                }
                const uint64_t bits = p.NP * (uint64_t)w;
                col_begin[p.col_base + b + 1] =
                    col_begin[p.col_base + b] + (bits ? ((c.base + bits - 1) >> 6) - (c.base >> 6) + 1 : 0);
            }
            rbase = Nm * w;
            metas[s][0] = (uint64_t)w << 56;
            if (unary) {
                dbase = icef ? Nm + (set_sum[s] >> w) + 1 : Nm + Hc;
                // select samples are 32-bit positions in the unary part
                if (dbase > (1ull << 32)) return PHOBIC_ERR_INVALID_ARG;
                metas[s][1] = 0;
                bp = Nm * w + dbase + 32 * ((Nm + 63) / 64) + 64 + 64 + 8;
            } else if (icd) {
                dd[s].dict_width = dw;
                dd[s].dict_base = 0;
                dbase = K * dw;
                metas[s][1] = (uint64_t)dw << 56;
                bp = Nm * w + K * dw + 64 + 64 + 8 + 8;
            } else {
                bp = Nm * w + 64 + 8;
            }
        }
        for (uint32_t b = 0; b < p.B && !mono; b++) {
            ColDesc& c = cd[p.col_base + b];
            const uint64_t c_id = p.col_base + b;
            if (icmix && b < cmix) {
                // a Compact column of the mixture: values in the shared low array
                c.base = rbase;
                c.hi_base = dbase;
                c.samp_base = 0;
                metas[s][2 * b] = rbase | ((uint64_t)c.width << 56);
                metas[s][2 * b + 1] = dbase;
                rbase += p.NP * (uint64_t)c.width;
                bp += p.NP * (uint64_t)c.width + 64 + 8;
            } else if (unary) {
                // c.width = Rice parameter / Elias-Fano low bits (set above); dbase counts
                // unary bits: IC-R N_P + sum (v >> l); IC-EF N_P + (E_last >> l) + 1
                const uint64_t H = icef ? p.NP + (hK[c_id] >> c.width) + 1 : p.NP + hK[c_id];
                c.base = rbase;
                c.hi_base = dbase;
                c.samp_base = (uint64_t)(b - cmix) * ns;
                metas[s][2 * b] = rbase | ((uint64_t)c.width << 56);
                metas[s][2 * b + 1] = dbase;
                rbase += p.NP * (uint64_t)c.width;
                dbase += H;
                bp += p.NP * (uint64_t)c.width + H + 32 * ns + 64 + 64 + 8;
            } else if (!icd) {
                c.width = bitlen64(hcolmax[c_id]);
                c.base = rbase;
                metas[s][b] = rbase | ((uint64_t)c.width << 56);
                rbase += p.NP * (uint64_t)c.width;
                bp += p.NP * (uint64_t)c.width + 64 + 8;
            } else {
                const uint64_t K = hK[c_id];
                c.width = bitlen64(K - 1);
                c.dict_width = bitlen64(hcolmax[c_id]);
                c.base = rbase;
                c.dict_base = dbase;
                metas[s][2 * b] = rbase | ((uint64_t)c.width << 56);
                metas[s][2 * b + 1] = dbase | ((uint64_t)c.dict_width << 56);
                rbase += p.NP * (uint64_t)c.width;
                dbase += K * (uint64_t)c.dict_width;
                bp += p.NP * (uint64_t)c.width + K * (uint64_t)c.dict_width + 64 + 64 + 8 + 8;
            }
            const uint64_t bits = p.NP * (uint64_t)c.width;
            col_begin[c_id + 1] = col_begin[c_id] + (bits ? ((c.base + bits - 1) >> 6) - (c.base >> 6) + 1 : 0);
        }
        p.n_pil = packed_words(rbase);
        p.a_pil = aw;
        aw += p.n_pil;
        p.samp_words = !unary ? 0 : mono ? ((Nm + 63) / 64 + 1) / 2 : ((uint64_t)(p.B - cmix) * ns + 1) / 2;
        p.mix_c = cmix;
        p.n_dict = icd ? packed_words(dbase) : unary ? p.samp_words + packed_words(dbase) : 0;
        p.a_dict = aw;
        aw += p.n_dict;
        for (uint32_t b = 0; b < p.B; b++) {
            cd[p.col_base + b].dst_word = p.a_pil;
            cd[p.col_base + b].dict_dst_word = p.a_dict;
            cd[p.col_base + b].samp_dst_word = (icmix && b < cmix) ? ~0ull : p.a_dict;
            cd[p.col_base + b].hi_dst_word = p.a_dict + p.samp_words;
        }
        if (mono && icd) dd[s].dict_dst_word = p.a_dict;
        // Elias-Fano remap of slots >= n
        const uint64_t N = p.M - p.n;
        if (N) {
            p.ef_l = (p.n / N >= 1) ? bitlen64(p.n / N) - 1 : 0;
            p.n_low = packed_words(N * (uint64_t)p.ef_l);
            p.n_high = packed_words(N + (p.n >> p.ef_l) + 1);
            p.n_samp = (N + 63) / 64;
            p.a_low = aw;
            aw += p.n_low;
            p.a_high = aw;
            aw += p.n_high;
            p.a_samp = aw;
            aw += p.n_samp;
            remap_sets.push_back(s);
        }
        if (prm.keep_pilots) {
            p.a_pilots = aw;
            aw += ((uint64_t)p.B * p.NP + 1) / 2;
        }
        // space accounting (fixed spec)
        p.bits_header = 9 * 64;
        p.bits_offsets = (p.NP + 1) * (uint64_t)p.off_w + 64 + 64 + 8;
        p.bits_pilots = bp;
        p.bits_remap = N ? N * (uint64_t)p.ef_l + (N + (p.n >> p.ef_l) + 1) + 64 * ((N + 63) / 64) + 3 * 64 : 0;
        p.bits_total = p.bits_header + p.bits_offsets + p.bits_pilots + p.bits_remap;
        od[s].dmin = p.dmin;
        od[s].width = p.off_w;
        od[s].dst_word = p.a_off;
    }
    SharedMem* mem = new (std::nothrow) SharedMem();
    if (!mem) return PHOBIC_ERR_OOM;
    {
        cudaError_t e = cudaMallocAsync(&mem->ptr, aw * 8, st);
        if (e != cudaSuccess) {
            delete mem;
            return from_cuda(e);
        }
        mem->bytes = aw * 8;
        mem->pooled = true;
    }
    struct MemGuard {
        SharedMem*& m;
        cudaStream_t st;
        ~MemGuard() {
            if (m) {
                cudaFreeAsync(m->ptr, st);
                delete m;
            }
        }
    } mem_guard{mem, st};
    uint64_t* arena = static_cast<uint64_t*>(mem->ptr);
    CK(cudaMemsetAsync(arena, 0, aw * 8, st));
    CK(h2d(arena, tables.data(), tables.size(), st));
    for (uint32_t s = 0; s < S; s++) CK(h2d(arena + pl[s].a_meta, metas[s].data(), metas[s].size(), st));

    // ---- K5 / K6 packing (all sets, one launch each)
    uint64_t *d_obeg, *d_cbeg;
    CK(tmp.alloc(&d_obeg, (S + 1) * 8));
    CK(tmp.alloc(&d_cbeg, (cols_total + 1) * 8));
    CK(h2d(d_od, od.data(), S, st));
    CK(h2d(d_cd, cd.data(), cols_total, st));
    CK(h2d(d_obeg, off_begin.data(), S + 1, st));
    CK(h2d(d_cbeg, col_begin.data(), cols_total + 1, st));
    CK(launch_offset_pack(T, d_od, S, d_obeg, off_begin[S], arena, st));
    if (!icef)  // IC-C values, IC-D ranks, IC-R low parts
        CK(launch_pack_columns(pilots, d_cd, (uint32_t)cols_total, d_cbeg, col_begin[cols_total], icd, bitmaps,
                               brank, arena, st));
    if (icr || icmix) CK(launch_rice_unary(pilots, d_cd, (uint32_t)cols_total, arena, st));
    if (icef) CK(launch_ef_columns(pilots, d_cd, (uint32_t)cols_total, arena, st));
    if (icd) {
        uint64_t* d_bmbeg;
        CK(tmp.alloc(&d_bmbeg, (ndict + 1) * 8));
        CK(h2d(d_bmbeg, bm_begin.data(), ndict + 1, st));
        if (mono) CK(h2d(d_dd, dd.data(), S, st));
        CK(launch_dict_pack_values(mono ? d_dd : d_cd, (uint32_t)ndict, d_bmbeg, bm_begin[ndict], bitmaps, brank,
                                   arena, st));
    }
    CK(ev.mark(6, st));

    // ---- K7: Elias-Fano remap of slots >= n (sets with alpha < 1)
    if (!remap_sets.empty()) {
        const uint32_t R = (uint32_t)remap_sets.size();
        std::vector<RemapDesc> rd(R);
        std::vector<uint64_t> zb(R + 1, 0), tb(R + 1, 0), fb(R + 1, 0), lb(R + 1, 0);
        for (uint32_t r = 0; r < R; r++) {
            const SetPlan& p = pl[remap_sets[r]];
            rd[r] = RemapDesc{p.g0, p.n, p.M, fb[r], p.a_low, p.a_high, p.a_samp, p.ef_l, 0};
            zb[r + 1] = zb[r] + (((p.g0 + p.n - 1) >> 5) - (p.g0 >> 5) + 1);
            tb[r + 1] = tb[r] + (((p.g0 + p.M - 1) >> 5) - ((p.g0 + p.n) >> 5) + 1);
            fb[r + 1] = fb[r] + (p.M - p.n);
            lb[r + 1] = lb[r] + p.n_low;
        }
        RemapDesc* d_rd;
        uint64_t* d_beg;
        void* rs;
        CK(tmp.alloc(&d_rd, (size_t)R * sizeof(RemapDesc)));
        CK(tmp.alloc(&d_beg, 4 * (size_t)(R + 1) * 8));
        CK(tmp.alloc(&rs, remap_scratch_bytes(zb[R], tb[R], fb[R])));
        CK(h2d(d_rd, rd.data(), R, st));
        CK(h2d(d_beg, zb.data(), R + 1, st));
        CK(h2d(d_beg + (R + 1), tb.data(), R + 1, st));
        CK(h2d(d_beg + 2 * (R + 1), fb.data(), R + 1, st));
        CK(h2d(d_beg + 3 * (R + 1), lb.data(), R + 1, st));
        CK(launch_remap(taken, d_rd, R, d_beg, zb[R], d_beg + (R + 1), tb[R], d_beg + 2 * (R + 1), fb[R],
                        d_beg + 3 * (R + 1), lb[R], arena, rs, st));
    }
    CK(ev.mark(7, st));
    if (prm.keep_pilots)
        for (uint32_t s = 0; s < S; s++)
            CK(cudaMemcpyAsync(arena + pl[s].a_pilots, pilots + pl[s].pilot_base, (uint64_t)pl[s].B * pl[s].NP * 4,
                               cudaMemcpyDeviceToDevice, st));
    CK(wait_stream(st));
    CK(cudaGetLastError());

    // ---- handles
    std::vector<phobic_handle*> hs(S, nullptr);
    for (uint32_t s = 0; s < S; s++) {
        hs[s] = new (std::nothrow) phobic_handle();
        if (!hs[s]) {
            for (auto* h : hs) delete h;
            return PHOBIC_ERR_OOM;
        }
    }
    mem->refs.store((int)S);
    for (uint32_t s = 0; s < S; s++) {
        const SetPlan& p = pl[s];
        phobic_handle* h = hs[s];
        h->prm = prm;
        h->prm.partition_size = p.P;
        h->prm.s_max = s_max;
        h->mem = mem;
        h->table = arena + (size_t)p.table_idx * kTablePoints;
        h->off_words = arena + p.a_off;
        h->n_off_words = p.n_off;
        h->col_meta = arena + p.a_meta;
        h->n_col_meta = p.n_meta;
        h->pil_words = arena + p.a_pil;
        h->n_pil_words = p.n_pil;
        h->dict_words = p.n_dict ? arena + p.a_dict : nullptr;
        h->n_dict_words = p.n_dict;
        if (p.M > p.n) {
            h->ef_low = arena + p.a_low;
            h->ef_high = arena + p.a_high;
            h->ef_samples = arena + p.a_samp;
            h->n_ef_low = p.n_low;
            h->n_ef_high = p.n_high;
            h->n_ef_samples = p.n_samp;
        }
        if (prm.keep_pilots) h->pilots = reinterpret_cast<uint32_t*>(arena + p.a_pilots);
        phobic_info& I = h->info;
        std::memset(&I, 0, sizeof(I));
        I.n = p.n;
        I.M = p.M;
        I.num_partitions = p.NP;
        I.num_buckets = p.B;
        I.partition_size = p.P;
        I.lambda = prm.lambda;
        I.alpha = prm.alpha;
        I.epsilon = p.eps;
        I.encoder = prm.encoder;
        I.pilot_mode = prm.pilot_mode;
        I.seed = prm.seed;
        I.bucket_function = prm.bucket_function;
        I.compact_columns = p.mix_c;
        I.max_partition = max_n;
        I.bits_header = p.bits_header;
        I.bits_offsets = p.bits_offsets;
        I.bits_pilots = p.bits_pilots;
        I.bits_remap = p.bits_remap;
        I.bits_total = p.bits_total;
        I.device_bytes = 8 * (kTablePoints + p.n_off + p.n_meta + p.n_pil + p.n_dict + p.n_low + p.n_high +
                              p.n_samp) + (prm.keep_pilots ? (uint64_t)p.B * p.NP * 4 : 0);
        QueryView& v = h->view;
        v.n = p.n;
        v.M = p.M;
        v.NP = p.NP;
        v.B = p.B;
        v.encoder = prm.encoder;
        v.pilot_mode = prm.pilot_mode;
        v.off_w = p.off_w;
        v.kseed = kseed;
        v.off_Q = p.Q;
        v.off_dmin = p.dmin;
        v.table = h->table;
        v.off_words = h->off_words;
        v.col_meta = h->col_meta;
        v.pil_words = h->pil_words;
        v.dict_words = h->dict_words;
        v.ef_N = p.M - p.n;
        v.ef_l = p.ef_l;
        v.ef_low = h->ef_low;
        v.ef_high = h->ef_high;
        v.ef_samples = h->ef_samples;
        v.rice_high = unary ? arena + p.a_dict + p.samp_words : nullptr;
        v.rice_ns = unary ? (uint32_t)((p.NP + 63) / 64) : 0;
        v.mix_c = p.mix_c;
        v.small_bits = (h->n_pil_words < (1ull << 26) && h->n_dict_words < (1ull << 26)) ? 1 : 0;
        v.key_kind = key_kind;
        v.string_seed = prm.seed;
        if (ev.on) {
            h->has_timings = true;
            h->timings.sort_ms = ev.between(0, 1);
            h->timings.sizes_ms = ev.between(1, 2);
            h->timings.search_ms = ev.between(3, 4);
            h->timings.encode_ms = ev.between(5, 6);
            h->timings.remap_ms = ev.between(6, 7);
            h->timings.total_ms = ev.between(0, 7);
            h->timings.search_s_tries = hst[12];
            h->timings.search_steps = hst[13];
        }
    }
    mem = nullptr;  // the handles own it now
    *out = hs;
    return PHOBIC_OK;
}

phobic_status build_impl(const uint64_t* in, int hash_input, uint64_t n, const phobic_params& prm, cudaStream_t st,
                         phobic_handle** out, uint32_t key_kind = 0) {
    std::vector<phobic_handle*> hs;
    phobic_status s = build_sets(in, hash_input, {SetIn{0, n, prm.partition_size}}, prm, st, key_kind, &hs);
    if (s == PHOBIC_OK) *out = hs[0];
    return s;
}

}  // namespace

extern "C" {

void phobic_params_init(phobic_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->lambda = 7.0;
    p->alpha = 1.0;
    p->partition_size = 2500;
    p->encoder = PHOBIC_ENC_IC_C;
    p->pilot_mode = PHOBIC_PILOT_ADDITIVE;
    p->s_max = 0;
    p->seed = 0;
}

phobic_status phobic_build_ex(const uint64_t* d_keys, uint64_t n, const phobic_params* params, phobic_stream_t stream,
                              phobic_handle** out) {
    if (!out) return PHOBIC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!d_keys || !params) return PHOBIC_ERR_INVALID_ARG;
    phobic_status s = check_params(n, *params);
    if (s != PHOBIC_OK) return s;
    return build_impl(d_keys, 1, n, *params, (cudaStream_t)stream, out);
}

phobic_status phobic_build(const uint64_t* d_keys, uint64_t n, double lambda, double alpha, uint32_t partition_size,
                           uint64_t seed, phobic_stream_t stream, phobic_handle** out) {
    phobic_params p;
    phobic_params_init(&p);
    p.lambda = lambda;
    p.alpha = alpha;
    p.partition_size = partition_size;
    p.seed = seed;
    return phobic_build_ex(d_keys, n, &p, stream, out);
}

phobic_status phobic_build_batch(const uint64_t* d_keys, const uint64_t* h_set_offsets, uint32_t n_sets,
                                 const uint32_t* h_partition_sizes, const phobic_params* params,
                                 phobic_stream_t stream, phobic_handle** out_handles) {
    if (!out_handles || n_sets == 0) return PHOBIC_ERR_INVALID_ARG;
    for (uint32_t s = 0; s < n_sets; s++) out_handles[s] = nullptr;
    if (!d_keys || !h_set_offsets || !params) return PHOBIC_ERR_INVALID_ARG;
    std::vector<SetIn> sets(n_sets);
    for (uint32_t s = 0; s < n_sets; s++) {
        if (h_set_offsets[s + 1] <= h_set_offsets[s]) return PHOBIC_ERR_INVALID_ARG;  // every set non-empty
        phobic_params p = *params;
        if (h_partition_sizes) p.partition_size = h_partition_sizes[s];
        phobic_status st = check_params(h_set_offsets[s + 1] - h_set_offsets[s], p);
        if (st != PHOBIC_OK) return st;
        sets[s] = SetIn{h_set_offsets[s], h_set_offsets[s + 1] - h_set_offsets[s], p.partition_size};
    }
    std::vector<phobic_handle*> hs;
    phobic_status st = build_sets(d_keys + h_set_offsets[0], 1, [&] {
        for (auto& x : sets) x.key_base -= h_set_offsets[0];
        return sets;
    }(), *params, (cudaStream_t)stream, 0, &hs);
    if (st != PHOBIC_OK) return st;
    for (uint32_t s = 0; s < n_sets; s++) out_handles[s] = hs[s];
    return PHOBIC_OK;
}

phobic_status phobic_build_host(const uint64_t* h_keys, uint64_t n, const phobic_params* params,
                                phobic_stream_t stream, phobic_handle** out) {
    if (!out) return PHOBIC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!h_keys || !params) return PHOBIC_ERR_INVALID_ARG;
    phobic_status s = check_params(n, *params);
    if (s != PHOBIC_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    ensure_pool();
    uint64_t* d = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&d, n * 8, st);
    if (e != cudaSuccess) return from_cuda(e);
    e = cudaMemcpyAsync(d, h_keys, n * 8, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
        cudaFreeAsync(d, st);
        return from_cuda(e);
    }
    s = build_impl(d, 1, n, *params, st, out);
    cudaFreeAsync(d, st);
    return s;
}

phobic_status phobic_table_offsets(const uint64_t* d_start, uint64_t num_partitions, double alpha, uint64_t* d_T,
                                   uint64_t* h_stats, phobic_stream_t stream) {
    if (!d_start || !d_T || num_partitions == 0 || !(alpha > 0.0) || alpha > 1.0) return PHOBIC_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    ensure_pool();
    Arena tmp(st);
    uint64_t* stats;
    void* scratch;
    CK(tmp.alloc(&stats, 64));
    CK(tmp.alloc(&scratch, sizes_scratch_bytes(num_partitions)));
    CK(launch_sizes(d_start, num_partitions, alpha, d_T, stats, scratch, st));
    uint64_t hs[3];
    CK(d2h(hs, stats, 3, st));
    CK(wait_stream(st));
    CK(cudaGetLastError());
    if (h_stats) std::memcpy(h_stats, hs, sizeof(hs));
    return PHOBIC_OK;
}

phobic_status phobic_search_partitions(const uint64_t* d_sorted, uint64_t n_local, const uint64_t* d_start,
                                       const uint64_t* d_T, uint64_t n, uint64_t num_partitions, uint64_t j0,
                                       uint64_t j1, const phobic_params* params, uint32_t* d_pilots, uint32_t* d_taken,
                                       phobic_stream_t stream) {
    if (!params || !d_start || !d_T || !d_pilots) return PHOBIC_ERR_INVALID_ARG;
    phobic_status s = check_params(n, *params);
    if (s != PHOBIC_OK) return s;
    if (num_partitions != num_partitions_of(n, params->partition_size) || j0 > j1 || j1 > num_partitions)
        return PHOBIC_ERR_INVALID_ARG;
    if (j0 == j1) return PHOBIC_OK;
    if (!d_sorted && n_local) return PHOBIC_ERR_INVALID_ARG;
    ShardCtl sc{kShardSearch, d_sorted, n_local, d_start, d_T, j0, j1, d_pilots, d_taken};
    std::vector<phobic_handle*> hs;
    return build_sets(nullptr, 0, {SetIn{0, n, params->partition_size}}, *params,
                      reinterpret_cast<cudaStream_t>(stream), 0, &hs, &sc);
}

phobic_status phobic_assemble(const uint64_t* d_start, uint64_t n, const uint32_t* d_pilots, const uint32_t* d_taken,
                              const phobic_params* params, phobic_stream_t stream, phobic_handle** out) {
    if (!out) return PHOBIC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!params || !d_start || !d_pilots) return PHOBIC_ERR_INVALID_ARG;
    phobic_status s = check_params(n, *params);
    if (s != PHOBIC_OK) return s;
    ShardCtl sc{kShardAssemble, nullptr, 0, d_start, nullptr, 0, 0, const_cast<uint32_t*>(d_pilots),
                const_cast<uint32_t*>(d_taken)};
    std::vector<phobic_handle*> hs;
    s = build_sets(nullptr, 0, {SetIn{0, n, params->partition_size}}, *params, reinterpret_cast<cudaStream_t>(stream), 0,
                   &hs, &sc);
    if (s == PHOBIC_OK) *out = hs[0];
    return s;
}

phobic_status phobic_query(const phobic_handle* h, const uint64_t* d_keys, uint64_t* d_out, uint64_t m,
                           phobic_stream_t stream) {
    if (!h || h->view.key_kind != 0) return PHOBIC_ERR_INVALID_ARG;
    if (m == 0) return PHOBIC_OK;
    if (!d_keys || !d_out) return PHOBIC_ERR_INVALID_ARG;
    return from_cuda(launch_query(h->view, d_keys, d_out, m, (cudaStream_t)stream));
}

phobic_status phobic_query_multi(const phobic_handle* const* handles, const uint64_t* const* d_keys,
                                 uint64_t* const* d_outs, const uint64_t* counts, uint32_t n_req,
                                 phobic_stream_t stream) {
    if (n_req == 0) return PHOBIC_OK;
    if (!handles || !d_keys || !d_outs || !counts) return PHOBIC_ERR_INVALID_ARG;
    std::vector<MultiQuery> reqs;
    reqs.reserve(n_req);
    uint64_t total = 0;
    for (uint32_t r = 0; r < n_req; r++) {
        const phobic_handle* h = handles[r];
        if (!h || h->view.key_kind != 0) return PHOBIC_ERR_INVALID_ARG;
        if (counts[r] == 0) continue;
        if (!d_keys[r] || !d_outs[r]) return PHOBIC_ERR_INVALID_ARG;
        reqs.push_back(MultiQuery{h->view, d_keys[r], d_outs[r], total});
        total += counts[r];
    }
    if (reqs.empty()) return PHOBIC_OK;
    cudaStream_t st = (cudaStream_t)stream;
    MultiQuery* d = nullptr;
    const size_t bytes = reqs.size() * sizeof(MultiQuery);
    cudaError_t e = cudaMallocAsync(&d, bytes, st);
    if (e != cudaSuccess) return from_cuda(e);
    // from pageable memory: returns once the descriptors are staged
    e = cudaMemcpyAsync(d, reqs.data(), bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_query_multi(d, (uint32_t)reqs.size(), total, st);
    cudaError_t e2 = cudaFreeAsync(d, st);
    return from_cuda(e != cudaSuccess ? e : e2);
}

}  // extern "C"

namespace {
// Per host thread: the second stream and the events of the chunked host query.
struct QueryPipe {
    cudaStream_t out = nullptr;
    cudaEvent_t queried[3] = {}, copied[3] = {};
    bool ok = false;
    QueryPipe() {
        ok = cudaStreamCreateWithFlags(&out, cudaStreamNonBlocking) == cudaSuccess;
        for (int i = 0; i < 3 && ok; i++)
            ok = cudaEventCreateWithFlags(&queried[i], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&copied[i], cudaEventDisableTiming) == cudaSuccess;
    }
};
}  // namespace

extern "C" {

// Chunks of keys go in on `stream`, are queried there, and their results go
// out on a second stream, through three device slots: the copy of chunk c+1 in,
// the query of chunk c and the copy of chunk c-1 out overlap (the two
// directions use separate copy engines).
phobic_status phobic_query_host(const phobic_handle* h, const uint64_t* h_keys, uint64_t* h_out, uint64_t m,
                                phobic_stream_t stream) {
    if (!h || h->view.key_kind != 0) return PHOBIC_ERR_INVALID_ARG;
    if (m == 0) return PHOBIC_OK;
    if (!h_keys || !h_out) return PHOBIC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    ensure_pool();
    constexpr uint64_t kChunk = 1ull << 22;
    thread_local QueryPipe pipe;
    const uint64_t slots = m <= kChunk ? 1 : 3;
    const uint64_t cap = m <= kChunk ? m : kChunk;
    if (slots > 1 && !pipe.ok) return PHOBIC_ERR_CUDA;
    uint64_t* d = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&d, slots * cap * 16, st);
    if (e != cudaSuccess) return from_cuda(e);
    if (slots == 1) {
        e = cudaMemcpyAsync(d, h_keys, m * 8, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = launch_query(h->view, d, d + m, m, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_out, d + m, m * 8, cudaMemcpyDeviceToHost, st);
    } else {
        // the out stream must not run ahead of the allocation on `stream`
        e = cudaEventRecord(pipe.queried[0], st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(pipe.out, pipe.queried[0], 0);
        for (uint64_t c = 0, at = 0; at < m && e == cudaSuccess; c++, at += kChunk) {
            const uint64_t len = m - at < kChunk ? m - at : kChunk;
            const uint64_t slot = c % 3;
            uint64_t* din = d + slot * cap * 2;
            uint64_t* dout = din + cap;
            if (c >= 3) e = cudaStreamWaitEvent(st, pipe.copied[slot], 0);  // the slot's last results are out
            if (e == cudaSuccess) e = cudaMemcpyAsync(din, h_keys + at, len * 8, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = launch_query(h->view, din, dout, len, st);
            if (e == cudaSuccess) e = cudaEventRecord(pipe.queried[slot], st);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(pipe.out, pipe.queried[slot], 0);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(h_out + at, dout, len * 8, cudaMemcpyDeviceToHost, pipe.out);
            if (e == cudaSuccess) e = cudaEventRecord(pipe.copied[slot], pipe.out);
        }
        // the buffer is freed on `stream` after the last copy out
        for (int i = 0; i < 3 && e == cudaSuccess; i++) e = cudaStreamWaitEvent(st, pipe.copied[i], 0);
    }
    const cudaError_t e2 = cudaFreeAsync(d, st);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return from_cuda(e);
}

double phobic_bits_per_key(const phobic_handle* h) {
    if (!h || h->info.n == 0) return std::nan("");
    return (double)h->info.bits_total / (double)h->info.n;
}

phobic_status phobic_get_info(const phobic_handle* h, phobic_info* info) {
    if (!h || !info) return PHOBIC_ERR_INVALID_ARG;
    *info = h->info;
    return PHOBIC_OK;
}

phobic_status phobic_copy_pilots(const phobic_handle* h, uint32_t* d_out, phobic_stream_t stream) {
    if (!h || !d_out || !h->pilots) return PHOBIC_ERR_INVALID_ARG;
    return from_cuda(cudaMemcpyAsync(d_out, h->pilots, (uint64_t)h->info.num_buckets * h->info.num_partitions * 4,
                                     cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
}

phobic_status phobic_get_timings(const phobic_handle* h, phobic_timings* t) {
    if (!h || !t || !h->has_timings) return PHOBIC_ERR_INVALID_ARG;
    *t = h->timings;
    return PHOBIC_OK;
}

uint64_t phobic_kernel_launches(void) { return phobic::g_launches.load(); }

}  // extern "C"

namespace phobic {
const QueryView* handle_view(const phobic_handle* h) { return h ? &h->view : nullptr; }
}  // namespace phobic

extern "C" {

phobic_status phobic_trim(uint64_t keep_bytes) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PHOBIC_ERR_CUDA;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return PHOBIC_ERR_CUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return PHOBIC_ERR_CUDA;
    return cudaMemPoolTrimTo(pool, (size_t)keep_bytes) == cudaSuccess ? PHOBIC_OK : PHOBIC_ERR_CUDA;
}

phobic_status phobic_pool_bytes(uint64_t* reserved, uint64_t* used) {
    if (!reserved || !used) return PHOBIC_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PHOBIC_ERR_CUDA;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return PHOBIC_ERR_CUDA;
    uint64_t r = 0, u = 0;
    if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &r) != cudaSuccess ||
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &u) != cudaSuccess)
        return PHOBIC_ERR_CUDA;
    *reserved = r;
    *used = u;
    return PHOBIC_OK;
}

void phobic_free(phobic_handle* h) { handle_destroy(h); }

const char* phobic_status_str(phobic_status s) {
    switch (s) {
        case PHOBIC_OK: return "ok";
        case PHOBIC_ERR_INVALID_ARG: return "invalid argument";
        case PHOBIC_ERR_OOM: return "out of memory";
        case PHOBIC_ERR_DUP_HASH: return "duplicate master hash (duplicate keys)";
        case PHOBIC_ERR_SEARCH_LIMIT: return "pilot search limit reached";
        case PHOBIC_ERR_PARTITION_TOO_LARGE: return "partition too large for the search kernel";
        case PHOBIC_ERR_CUDA: return "CUDA error";
        case PHOBIC_ERR_TIMEOUT: return "device wait timed out";
        case PHOBIC_ERR_FORMAT: return "malformed serialized structure";
    }
    return "unknown status";
}

// ---------------------------------------------------------- serialization ---
// Layout (u64 words): magic, version, n, M, NP, B, P, lambda bits, alpha bits,
// seed, encoder, pilot_mode, off_w, off_Q, off_dmin, ef_l, then the word counts
// of off_words, col_meta, pil_words, dict_words, ef_low, ef_high, ef_samples,
// then bits_header..bits_total (5), then the arrays in that order.
static const int kHeaderWords = 16 + 7 + 5;

phobic_status phobic_export(const phobic_handle* h, void* h_buf, size_t* len) {
    if (!h || !len) return PHOBIC_ERR_INVALID_ARG;
    const uint64_t counts[7] = {h->n_off_words, h->n_col_meta, h->n_pil_words, h->n_dict_words,
                                h->n_ef_low,    h->n_ef_high,  h->n_ef_samples};
    const uint64_t* arrays[7] = {h->off_words, h->col_meta, h->pil_words, h->dict_words,
                                 h->ef_low,    h->ef_high,  h->ef_samples};
    uint64_t words = kHeaderWords;
    for (int i = 0; i < 7; i++) words += counts[i];
    const size_t need = words * 8;
    if (!h_buf) {
        *len = need;
        return PHOBIC_OK;
    }
    if (*len < need) return PHOBIC_ERR_INVALID_ARG;
    uint64_t* o = static_cast<uint64_t*>(h_buf);
    const phobic_info& I = h->info;
    uint64_t lam, alp;
    std::memcpy(&lam, &I.lambda, 8);
    std::memcpy(&alp, &I.alpha, 8);
    uint64_t hdr[kHeaderWords] = {kMagic, kFormatVersion, I.n, I.M, I.num_partitions, I.num_buckets,
                                  I.partition_size, lam, alp, I.seed,
                                  (uint64_t)I.encoder | ((uint64_t)I.bucket_function << 32) |
                                      ((uint64_t)I.compact_columns << 40),
                                  (uint64_t)I.pilot_mode | ((uint64_t)h->view.key_kind << 32), h->view.off_w,
                                  h->view.off_Q, (uint64_t)h->view.off_dmin, h->view.ef_l};
    for (int i = 0; i < 7; i++) hdr[16 + i] = counts[i];
    hdr[23] = I.bits_header;
    hdr[24] = I.bits_offsets;
    hdr[25] = I.bits_pilots;
    hdr[26] = I.bits_remap;
    hdr[27] = I.bits_total;
    std::memcpy(o, hdr, sizeof(hdr));
    uint64_t at = kHeaderWords;
    for (int i = 0; i < 7; i++) {
        if (counts[i]) {
            cudaError_t e = cudaMemcpy(o + at, arrays[i], counts[i] * 8, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return from_cuda(e);
        }
        at += counts[i];
    }
    *len = need;
    return PHOBIC_OK;
}

// Host-side validation of phobic_export bytes: every check that the device
// copies and the query kernels rely on (sizes, metadata inside their arrays,
// unary regions and select samples).  Fills the parsed parameters and counts.
struct ParsedExport {
    phobic_params p;
    uint64_t n, M, NP, B;
    uint32_t key_kind;
    uint64_t counts[7];
    uint64_t words;
    uint64_t cmix, rice_sw;
    bool unary_enc;
};

// width <= 64 bits at bit o of a packed array; the caller keeps o + width within
// the array's bits and the array ends with a padding word
static uint64_t host_bits(const uint64_t* words, uint64_t o, uint32_t width) {
    if (width == 0) return 0;
    const uint64_t i = o >> 6;
    const uint32_t sh = (uint32_t)(o & 63);
    uint64_t v = words[i] >> sh;
    if (sh + width > 64) v |= words[i + 1] << (64 - sh);
    return width == 64 ? v : (v & ((1ull << width) - 1));
}

static phobic_status parse_export(const void* h_buf, size_t len, ParsedExport* pe) {
    if (!h_buf || len < kHeaderWords * 8 || (len & 7)) return PHOBIC_ERR_FORMAT;
    const uint64_t* w = static_cast<const uint64_t*>(h_buf);
    if (w[0] != kMagic || w[1] != kFormatVersion) return PHOBIC_ERR_FORMAT;
    phobic_params& p = pe->p;
    phobic_params_init(&p);
    const uint64_t n = w[2], M = w[3], NP = w[4], B = w[5], P = w[6];
    std::memcpy(&p.lambda, &w[7], 8);
    std::memcpy(&p.alpha, &w[8], 8);
    p.partition_size = (uint32_t)P;
    p.seed = w[9];
    p.encoder = (uint32_t)w[10];
    p.bucket_function = (uint32_t)((w[10] >> 32) & 0xFF);
    p.compact_columns = (uint32_t)(w[10] >> 40);
    p.pilot_mode = (uint32_t)w[11];
    const uint32_t key_kind = (uint32_t)(w[11] >> 32);
    if (key_kind > 1) return PHOBIC_ERR_FORMAT;
    if (P != p.partition_size || check_params(n, p) != PHOBIC_OK) return PHOBIC_ERR_FORMAT;
    if (NP != num_partitions(n, p.partition_size) || B != num_buckets(p.lambda, p.partition_size) || M < n)
        return PHOBIC_ERR_FORMAT;
    uint64_t* counts = pe->counts;
    uint64_t words = kHeaderWords;
    for (int i = 0; i < 7; i++) {
        counts[i] = w[16 + i];
        if (counts[i] > (len / 8)) return PHOBIC_ERR_FORMAT;
        words += counts[i];
    }
    if (words * 8 != len) return PHOBIC_ERR_FORMAT;
    const uint64_t off_w = w[12];
    if (off_w > 64 || w[15] > 63) return PHOBIC_ERR_FORMAT;
    if (counts[0] < packed_words((NP + 1) * off_w)) return PHOBIC_ERR_FORMAT;
    // offsets: T_j = floor(j Q / 2^32) + dmin + D_j runs from 0 to M without
    // decreasing, every partition's table below 2^16 slots (as the search
    // requires), so that a query's slot always lies in [0, M)
    // (width 0: every D_j = 0, so T_j = floor(j Q / 2^32) + dmin is checked in
    // closed form; otherwise the N_P + 1 stored values, which the file holds)
    if (off_w == 0) {
        const uint64_t Q = w[13];
        const uint64_t step = (Q >> 32) + ((Q & 0xFFFFFFFFull) ? 1 : 0);  // largest T_{j+1} - T_j
        if (w[14] != 0 || step >= 65536 || (uint64_t)(((unsigned __int128)NP * Q) >> 32) != M)
            return PHOBIC_ERR_FORMAT;
    } else {
        const uint64_t* ow = w + kHeaderWords;
        uint64_t prev = 0;
        for (uint64_t j = 0; j <= NP; j++) {
            const uint64_t T = (uint64_t)(((unsigned __int128)j * w[13]) >> 32) + w[14] +
                               host_bits(ow, j * off_w, (uint32_t)off_w);
            if (j == 0 ? T != 0 : (T < prev || T - prev >= 65536)) return PHOBIC_ERR_FORMAT;
            prev = T;
        }
        if (prev != M) return PHOBIC_ERR_FORMAT;
    }
    // Elias-Fano remap of slots [n, M): its three arrays have the sizes of N = M - n
    // values with the low-bit count of the build, the high part holds exactly N
    // ones and every sample is the position of its one
    if (M > n) {
        const uint64_t N = M - n, l = w[15];
        if (l != ((n / N >= 1) ? bitlen64(n / N) - 1 : 0)) return PHOBIC_ERR_FORMAT;
        const uint64_t hbits = N + (n >> l) + 1;
        if (counts[4] != packed_words(N * l) || counts[5] != packed_words(hbits) || counts[6] != (N + 63) / 64)
            return PHOBIC_ERR_FORMAT;
    }
    // a mono encoder has the layout of its column encoder with one column of B N_P values
    const bool mono = p.encoder >= PHOBIC_ENC_MONO_C;
    const uint32_t enc = mono ? p.encoder - PHOBIC_ENC_MONO_C : p.encoder;
    const uint64_t ncol = mono ? 1 : B, nv = mono ? B * NP : NP;
    if (counts[1] != (enc == PHOBIC_ENC_IC_C ? ncol : 2 * ncol)) return PHOBIC_ERR_FORMAT;
    if (counts[2] == 0 || (enc == PHOBIC_ENC_IC_D && counts[3] == 0)) return PHOBIC_ERR_FORMAT;
    if ((M > n) != (counts[4] != 0 && counts[5] != 0 && counts[6] != 0)) return PHOBIC_ERR_FORMAT;
    // every metadata entry must address inside its array
    {
        const uint64_t* meta = w + kHeaderWords + counts[0];
        for (uint64_t b = 0; b < ncol; b++) {
            for (int t = 0; t < (enc == PHOBIC_ENC_IC_C ? 1 : 2); t++) {
                uint64_t mv = meta[enc == PHOBIC_ENC_IC_C ? b : 2 * b + t];
                uint64_t base = mv & ((1ull << 56) - 1), wd = mv >> 56;
                uint64_t cnt = (t == 0) ? nv : 0;
                if (wd > 32) return PHOBIC_ERR_FORMAT;
                uint64_t arr = (t == 0) ? counts[2] : counts[3];
                if (t == 0 && base + cnt * wd > (arr - 1) * 64) return PHOBIC_ERR_FORMAT;
                if (t == 1 && base > (arr - 1) * 64) return PHOBIC_ERR_FORMAT;
            }
        }
    }
    // IC-R: every column's unary region lies inside the array, holds exactly N_P
    // ones, and each select sample is the position of its 64k-th one, so the
    // query's scans never leave the column
    uint64_t rice_sw = 0;
    const bool unary_enc = enc == PHOBIC_ENC_IC_R || enc == PHOBIC_ENC_IC_EF || enc == PHOBIC_ENC_IC_CR;
    const uint64_t cmix = enc == PHOBIC_ENC_IC_CR ? std::min<uint64_t>(p.compact_columns, B) : 0;
    if (enc == PHOBIC_ENC_IC_CR && p.compact_columns > B) return PHOBIC_ERR_FORMAT;  // exported clamped
    if (mono && p.compact_columns) return PHOBIC_ERR_FORMAT;
    if (unary_enc) {
        const uint64_t ns = (nv + 63) / 64;
        rice_sw = ((ncol - cmix) * ns + 1) / 2;
        if (counts[3] < rice_sw + 1) return PHOBIC_ERR_FORMAT;
        const uint64_t* meta = w + kHeaderWords + counts[0];
        const uint32_t* samp = reinterpret_cast<const uint32_t*>(w + kHeaderWords + counts[0] + counts[1] + counts[2]);
        const uint64_t* high = w + kHeaderWords + counts[0] + counts[1] + counts[2] + rice_sw;
        const uint64_t hbits = (counts[3] - rice_sw - 1) * 64;  // the last word is padding
        for (uint64_t b = 0; b < ncol; b++) {
            const uint64_t hb = meta[2 * b + 1], he = b + 1 < ncol ? meta[2 * b + 3] : hbits;
            if (b < cmix) {  // a Compact column of a mixture: no unary bits
                if ((meta[2 * b] >> 56) > 32 || hb != he) return PHOBIC_ERR_FORMAT;
                continue;
            }
            if ((meta[2 * b] >> 56) > 31 || hb > he || he > hbits) return PHOBIC_ERR_FORMAT;
            uint64_t ones = 0;
            for (uint64_t bit = hb; bit < he; bit++) {
                if (!((high[bit >> 6] >> (bit & 63)) & 1)) continue;
                if (ones >= nv) return PHOBIC_ERR_FORMAT;
                if (ones % 64 == 0 && samp[(b - cmix) * ns + ones / 64] != bit - hb) return PHOBIC_ERR_FORMAT;
                ones++;
            }
            if (ones != nv) return PHOBIC_ERR_FORMAT;
        }
    }
    // IC-D: every rank addresses a value of its column's dictionary (K values of
    // dict_width bits from the column's dictionary base up to the next one's)
    if (enc == PHOBIC_ENC_IC_D) {
        const uint64_t* meta = w + kHeaderWords + counts[0];
        const uint64_t* rk = w + kHeaderWords + counts[0] + counts[1];
        const uint64_t dbits = (counts[3] - 1) * 64;
        for (uint64_t b = 0; b < ncol; b++) {
            const uint64_t rm = meta[2 * b], dm = meta[2 * b + 1];
            const uint32_t rw = (uint32_t)(rm >> 56), dw = (uint32_t)(dm >> 56);
            const uint64_t db = dm & ((1ull << 56) - 1);
            const uint64_t de = b + 1 < ncol ? (meta[2 * b + 3] & ((1ull << 56) - 1)) : dbits;
            if (de < db || de > dbits) return PHOBIC_ERR_FORMAT;
            if (dw == 0) continue;  // every value is 0: nothing is read
            const uint64_t K = (de - db) / dw;
            if (K == 0) return PHOBIC_ERR_FORMAT;
            if (rw == 0) continue;  // every rank is 0 (and the ranks take no bits of the file)
            for (uint64_t j = 0; j < nv; j++)
                if (host_bits(rk, (rm & ((1ull << 56) - 1)) + j * rw, rw) >= K) return PHOBIC_ERR_FORMAT;
        }
    }
    if (M > n) {
        const uint64_t N = M - n;
        const uint64_t hbits = N + (n >> w[15]) + 1;
        const uint64_t* high = w + kHeaderWords + counts[0] + counts[1] + counts[2] + counts[3] + counts[4];
        const uint64_t* samp = high + counts[5];
        uint64_t ones = 0;
        for (uint64_t bit = 0; bit < hbits; bit++) {
            if (!((high[bit >> 6] >> (bit & 63)) & 1)) continue;
            if (ones >= N) return PHOBIC_ERR_FORMAT;
            if (ones % 64 == 0 && samp[ones / 64] != bit) return PHOBIC_ERR_FORMAT;
            ones++;
        }
        if (ones != N) return PHOBIC_ERR_FORMAT;
    }
    pe->n = n;
    pe->M = M;
    pe->NP = NP;
    pe->B = B;
    pe->key_kind = key_kind;
    pe->words = words;
    pe->cmix = cmix;
    pe->rice_sw = rice_sw;
    pe->unary_enc = unary_enc;
    return PHOBIC_OK;
}

// phobic_info of validated export bytes (no device memory)
static void info_of_export(const ParsedExport& pe, const uint64_t* w, phobic_info* I) {
    std::memset(I, 0, sizeof(*I));
    I->n = pe.n;
    I->M = pe.M;
    I->num_partitions = pe.NP;
    I->num_buckets = (uint32_t)pe.B;
    I->partition_size = pe.p.partition_size;
    I->lambda = pe.p.lambda;
    I->alpha = pe.p.alpha;
    I->epsilon = eps_of(pe.p.lambda, pe.p.partition_size);
    I->encoder = pe.p.encoder;
    I->pilot_mode = pe.p.pilot_mode;
    I->seed = pe.p.seed;
    I->bucket_function = pe.p.bucket_function;
    I->compact_columns = (uint32_t)pe.cmix;
    I->bits_header = w[23];
    I->bits_offsets = w[24];
    I->bits_pilots = w[25];
    I->bits_remap = w[26];
    I->bits_total = w[27];
    I->device_bytes = kTablePoints * 8 + 8 * (pe.words - kHeaderWords);
}

phobic_status phobic_inspect(const void* h_buf, size_t len, phobic_info* out) {
    if (!out) return PHOBIC_ERR_INVALID_ARG;
    ParsedExport pe;
    const phobic_status st = parse_export(h_buf, len, &pe);
    if (st != PHOBIC_OK) return st;
    info_of_export(pe, static_cast<const uint64_t*>(h_buf), out);
    return PHOBIC_OK;
}

phobic_status phobic_import(const void* h_buf, size_t len, phobic_stream_t stream, phobic_handle** out) {
    if (!out) return PHOBIC_ERR_INVALID_ARG;
    *out = nullptr;
    ParsedExport pe;
    {
        const phobic_status st = parse_export(h_buf, len, &pe);
        if (st != PHOBIC_OK) return st;
    }
    const uint64_t* w = static_cast<const uint64_t*>(h_buf);
    const phobic_params& p = pe.p;
    const uint64_t n = pe.n, M = pe.M, NP = pe.NP, B = pe.B, words = pe.words, cmix = pe.cmix, rice_sw = pe.rice_sw;
    const uint64_t* counts = pe.counts;
    const uint32_t key_kind = pe.key_kind;
    const bool unary_enc = pe.unary_enc;
    const uint64_t off_w = w[12];
    (void)stream;  // the copies below are synchronous
    phobic_handle* h = new (std::nothrow) phobic_handle();
    if (!h) return PHOBIC_ERR_OOM;
    h->prm = p;
    info_of_export(pe, w, &h->info);
    uint64_t** dst[7] = {&h->off_words, &h->col_meta, &h->pil_words, &h->dict_words,
                         &h->ef_low,    &h->ef_high,  &h->ef_samples};
    uint64_t* cnts[7] = {&h->n_off_words, &h->n_col_meta, &h->n_pil_words, &h->n_dict_words,
                         &h->n_ef_low,    &h->n_ef_high,  &h->n_ef_samples};
    std::vector<uint64_t> table1(kTablePoints + 1), table(kTablePoints);
    make_table(p.lambda, p.alpha, p.partition_size, table1.data(), p.bucket_function);
    pack_bucket_table(table1.data(), table.data());
    // one allocation: the packed table, then the seven arrays in file order
    SharedMem* mem = new (std::nothrow) SharedMem();
    if (!mem) {
        delete h;
        return PHOBIC_ERR_OOM;
    }
    cudaError_t e = cudaMalloc(&mem->ptr, (kTablePoints + (words - kHeaderWords)) * 8);
    if (e != cudaSuccess) {
        delete mem;
        delete h;
        return from_cuda(e);
    }
    mem->refs.store(1);
    h->mem = mem;
    uint64_t* arena = static_cast<uint64_t*>(mem->ptr);
    h->table = arena;
    e = cudaMemcpy(h->table, table.data(), table.size() * 8, cudaMemcpyHostToDevice);
    uint64_t at = kHeaderWords, aw = kTablePoints;
    for (int i = 0; i < 7 && e == cudaSuccess; i++) {
        *cnts[i] = counts[i];
        if (counts[i]) {
            *dst[i] = arena + aw;
            e = cudaMemcpy(*dst[i], w + at, counts[i] * 8, cudaMemcpyHostToDevice);
        }
        at += counts[i];
        aw += counts[i];
    }
    if (e != cudaSuccess) {
        handle_destroy(h);
        return from_cuda(e);
    }
    QueryView& v = h->view;
    v.n = n;
    v.M = M;
    v.NP = NP;
    v.B = (uint32_t)B;
    v.encoder = p.encoder;
    v.pilot_mode = p.pilot_mode;
    v.off_w = (uint32_t)off_w;
    v.kseed = key_seed(p.seed);
    v.off_Q = w[13];
    v.off_dmin = (int64_t)w[14];
    v.table = h->table;
    v.off_words = h->off_words;
    v.col_meta = h->col_meta;
    v.pil_words = h->pil_words;
    v.dict_words = h->dict_words;
    v.ef_N = M - n;
    v.ef_l = (uint32_t)w[15];
    v.ef_low = h->ef_low;
    v.ef_high = h->ef_high;
    v.ef_samples = h->ef_samples;
    v.rice_high = unary_enc ? h->dict_words + rice_sw : nullptr;
    v.rice_ns = unary_enc ? (uint32_t)((NP + 63) / 64) : 0;
    v.mix_c = (uint32_t)cmix;
    v.small_bits = (h->n_pil_words < (1ull << 26) && h->n_dict_words < (1ull << 26)) ? 1 : 0;
    v.key_kind = key_kind;
    v.string_seed = p.seed;
    *out = h;
    return PHOBIC_OK;
}

// ---------------------------------------------------------- stage entry points
phobic_status phobic_hash_u64(const uint64_t* d_keys, uint64_t n, uint64_t seed, uint64_t* d_hk,
                              phobic_stream_t stream) {
    if (n == 0) return PHOBIC_OK;
    if (!d_keys || !d_hk) return PHOBIC_ERR_INVALID_ARG;
    return from_cuda(launch_hash_u64(d_keys, n, key_seed(seed), d_hk, (cudaStream_t)stream));
}

namespace {
phobic_status partition_sort_impl(const uint64_t* d_hk, uint64_t n, uint64_t num_partitions, uint64_t* d_sorted,
                                  uint64_t* d_start, phobic_stream_t stream, const SortWaitTest* wait_test) {
    if (n == 0 || num_partitions == 0 || !d_hk || !d_sorted || !d_start) return PHOBIC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    ensure_pool();
    Arena tmp(st);
    void* scratch;
    uint32_t* err;
    CK(tmp.alloc(&scratch, sort_scratch_bytes(n, num_partitions)));
    CK(tmp.alloc(&err, 16));
    CK(cudaMemsetAsync(err, 0, 16, st));
    CK(launch_partition_sort(d_hk, 0, 0, n, num_partitions, d_sorted, d_start, scratch, err, st, wait_test));
    uint32_t herr = 0;
    CK(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return herr ? PHOBIC_ERR_TIMEOUT : PHOBIC_OK;
}
}  // namespace

phobic_status phobic_partition_sort(const uint64_t* d_hk, uint64_t n, uint64_t num_partitions, uint64_t* d_sorted,
                                    uint64_t* d_start, phobic_stream_t stream) {
    return partition_sort_impl(d_hk, n, num_partitions, d_sorted, d_start, stream, nullptr);
}

phobic_status phobic_selftest_sort_wait_timeout(const uint64_t* d_hk, uint64_t n, uint64_t num_partitions,
                                                uint64_t mute_tile, uint32_t spin_limit, uint64_t* d_sorted,
                                                uint64_t* d_start, phobic_stream_t stream) {
    if (spin_limit == 0) return PHOBIC_ERR_INVALID_ARG;
    const SortWaitTest t{mute_tile, spin_limit};
    return partition_sort_impl(d_hk, n, num_partitions, d_sorted, d_start, stream, &t);
}

phobic_status phobic_bucket_table_ex(double lambda, double alpha, uint32_t partition_size, uint32_t bucket_function,
                                     uint64_t* h_table) {
    if (!h_table || !(lambda > 0.0) || !(alpha > 0.0) || alpha > 1.0 || partition_size == 0 ||
        bucket_function > PHOBIC_BUCKET_UNIFORM)
        return PHOBIC_ERR_INVALID_ARG;
    make_table(lambda, alpha, partition_size, h_table, bucket_function);
    return PHOBIC_OK;
}

phobic_status phobic_bucket_table(double lambda, double alpha, uint32_t partition_size, uint64_t* h_table) {
    if (!h_table || !(lambda > 0.0) || !(alpha > 0.0) || alpha > 1.0 || partition_size == 0)
        return PHOBIC_ERR_INVALID_ARG;
    make_table(lambda, alpha, partition_size, h_table);
    return PHOBIC_OK;
}

}  // extern "C"

extern "C" phobic_status phobic_build_strings(const uint8_t* d_bytes, const uint64_t* d_offsets, uint64_t n,
                                              const phobic_params* params, phobic_stream_t stream,
                                              phobic_handle** out) {
    if (!out) return PHOBIC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!d_bytes || !d_offsets || !params) return PHOBIC_ERR_INVALID_ARG;
    phobic_status s = check_params(n, *params);
    if (s != PHOBIC_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    ensure_pool();
    uint64_t* hk = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&hk, n * 8, st);
    if (e != cudaSuccess) return from_cuda(e);
    e = launch_hash_strings(d_bytes, d_offsets, n, params->seed, hk, st);
    if (e == cudaSuccess) s = build_impl(hk, 0, n, *params, st, out, 1);
    else s = from_cuda(e);
    cudaFreeAsync(hk, st);
    return s;
}

extern "C" phobic_status phobic_query_strings(const phobic_handle* h, const uint8_t* d_bytes,
                                              const uint64_t* d_offsets, uint64_t* d_out, uint64_t m,
                                              phobic_stream_t stream) {
    if (!h || h->view.key_kind != 1) return PHOBIC_ERR_INVALID_ARG;
    if (m == 0) return PHOBIC_OK;
    if (!d_bytes || !d_offsets || !d_out) return PHOBIC_ERR_INVALID_ARG;
    return from_cuda(launch_query_strings(h->view, d_bytes, d_offsets, d_out, m, (cudaStream_t)stream));
}

extern "C" phobic_status phobic_hash_strings(const uint8_t* d_bytes, const uint64_t* d_offsets, uint64_t n,
                                             uint64_t seed, uint64_t* d_hk, phobic_stream_t stream) {
    if (n == 0) return PHOBIC_OK;
    if (!d_bytes || !d_offsets || !d_hk) return PHOBIC_ERR_INVALID_ARG;
    return from_cuda(launch_hash_strings(d_bytes, d_offsets, n, seed, d_hk, (cudaStream_t)stream));
}
