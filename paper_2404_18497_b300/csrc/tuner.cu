// Autotuner for batched construction.
//
// Thousands of key sets of uneven sizes are built in one batched launch
// sequence (phobic_build_batch).  Three knobs change its speed:
//   * the expected partition size P of each set, in {1024, 2500, 4096};
//   * the number of warps that share one partition, in {1, 2, 4};
//   * the number of displacements per lane-window (candidate width), 32 or 64.
// The last two never change a result.  P changes the structure that is built
// (N_P and B follow from it), but every choice is an exact PHOBIC construction
// with that P, reported in the handle's info and reproduced by any builder
// given the same P.
//
// The tuner measures instead of modelling: trial batches of synthetic distinct
// keys (a SplitMix64 counter stream: the finaliser is a bijection, so distinct
// counters give distinct keys) are built through the public entry point and
// timed on the host around the call, which is host-synchronous.
//   1. Sets are grouped into decade size classes [10^c, 10^(c+1)).  For each
//      class, a trial batch repeats the class's own set sizes until it holds
//      at least kClassTrialKeys keys.  Each P is timed; the fastest wins,
//      except that a P within kTieFrac of the fastest with fewer bits per key
//      is preferred.
//   2. With the chosen P per set, a deterministic subsample of the batch (every
//      k-th set) is built with each of the six (warps, width) pairs and the
//      fastest pair is kept, then with each search schedule.  Those knobs trade
//      parallelism inside a partition against the number of partitions in
//      flight, so the subsample keeps enough partitions to fill the GPU several
//      times over (kLaunchTrialWaves waves of one-warp CTAs, or the whole batch
//      when it has fewer), with at most kLaunchTrialMaxKeys keys.  A subsample
//      of far fewer partitions than the batch favours several warps per
//      partition, which the full batch, many waves deep, does not repay.
// Every time is a slope: a trial batch and its first half are both built, and
// their difference in time over their difference in keys is the time per key.
// A launch ends with its last wave of partitions draining, which costs about
// one partition's lifetime whatever the launch's size; in a trial of a few
// waves that drain would decide between knobs that differ in per-partition
// latency rather than in throughput, which is what a batch of hundreds of
// waves sees.  The difference cancels it (and the host's fixed costs).
// Decisions are cached per device and parameter set: per size class for P,
// per power of two of the batch's partition count for (warps, width).
// The paper has no counterpart; this is a deployment convenience.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/phobic.h"
#include "phobic_dev.cuh"
#include "phobic_kernels.cuh"

namespace {

constexpr uint64_t kClassTrialKeys = 1ull << 24;
constexpr uint64_t kLaunchTrialWaves = 8;         // of 32 one-warp CTAs per SM
constexpr uint64_t kLaunchTrialMaxKeys = 1ull << 27;
constexpr double kTieFrac = 0.03;
constexpr int kReps = 2;
constexpr uint32_t kPChoices[PHOBIC_TUNE_P_CHOICES] = {1024, 2500, 4096};
constexpr uint32_t kWarpChoices[3] = {1, 2, 4};
constexpr uint32_t kWidthChoices[2] = {32, 64};

// keys[i] = SplitMix64 output for counter salt + i + 1
__global__ void k_trial_keys(uint64_t* __restrict__ out, uint64_t n, uint64_t salt) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = phobic::mix64((salt + i + 1) * 0x9E3779B97F4A7C15ull);
}

struct ParamKey {
    int dev;
    double lambda, alpha;
    uint32_t encoder, mode, s_max, bucket_fn;
    bool operator<(const ParamKey& o) const {
        return std::tie(dev, lambda, alpha, encoder, mode, s_max, bucket_fn) <
               std::tie(o.dev, o.lambda, o.alpha, o.encoder, o.mode, o.s_max, o.bucket_fn);
    }
};

struct ClassResult {
    uint32_t P;
    float ns_per_key[PHOBIC_TUNE_P_CHOICES];
    float bits_per_key[PHOBIC_TUNE_P_CHOICES];
};
struct LaunchResult {
    uint32_t warps, width, schedule;
    float ns_per_key[6];
    float schedule_ns_per_key[2];  // one CTA per partition, the work queue (chosen warps and width)
};

std::mutex g_mu;
std::map<std::pair<ParamKey, int>, ClassResult> g_class;
std::map<std::pair<ParamKey, int>, LaunchResult> g_launch;

int size_class(uint64_t n) {
    int c = 0;
    while (n >= 10) {
        n /= 10;
        c++;
    }
    return c;
}

uint64_t partitions_of(uint64_t n, uint32_t P) { return std::max<uint64_t>(1, (n + P - 1) / P); }

int log2_floor(uint64_t v) {
    int r = 0;
    while (v > 1) {
        v >>= 1;
        r++;
    }
    return r;
}

// Device keys for a trial, grown on demand and kept for the process.
struct TrialKeys {
    uint64_t* ptr = nullptr;
    uint64_t cap = 0;
};
std::map<int, TrialKeys> g_keys;

phobic_status trial_keys(uint64_t n, cudaStream_t st, const uint64_t** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PHOBIC_ERR_CUDA;
    TrialKeys& t = g_keys[dev];
    if (t.cap < n) {
        if (t.ptr) cudaFree(t.ptr);
        t.ptr = nullptr;
        t.cap = 0;
        if (cudaMalloc(&t.ptr, n * sizeof(uint64_t)) != cudaSuccess) return PHOBIC_ERR_OOM;
        t.cap = n;
        uint64_t blocks = std::min<uint64_t>((n + 255) / 256, 148 * 16);
        k_trial_keys<<<(unsigned)blocks, 256, 0, st>>>(t.ptr, n, 0x5EEDull);
        phobic::note_launches(1);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return PHOBIC_ERR_CUDA;
    }
    *out = t.ptr;
    return PHOBIC_OK;
}

// Best-of-kReps wall time (seconds) of a batched build of sets with the given
// sizes and partition sizes; bits per key over the whole trial in *bits.
phobic_status time_build(const std::vector<uint64_t>& sizes, const std::vector<uint32_t>& Ps,
                         const phobic_params& prm, cudaStream_t st, double* seconds, double* bits) {
    std::vector<uint64_t> off(sizes.size() + 1, 0);
    for (size_t i = 0; i < sizes.size(); i++) off[i + 1] = off[i] + sizes[i];
    const uint64_t* keys = nullptr;
    phobic_status s = trial_keys(off.back(), st, &keys);
    if (s != PHOBIC_OK) return s;
    std::vector<phobic_handle*> hs(sizes.size(), nullptr);
    double best = 1e30;
    for (int r = 0; r < kReps; r++) {
        const auto t0 = std::chrono::steady_clock::now();
        s = phobic_build_batch(keys, off.data(), (uint32_t)sizes.size(), Ps.data(), &prm, st, hs.data());
        const auto t1 = std::chrono::steady_clock::now();
        if (s != PHOBIC_OK) return s;
        best = std::min(best, std::chrono::duration<double>(t1 - t0).count());
        if (r == kReps - 1) {
            double tb = 0;
            for (size_t i = 0; i < hs.size(); i++) tb += phobic_bits_per_key(hs[i]) * (double)sizes[i];
            *bits = tb / (double)off.back();
        }
        for (auto*& h : hs) {
            phobic_free(h);
            h = nullptr;
        }
    }
    *seconds = best;
    return PHOBIC_OK;
}

// Steady-state seconds per key of a batched build: the time of `sizes` minus
// that of its first half, over the keys the second half adds (one set: its
// time over its keys).  Bits per key of the whole trial in *bits.
phobic_status time_slope(const std::vector<uint64_t>& sizes, const std::vector<uint32_t>& Ps,
                         const phobic_params& prm, cudaStream_t st, double* sec_per_key, double* bits) {
    double full = 0;
    phobic_status s = time_build(sizes, Ps, prm, st, &full, bits);
    if (s != PHOBIC_OK) return s;
    const size_t h = sizes.size() / 2;
    uint64_t keys_all = 0, keys_second = 0;
    for (size_t i = 0; i < sizes.size(); i++) {
        keys_all += sizes[i];
        if (i >= h) keys_second += sizes[i];
    }
    if (h == 0) {
        *sec_per_key = full / (double)keys_all;
        return PHOBIC_OK;
    }
    const std::vector<uint64_t> s1(sizes.begin(), sizes.begin() + h);
    const std::vector<uint32_t> p1(Ps.begin(), Ps.begin() + h);
    double half = 0, bits_half = 0;
    s = time_build(s1, p1, prm, st, &half, &bits_half);
    if (s != PHOBIC_OK) return s;
    // a difference below a tenth of the full time is noise: fall back to the full time
    const double d = full - half;
    *sec_per_key = d > 0.1 * full ? d / (double)keys_second : full / (double)keys_all;
    return PHOBIC_OK;
}

}  // namespace

extern "C" phobic_status phobic_tune_batch(const uint64_t* h_set_offsets, uint32_t n_sets,
                                           const phobic_params* params, phobic_stream_t stream,
                                           uint32_t* h_partition_sizes_out, phobic_params* params_out,
                                           phobic_tune_info* info) {
    if (!h_set_offsets || n_sets == 0 || !params || !h_partition_sizes_out || !params_out)
        return PHOBIC_ERR_INVALID_ARG;
    for (uint32_t s = 0; s < n_sets; s++)
        if (h_set_offsets[s + 1] <= h_set_offsets[s]) return PHOBIC_ERR_INVALID_ARG;
    // a candidate partition size below lambda is not a valid build; none left: refuse
    if (!(params->lambda > 0.0) || params->lambda > (double)kPChoices[PHOBIC_TUNE_P_CHOICES - 1])
        return PHOBIC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PHOBIC_ERR_CUDA;
    const ParamKey pk{dev,           params->lambda,     params->alpha,          params->encoder,
                      params->pilot_mode, params->s_max, params->bucket_function};
    phobic_params base = *params;
    base.keep_pilots = 0;
    base.record_timings = 0;
    base.warps_per_partition = 1;
    base.candidate_width = 64;
    base.search_schedule = 1;
    if (info) *info = phobic_tune_info{};

    std::lock_guard<std::mutex> lock(g_mu);
    // ---- 1. partition size per decade size class
    std::map<int, std::vector<uint64_t>> by_class;
    for (uint32_t s = 0; s < n_sets; s++) {
        const uint64_t n = h_set_offsets[s + 1] - h_set_offsets[s];
        by_class[size_class(n)].push_back(n);
    }
    std::map<int, uint32_t> chosen;
    for (auto& kv : by_class) {
        const int c = kv.first;
        auto it = g_class.find({pk, c});
        if (it == g_class.end()) {
            // the class's own sizes, in input order, repeated up to the trial size
            std::vector<uint64_t> sizes;
            uint64_t tot = 0;
            for (size_t i = 0; tot < kClassTrialKeys; i++) {
                sizes.push_back(kv.second[i % kv.second.size()]);
                tot += sizes.back();
            }
            ClassResult cr{};
            double best = 1e30;
            for (int i = 0; i < PHOBIC_TUNE_P_CHOICES; i++) {
                double sec = 0, bits = 0;
                phobic_params p = base;
                p.partition_size = kPChoices[i];
                if ((double)kPChoices[i] < p.lambda) {  // never picked
                    cr.ns_per_key[i] = cr.bits_per_key[i] = INFINITY;
                    continue;
                }
                std::vector<uint32_t> Ps(sizes.size(), kPChoices[i]);
                phobic_status s = time_slope(sizes, Ps, p, st, &sec, &bits);
                if (s != PHOBIC_OK) return s;
                cr.ns_per_key[i] = (float)(sec * 1e9);
                cr.bits_per_key[i] = (float)bits;
                best = std::min(best, (double)cr.ns_per_key[i]);
            }
            int pick = -1;
            for (int i = 0; i < PHOBIC_TUNE_P_CHOICES; i++)
                if (cr.ns_per_key[i] <= best * (1.0 + kTieFrac) &&
                    (pick < 0 || cr.bits_per_key[i] < cr.bits_per_key[pick]))
                    pick = i;
            cr.P = kPChoices[pick];
            it = g_class.emplace(std::make_pair(pk, c), cr).first;
        } else if (info) {
            info->cached_classes++;
        }
        chosen[c] = it->second.P;
        if (info && c < PHOBIC_TUNE_MAX_CLASSES) {
            phobic_tune_class& tc = info->classes[c];
            tc.sets = (uint32_t)kv.second.size();
            tc.partition_size = it->second.P;
            for (int i = 0; i < PHOBIC_TUNE_P_CHOICES; i++) {
                tc.ns_per_key[i] = it->second.ns_per_key[i];
                tc.bits_per_key[i] = it->second.bits_per_key[i];
            }
        }
    }
    uint64_t total_parts = 0, total = h_set_offsets[n_sets] - h_set_offsets[0];
    for (uint32_t s = 0; s < n_sets; s++) {
        const uint64_t n = h_set_offsets[s + 1] - h_set_offsets[s];
        h_partition_sizes_out[s] = chosen[size_class(n)];
        total_parts += partitions_of(n, h_partition_sizes_out[s]);
    }

    // ---- 2. warps per partition and candidate width for the whole launch
    const int lk = log2_floor(total_parts);
    auto it = g_launch.find({pk, lk});
    if (it == g_launch.end()) {
        int sms = 148;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const uint64_t want_parts = std::min<uint64_t>(total_parts, kLaunchTrialWaves * 32 * (uint64_t)sms);
        // every stride-th set: about total_parts / stride partitions and total / stride keys
        uint64_t stride = std::max<uint64_t>(1, total_parts / want_parts);
        stride = std::max<uint64_t>(stride, (total + kLaunchTrialMaxKeys - 1) / kLaunchTrialMaxKeys);
        std::vector<uint64_t> sizes;
        std::vector<uint32_t> Ps;
        uint64_t tot = 0;
        for (uint32_t s = 0; s < n_sets; s += (uint32_t)std::min<uint64_t>(stride, n_sets)) {
            sizes.push_back(h_set_offsets[s + 1] - h_set_offsets[s]);
            Ps.push_back(h_partition_sizes_out[s]);
            tot += sizes.back();
        }
        LaunchResult lr{};
        double best = 1e30;
        int k = 0;
        for (uint32_t w : kWarpChoices)
            for (uint32_t cw : kWidthChoices) {
                phobic_params p = base;
                p.warps_per_partition = w;
                p.candidate_width = cw;
                double sec = 0, bits = 0;
                phobic_status s = time_slope(sizes, Ps, p, st, &sec, &bits);
                if (s != PHOBIC_OK) return s;
                lr.ns_per_key[k] = (float)(sec * 1e9);
                if (lr.ns_per_key[k] < best) {
                    best = lr.ns_per_key[k];
                    lr.warps = w;
                    lr.width = cw;
                }
                k++;
            }
        // the schedule, with the chosen knobs: one CTA per partition (1) or the
        // persistent CTAs over the device work queue (2); the faster one is kept
        for (int sc = 0; sc < 2; sc++) {
            phobic_params p = base;
            p.warps_per_partition = lr.warps;
            p.candidate_width = lr.width;
            p.search_schedule = sc + 1;
            double sec = 0, bits = 0;
            phobic_status s = time_slope(sizes, Ps, p, st, &sec, &bits);
            if (s != PHOBIC_OK) return s;
            lr.schedule_ns_per_key[sc] = (float)(sec * 1e9);
        }
        lr.schedule = lr.schedule_ns_per_key[0] < lr.schedule_ns_per_key[1] ? 1 : 2;
        it = g_launch.emplace(std::make_pair(pk, lk), lr).first;
    } else if (info) {
        info->cached_launch = 1;
    }
    *params_out = *params;
    params_out->warps_per_partition = it->second.warps;
    params_out->candidate_width = it->second.width;
    params_out->search_schedule = it->second.schedule;
    if (info) {
        info->warps_per_partition = it->second.warps;
        info->candidate_width = it->second.width;
        info->search_schedule = it->second.schedule;
        info->schedule_ns_per_key[0] = it->second.schedule_ns_per_key[0];
        info->schedule_ns_per_key[1] = it->second.schedule_ns_per_key[1];
        for (int i = 0; i < 6; i++) info->launch_ns_per_key[i] = it->second.ns_per_key[i];
        info->total_partitions = total_parts;
    }
    return PHOBIC_OK;
}

extern "C" void phobic_tune_clear(void) {
    std::lock_guard<std::mutex> lock(g_mu);
    g_class.clear();
    g_launch.clear();
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto& kv : g_keys) {
        if (!kv.second.ptr) continue;
        cudaSetDevice(kv.first);
        cudaFree(kv.second.ptr);
    }
    g_keys.clear();
    cudaSetDevice(cur);
}
