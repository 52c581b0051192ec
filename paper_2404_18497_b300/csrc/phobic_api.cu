// libphobic C ABI: argument checks, build orchestration, the handle,
// serialization and space accounting.  Every step of construction and query
// runs in the kernels of k_*.cu; this file only sequences them, sizes buffers
// from the few scalars the device reports, and owns memory.
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
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

void make_table(double lambda, double alpha, uint32_t P, uint64_t* t) {
    const double eps = eps_of(lambda, P);
    for (int k = 0; k <= kTablePoints; k++) {
        const double x = (double)k / (double)kTablePoints;
        double g;
        if (alpha == 1.0) {
            g = x >= 1.0 ? 1.0 : eps * x + (1.0 - eps) * beta_star(x);
        } else {
            const double ax = alpha * x;
            g = (eps * ax + (1.0 - eps) * beta_star(ax)) / (eps * alpha + (1.0 - eps) * beta_star(alpha));
        }
        long long r = std::llround(g * 4294967296.0);
        if (r < 0) r = 0;
        if (r > 4294967296LL) r = 4294967296LL;
        t[k] = (uint64_t)r;
    }
}

uint32_t num_buckets(double lambda, uint32_t P) {
    double b = std::ceil((double)P / lambda);
    return b < 1.0 ? 1u : (uint32_t)b;
}

uint64_t num_partitions(uint64_t n, uint32_t P) {
    uint64_t np = (n + P - 1) / P;
    return np ? np : 1;
}

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
    void disown(void* p) {
        for (auto& q : ptrs)
            if (q == p) {
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
            if (buf) cudaFreeHost(buf);
            buf = nullptr;
            cap = 0;
            cudaError_t e = cudaMallocHost(&buf, bytes);
            if (e != cudaSuccess) return e;
            cap = bytes;
        }
        p = buf;
        return cudaSuccess;
    }
};

}  // namespace

struct phobic_handle {
    phobic_params prm;
    phobic_info info;
    QueryView view;
    // owned device buffers
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
    std::vector<void*> owned;
};

namespace {

void handle_destroy(phobic_handle* h) {
    if (!h) return;
    cudaDeviceSynchronize();
    for (void* p : h->owned) cudaFree(p);
    delete h;
}

phobic_status check_params(uint64_t n, const phobic_params& p) {
    if (n == 0) return PHOBIC_ERR_INVALID_ARG;
    if (!(p.lambda > 0.0) || !std::isfinite(p.lambda)) return PHOBIC_ERR_INVALID_ARG;
    if (!(p.alpha > 0.0) || p.alpha > 1.0) return PHOBIC_ERR_INVALID_ARG;
    if (p.partition_size == 0 || p.partition_size > kMaxPartitionSize) return PHOBIC_ERR_INVALID_ARG;
    if (p.encoder > PHOBIC_ENC_IC_D || p.pilot_mode > PHOBIC_PILOT_XOR) return PHOBIC_ERR_INVALID_ARG;
    if (p.warps_per_partition > 1) return PHOBIC_ERR_INVALID_ARG;  // one warp per partition
    if (p.candidate_width != 0 && p.candidate_width != 32 && p.candidate_width != 64) return PHOBIC_ERR_INVALID_ARG;
    return PHOBIC_OK;
}

// space accounting (fixed spec): header, offsets, pilot encoders with their
// metadata, Elias-Fano remap
void account(phobic_handle* h, const std::vector<uint32_t>& w1, const std::vector<uint32_t>& w2,
             const std::vector<uint64_t>& K) {
    phobic_info& I = h->info;
    const uint64_t NP = I.num_partitions;
    I.bits_header = 9 * 64;
    I.bits_offsets = (NP + 1) * (uint64_t)h->view.off_w + 64 + 64 + 8;
    uint64_t bp = 0;
    for (uint32_t b = 0; b < I.num_buckets; b++) {
        if (I.encoder == PHOBIC_ENC_IC_C)
            bp += NP * (uint64_t)w1[b] + 64 + 8;
        else
            bp += NP * (uint64_t)w1[b] + K[b] * (uint64_t)w2[b] + 64 + 64 + 8 + 8;
    }
    I.bits_pilots = bp;
    I.bits_remap = 0;
    const uint64_t N = I.M - I.n;
    if (N) {
        const uint32_t l = h->view.ef_l;
        I.bits_remap = N * (uint64_t)l + (N + (I.n >> l) + 1) + 64 * ((N + 63) / 64) + 3 * 64;
    }
    I.bits_total = I.bits_header + I.bits_offsets + I.bits_pilots + I.bits_remap;
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

// Builds from master hashes (already sorted by the caller's choice of path):
// `in` holds raw keys (hash_input = 1) or master hashes (hash_input = 0).
phobic_status build_impl(const uint64_t* in, int hash_input, uint64_t n, const phobic_params& prm, cudaStream_t st,
                         phobic_handle** out, uint32_t key_kind = 0) {
    ensure_pool();
    const uint64_t NP = num_partitions(n, prm.partition_size);
    const uint32_t B = num_buckets(prm.lambda, prm.partition_size);
    const uint64_t kseed = key_seed(prm.seed);
    Arena tmp(st), own(st);

    phobic_handle* h = new (std::nothrow) phobic_handle();
    if (!h) return PHOBIC_ERR_OOM;
    struct Guard {
        phobic_handle*& h;
        Arena& own;
        ~Guard() {
            if (h) delete h;
        }
    } guard{h, own};
    h->prm = prm;
    std::memset(&h->info, 0, sizeof(h->info));
    h->info.n = n;
    h->info.num_partitions = NP;
    h->info.num_buckets = B;
    h->info.partition_size = prm.partition_size;
    h->info.lambda = prm.lambda;
    h->info.alpha = prm.alpha;
    h->info.epsilon = eps_of(prm.lambda, prm.partition_size);
    h->info.encoder = prm.encoder;
    h->info.pilot_mode = prm.pilot_mode;
    h->info.seed = prm.seed;

    PhaseEvents ev;
    CK(ev.init(prm.record_timings != 0));

    // pinned scalars exchanged with the device
    PinnedBuf pin;
    CK(pin.alloc(4096 + (size_t)B * 16));
    uint64_t* hst = static_cast<uint64_t*>(pin.p);

    // ---- bucket table
    std::vector<uint64_t> table(kTablePoints + 1);
    make_table(prm.lambda, prm.alpha, prm.partition_size, table.data());
    CK(own.alloc(&h->table, table.size() * 8));
    CK(h2d(h->table, table.data(), table.size(), st));

    // ---- K1 + K2: hash, partition sort, partition starts
    uint64_t *sorted, *start, *T, *stats;
    uint32_t* status;
    void* sort_scratch;
    CK(tmp.alloc(&sorted, n * 8));
    CK(tmp.alloc(&start, (NP + 1) * 8));
    CK(tmp.alloc(&T, (NP + 1) * 8));
    CK(tmp.alloc(&stats, 64));
    CK(tmp.alloc(&status, 64));
    CK(cudaMemsetAsync(status, 0, 64, st));
    CK(tmp.alloc(&sort_scratch, sort_scratch_bytes(n, NP)));
    CK(ev.mark(0, st));
    CK(launch_partition_sort(in, hash_input, kseed, n, NP, sorted, start, sort_scratch, status, st));
    CK(ev.mark(1, st));
    tmp.release(sort_scratch);
    void* sizes_scratch;
    CK(tmp.alloc(&sizes_scratch, sizes_scratch_bytes(NP)));
    CK(launch_sizes(start, NP, prm.alpha, T, stats, sizes_scratch, st));
    CK(ev.mark(2, st));
    CK(d2h(hst, stats, 3, st));
    CK(d2h(reinterpret_cast<uint32_t*>(hst + 4), status, 1, st));
    CK(cudaStreamSynchronize(st));
    const uint64_t M = hst[0], max_n = hst[1], max_m = hst[2];
    if (reinterpret_cast<uint32_t*>(hst + 4)[0] == kDevTimeout) return PHOBIC_ERR_TIMEOUT;
    h->info.M = M;
    h->info.max_partition = max_n;
    // keys in shared memory only on request (debug / comparison); default: global scratch
    const char* ks = std::getenv("PHOBIC_KEYS_IN_SMEM");
    const bool keys_in_smem = ks && ks[0] == '1';
    if (max_m >= 65536 || max_n >= (1u << 31) ||
        search_smem_bytes((uint32_t)max_n, (uint32_t)max_m, B, keys_in_smem) > search_smem_limit())
        return PHOBIC_ERR_PARTITION_TOO_LARGE;
    uint32_t s_max = prm.s_max ? prm.s_max : 65536u;
    if (max_m > 0 && (uint64_t)s_max * max_m > 0xFFFFFFFFull) s_max = (uint32_t)(0xFFFFFFFFull / max_m);
    h->prm.s_max = s_max;

    // ---- K3 + K4: bucketing and pilot search
    uint32_t* pilots;
    uint32_t* taken = nullptr;
    CK(tmp.alloc(&pilots, (uint64_t)B * NP * 4));
    CK(cudaMemsetAsync(pilots, 0, (uint64_t)B * NP * 4, st));
    if (M > n) {
        CK(tmp.alloc(&taken, ((M + 31) / 32 + 1) * 4));
        CK(cudaMemsetAsync(taken, 0, ((M + 31) / 32 + 1) * 4, st));
    }
    uint64_t* bkeys = nullptr;
    if (!keys_in_smem) CK(tmp.alloc(&bkeys, n * 8));
    SearchLaunch sl;
    sl.bkeys = bkeys;
    sl.keys_in_smem = keys_in_smem ? 1 : 0;
    sl.window_bits = prm.candidate_width == 32 ? 32 : 64;
    sl.sorted = sorted;
    sl.start = start;
    sl.T = T;
    sl.table = h->table;
    sl.np = NP;
    sl.B = B;
    sl.mode = prm.pilot_mode;
    sl.s_max = s_max;
    sl.cap_n = (uint32_t)max_n;
    sl.cap_m = (uint32_t)max_m;
    sl.pilots = pilots;
    sl.taken_bits = taken;
    sl.status = status;
    unsigned long long* work = nullptr;
    if (prm.record_timings) {
        CK(tmp.alloc(&work, 16));
        CK(cudaMemsetAsync(work, 0, 16, st));
    }
    sl.work = work;
    CK(ev.mark(3, st));
    CK(launch_search(sl, st));
    CK(ev.mark(4, st));
    tmp.release(sorted);
    if (bkeys) tmp.release(bkeys);

    // ---- K5: offsets; K6: column maxima
    const uint64_t Q = (uint64_t)((((unsigned __int128)M) << 32) / NP);
    long long* mm;
    uint32_t* colmax;
    CK(tmp.alloc(&mm, 16));
    CK(tmp.alloc(&colmax, (size_t)B * 4));
    CK(ev.mark(5, st));
    CK(launch_offset_minmax(T, NP, Q, mm, st));
    CK(launch_column_max(pilots, NP, B, colmax, st));
    long long* hmm = reinterpret_cast<long long*>(hst + 8);
    uint32_t* hcolmax = reinterpret_cast<uint32_t*>(hst + 16);
    CK(d2h(hmm, mm, 2, st));
    CK(d2h(hcolmax, colmax, B, st));
    if (work) CK(d2h(hst + 12, reinterpret_cast<uint64_t*>(work), 2, st));
    CK(d2h(reinterpret_cast<uint32_t*>(hst + 4), status, 1, st));
    CK(cudaStreamSynchronize(st));
    switch (reinterpret_cast<uint32_t*>(hst + 4)[0]) {
        case kDevOk: break;
        case kDevDupHash: return PHOBIC_ERR_DUP_HASH;
        case kDevSearchLimit: return PHOBIC_ERR_SEARCH_LIMIT;
        default: return PHOBIC_ERR_TIMEOUT;
    }
    const int64_t dmin = hmm[0], dmax = hmm[1];
    const uint32_t off_w = bitlen64((uint64_t)(dmax - dmin));
    h->n_off_words = packed_words((NP + 1) * (uint64_t)off_w);
    CK(own.alloc(&h->off_words, h->n_off_words * 8));
    CK(launch_offset_pack(T, NP, Q, dmin, off_w, h->off_words, h->n_off_words, st));

    std::vector<uint32_t> w1(B), w2(B);
    std::vector<uint64_t> K(B, 0);
    std::vector<uint64_t> meta, wbegin(B + 1, 0);
    if (prm.encoder == PHOBIC_ENC_IC_C) {
        meta.resize(B);
        uint64_t base = 0;
        for (uint32_t b = 0; b < B; b++) {
            w1[b] = bitlen64(hcolmax[b]);
            meta[b] = base | ((uint64_t)w1[b] << 56);
            uint64_t bits = NP * (uint64_t)w1[b];
            wbegin[b + 1] = wbegin[b] + (bits ? ((base + bits - 1) >> 6) - (base >> 6) + 1 : 0);
            base += bits;
        }
        h->n_pil_words = packed_words(base);
        h->n_col_meta = B;
        uint64_t* dwb;
        CK(own.alloc(&h->col_meta, (size_t)B * 8));
        CK(tmp.alloc(&dwb, (size_t)(B + 1) * 8));
        CK(own.alloc(&h->pil_words, h->n_pil_words * 8));
        CK(h2d(h->col_meta, meta.data(), B, st));
        CK(h2d(dwb, wbegin.data(), B + 1, st));
        CK(cudaMemsetAsync(h->pil_words, 0, h->n_pil_words * 8, st));
        CK(launch_compact_pack(pilots, NP, B, h->col_meta, dwb, h->pil_words, wbegin[B], st));
    } else {
        // presence bitmaps over [0, max_b] per column
        std::vector<uint64_t> bm_base(B + 1, 0);
        for (uint32_t b = 0; b < B; b++) bm_base[b + 1] = bm_base[b] + ((uint64_t)hcolmax[b] + 64) / 64;
        uint64_t *dbm_base, *bitmaps, *brank, *dK;
        CK(tmp.alloc(&dbm_base, (size_t)(B + 1) * 8));
        CK(tmp.alloc(&bitmaps, bm_base[B] * 8));
        CK(tmp.alloc(&brank, bm_base[B] * 8));
        CK(tmp.alloc(&dK, (size_t)B * 8));
        CK(h2d(dbm_base, bm_base.data(), B + 1, st));
        CK(cudaMemsetAsync(bitmaps, 0, bm_base[B] * 8, st));
        CK(launch_dict_mark(pilots, NP, B, dbm_base, bitmaps, st));
        CK(launch_dict_rank(dbm_base, B, brank, bitmaps, dK, st));
        uint64_t* hK = hst + 16 + (B + 1) / 2 + 1;
        CK(d2h(hK, dK, B, st));
        CK(cudaStreamSynchronize(st));
        meta.resize(2 * (size_t)B);
        uint64_t rbase = 0, dbase = 0;
        for (uint32_t b = 0; b < B; b++) {
            K[b] = hK[b];
            w1[b] = bitlen64(K[b] - 1);         // rank width
            w2[b] = bitlen64(hcolmax[b]);       // dictionary value width
            meta[2 * b] = rbase | ((uint64_t)w1[b] << 56);
            meta[2 * b + 1] = dbase | ((uint64_t)w2[b] << 56);
            uint64_t bits = NP * (uint64_t)w1[b];
            wbegin[b + 1] = wbegin[b] + (bits ? ((rbase + bits - 1) >> 6) - (rbase >> 6) + 1 : 0);
            rbase += bits;
            dbase += K[b] * (uint64_t)w2[b];
        }
        h->n_pil_words = packed_words(rbase);
        h->n_dict_words = packed_words(dbase);
        h->n_col_meta = 2 * (uint64_t)B;
        uint64_t* dwb;
        CK(own.alloc(&h->col_meta, (size_t)B * 16));
        CK(tmp.alloc(&dwb, (size_t)(B + 1) * 8));
        CK(own.alloc(&h->pil_words, h->n_pil_words * 8));
        CK(own.alloc(&h->dict_words, h->n_dict_words * 8));
        CK(h2d(h->col_meta, meta.data(), 2 * (size_t)B, st));
        CK(h2d(dwb, wbegin.data(), B + 1, st));
        CK(cudaMemsetAsync(h->pil_words, 0, h->n_pil_words * 8, st));
        CK(cudaMemsetAsync(h->dict_words, 0, h->n_dict_words * 8, st));
        CK(launch_dict_pack(pilots, NP, B, dbm_base, bitmaps, brank, h->col_meta, dwb, h->pil_words, wbegin[B],
                            nullptr, h->dict_words, bm_base[B], st));
    }

    CK(ev.mark(6, st));
    // ---- K7: Elias-Fano remap of slots >= n
    uint32_t ef_l = 0;
    if (M > n) {
        const uint64_t N = M - n;
        ef_l = (n / N >= 1) ? bitlen64(n / N) - 1 : 0;
        h->n_ef_low = packed_words(N * (uint64_t)ef_l);
        h->n_ef_high = packed_words(N + (n >> ef_l) + 1);
        h->n_ef_samples = (N + 63) / 64;
        uint64_t* fs;
        void* rs;
        CK(tmp.alloc(&fs, N * 8));
        CK(tmp.alloc(&rs, remap_scratch_bytes(n, M)));
        CK(own.alloc(&h->ef_low, h->n_ef_low * 8));
        CK(own.alloc(&h->ef_high, h->n_ef_high * 8));
        CK(own.alloc(&h->ef_samples, h->n_ef_samples * 8));
        CK(launch_remap(taken, n, M, ef_l, fs, h->ef_low, h->n_ef_low, h->ef_high, h->n_ef_high, h->ef_samples, rs,
                        st));
    }
    CK(ev.mark(7, st));
    if (prm.keep_pilots) {
        h->pilots = pilots;
        tmp.disown(pilots);
        own.ptrs.push_back(pilots);
    }
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());

    // ---- view for the query kernel
    QueryView& v = h->view;
    v.n = n;
    v.M = M;
    v.NP = NP;
    v.B = B;
    v.encoder = prm.encoder;
    v.pilot_mode = prm.pilot_mode;
    v.off_w = off_w;
    v.kseed = kseed;
    v.off_Q = Q;
    v.off_dmin = dmin;
    v.table = h->table;
    v.off_words = h->off_words;
    v.col_meta = h->col_meta;
    v.pil_words = h->pil_words;
    v.dict_words = h->dict_words;
    v.ef_N = M - n;
    v.ef_l = ef_l;
    v.ef_low = h->ef_low;
    v.ef_high = h->ef_high;
    v.ef_samples = h->ef_samples;
    v.small_bits = (h->n_pil_words < (1ull << 26) && h->n_dict_words < (1ull << 26)) ? 1 : 0;
    v.key_kind = key_kind;
    v.string_seed = prm.seed;
    account(h, w1, w2, K);
    if (ev.on) {
        h->has_timings = true;
        h->timings.sort_ms = ev.between(0, 1);
        h->timings.sizes_ms = ev.between(1, 2);
        h->timings.search_ms = ev.between(3, 4);
        // encode spans host synchronisations (column widths, dictionary sizes);
        // it is reported as device time between its first and last event
        h->timings.encode_ms = ev.between(5, 6);
        h->timings.remap_ms = ev.between(6, 7);
        h->timings.total_ms = ev.between(0, 7);
        h->timings.search_s_tries = hst[12];
        h->timings.search_steps = hst[13];
    }

    // the handle takes the permanent buffers
    for (void* p : own.ptrs) h->owned.push_back(p);
    own.ptrs.clear();
    uint64_t dev_bytes = (kTablePoints + 1) * 8 + 8 * (h->n_off_words + h->n_col_meta + h->n_pil_words +
                                                     h->n_dict_words + h->n_ef_low + h->n_ef_high + h->n_ef_samples);
    if (h->pilots) dev_bytes += (uint64_t)B * NP * 4;  // counted once: pilots was moved into `own`
    h->info.device_bytes = dev_bytes;
    *out = h;
    h = nullptr;  // guard releases nothing
    return PHOBIC_OK;
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
    p->s_max = 65536;
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

phobic_status phobic_query(const phobic_handle* h, const uint64_t* d_keys, uint64_t* d_out, uint64_t m,
                           phobic_stream_t stream) {
    if (!h || h->view.key_kind != 0) return PHOBIC_ERR_INVALID_ARG;
    if (m == 0) return PHOBIC_OK;
    if (!d_keys || !d_out) return PHOBIC_ERR_INVALID_ARG;
    return from_cuda(launch_query(h->view, d_keys, d_out, m, (cudaStream_t)stream));
}

phobic_status phobic_query_host(const phobic_handle* h, const uint64_t* h_keys, uint64_t* h_out, uint64_t m,
                                phobic_stream_t stream) {
    if (!h || h->view.key_kind != 0) return PHOBIC_ERR_INVALID_ARG;
    if (m == 0) return PHOBIC_OK;
    if (!h_keys || !h_out) return PHOBIC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    ensure_pool();
    uint64_t* d = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&d, m * 16, st);
    if (e != cudaSuccess) return from_cuda(e);
    e = cudaMemcpyAsync(d, h_keys, m * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_query(h->view, d, d + m, m, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_out, d + m, m * 8, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(d, st);
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
                                  I.partition_size, lam, alp, I.seed, I.encoder, (uint64_t)I.pilot_mode | ((uint64_t)h->view.key_kind << 32), h->view.off_w,
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

phobic_status phobic_import(const void* h_buf, size_t len, phobic_stream_t stream, phobic_handle** out) {
    if (!out) return PHOBIC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!h_buf || len < kHeaderWords * 8 || (len & 7)) return PHOBIC_ERR_FORMAT;
    const uint64_t* w = static_cast<const uint64_t*>(h_buf);
    if (w[0] != kMagic || w[1] != kFormatVersion) return PHOBIC_ERR_FORMAT;
    phobic_params p;
    phobic_params_init(&p);
    const uint64_t n = w[2], M = w[3], NP = w[4], B = w[5], P = w[6];
    std::memcpy(&p.lambda, &w[7], 8);
    std::memcpy(&p.alpha, &w[8], 8);
    p.partition_size = (uint32_t)P;
    p.seed = w[9];
    p.encoder = (uint32_t)w[10];
    p.pilot_mode = (uint32_t)w[11];
    const uint32_t key_kind = (uint32_t)(w[11] >> 32);
    if (key_kind > 1) return PHOBIC_ERR_FORMAT;
    if (P != p.partition_size || check_params(n, p) != PHOBIC_OK) return PHOBIC_ERR_FORMAT;
    if (NP != num_partitions(n, p.partition_size) || B != num_buckets(p.lambda, p.partition_size) || M < n)
        return PHOBIC_ERR_FORMAT;
    uint64_t counts[7];
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
    if (counts[1] != (p.encoder == PHOBIC_ENC_IC_C ? B : 2 * B)) return PHOBIC_ERR_FORMAT;
    if (counts[2] == 0 || (p.encoder == PHOBIC_ENC_IC_D && counts[3] == 0)) return PHOBIC_ERR_FORMAT;
    if ((M > n) != (counts[4] != 0 && counts[5] != 0 && counts[6] != 0)) return PHOBIC_ERR_FORMAT;
    // every metadata entry must address inside its array
    {
        const uint64_t* meta = w + kHeaderWords + counts[0];
        for (uint64_t b = 0; b < B; b++) {
            for (int t = 0; t < (p.encoder == PHOBIC_ENC_IC_C ? 1 : 2); t++) {
                uint64_t mv = meta[p.encoder == PHOBIC_ENC_IC_C ? b : 2 * b + t];
                uint64_t base = mv & ((1ull << 56) - 1), wd = mv >> 56;
                uint64_t cnt = (t == 0) ? NP : 0;
                if (wd > 32) return PHOBIC_ERR_FORMAT;
                uint64_t arr = (t == 0) ? counts[2] : counts[3];
                if (t == 0 && base + cnt * wd > (arr - 1) * 64) return PHOBIC_ERR_FORMAT;
                if (t == 1 && base > (arr - 1) * 64) return PHOBIC_ERR_FORMAT;
            }
        }
    }
    (void)stream;  // the copies below are synchronous
    phobic_handle* h = new (std::nothrow) phobic_handle();
    if (!h) return PHOBIC_ERR_OOM;
    h->prm = p;
    std::memset(&h->info, 0, sizeof(h->info));
    phobic_info& I = h->info;
    I.n = n;
    I.M = M;
    I.num_partitions = NP;
    I.num_buckets = (uint32_t)B;
    I.partition_size = p.partition_size;
    I.lambda = p.lambda;
    I.alpha = p.alpha;
    I.epsilon = eps_of(p.lambda, p.partition_size);
    I.encoder = p.encoder;
    I.pilot_mode = p.pilot_mode;
    I.seed = p.seed;
    I.bits_header = w[23];
    I.bits_offsets = w[24];
    I.bits_pilots = w[25];
    I.bits_remap = w[26];
    I.bits_total = w[27];
    uint64_t** dst[7] = {&h->off_words, &h->col_meta, &h->pil_words, &h->dict_words,
                         &h->ef_low,    &h->ef_high,  &h->ef_samples};
    uint64_t* cnts[7] = {&h->n_off_words, &h->n_col_meta, &h->n_pil_words, &h->n_dict_words,
                         &h->n_ef_low,    &h->n_ef_high,  &h->n_ef_samples};
    std::vector<uint64_t> table(kTablePoints + 1);
    make_table(p.lambda, p.alpha, p.partition_size, table.data());
    cudaError_t e = cudaMalloc(&h->table, table.size() * 8);
    if (e == cudaSuccess) {
        h->owned.push_back(h->table);
        e = cudaMemcpy(h->table, table.data(), table.size() * 8, cudaMemcpyHostToDevice);
    }
    uint64_t at = kHeaderWords;
    for (int i = 0; i < 7 && e == cudaSuccess; i++) {
        *cnts[i] = counts[i];
        if (counts[i]) {
            e = cudaMalloc(dst[i], counts[i] * 8);
            if (e != cudaSuccess) break;
            h->owned.push_back(*dst[i]);
            e = cudaMemcpy(*dst[i], w + at, counts[i] * 8, cudaMemcpyHostToDevice);
        }
        at += counts[i];
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
    v.small_bits = (h->n_pil_words < (1ull << 26) && h->n_dict_words < (1ull << 26)) ? 1 : 0;
    v.key_kind = key_kind;
    v.string_seed = p.seed;
    I.device_bytes = (kTablePoints + 1) * 8 + 8 * (words - kHeaderWords);
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

phobic_status phobic_partition_sort(const uint64_t* d_hk, uint64_t n, uint64_t num_partitions, uint64_t* d_sorted,
                                    uint64_t* d_start, phobic_stream_t stream) {
    if (n == 0 || num_partitions == 0 || !d_hk || !d_sorted || !d_start) return PHOBIC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    ensure_pool();
    Arena tmp(st);
    void* scratch;
    uint32_t* err;
    CK(tmp.alloc(&scratch, sort_scratch_bytes(n, num_partitions)));
    CK(tmp.alloc(&err, 16));
    CK(cudaMemsetAsync(err, 0, 16, st));
    CK(launch_partition_sort(d_hk, 0, 0, n, num_partitions, d_sorted, d_start, scratch, err, st));
    uint32_t herr = 0;
    CK(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return herr ? PHOBIC_ERR_TIMEOUT : PHOBIC_OK;
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
