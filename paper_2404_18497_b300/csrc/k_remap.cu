// K7: remap of slots >= n onto free slots < n (alpha < 1), for every key set of
// a build in one launch per step.
//
// Section 5 ("Further Remarks") names PTHash's non-minimal trick.  The search
// runs on M = sum m_j > n slots.  Afterwards every occupied slot q >= n is sent
// to a free slot below n.  With F the free slots below n in increasing order
// and rank(q) the number of occupied slots in [n, q):
//     fs[q - n] = F[min(rank(q), |F| - 1)]      (fs = 0 when F is empty).
// A slot q >= n that no key occupies repeats the value of the next occupied
// slot, so fs is non-decreasing.  It is stored with Elias-Fano: l low bits per
// value; the high part in unary, with bit (fs_i >> l) + i set; and the position
// of every 64th one kept as a select sample.
//
// Each set's slots occupy bits [g0, g0 + M) of one global occupancy bitmap.
// Device steps: popcounts of the 32-bit words covering each set's [g0, g0 + n)
// (free slots) and [g0 + n, g0 + M) (occupied), flattened over all sets; two
// exclusive scans; compaction of F; the per-slot gather of fs; then the
// Elias-Fano words, written into each set's arrays.
#include "phobic_dev.cuh"
#include "phobic_kernels.cuh"

namespace phobic {

namespace {

// bits of word w of a u32 bitmap inside the global bit range [lo, hi);
// `want_zero` selects free slots instead of occupied ones
__device__ __forceinline__ uint32_t region_bits(const uint32_t* bm, uint64_t w, uint64_t lo, uint64_t hi, bool want_zero) {
    uint32_t v = bm[w];
    if (want_zero) v = ~v;
    const uint64_t b0 = w * 32;
    uint32_t mask = 0xFFFFFFFFu;
    if (b0 < lo) mask &= (lo - b0 >= 32) ? 0u : (0xFFFFFFFFu << (uint32_t)(lo - b0));
    if (b0 + 32 > hi) mask &= (hi <= b0) ? 0u : ((hi - b0 >= 32) ? 0xFFFFFFFFu : ((1u << (uint32_t)(hi - b0)) - 1));
    return v & mask;
}

__device__ __forceinline__ uint32_t find_set(const uint64_t* __restrict__ begin, uint32_t n, uint64_t t) {
    uint32_t lo = 0, hi = n;  // largest s with begin[s] <= t
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (__ldg(begin + mid) <= t) lo = mid; else hi = mid;
    }
    return lo;
}

// kind 0: free slots of [g0, g0 + n); kind 1: occupied slots of [g0 + n, g0 + M)
template <int kind>
__global__ void k_count_words(const uint32_t* __restrict__ bm, const RemapDesc* __restrict__ sets, uint32_t nsets,
                              const uint64_t* __restrict__ begin, uint32_t* __restrict__ cnt) {
    const uint64_t total = begin[nsets];
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t s = find_set(begin, nsets, t);
        const RemapDesc d = sets[s];
        const uint64_t lo = kind == 0 ? d.g0 : d.g0 + d.n;
        const uint64_t hi = kind == 0 ? d.g0 + d.n : d.g0 + d.M;
        const uint64_t w = (lo >> 5) + (t - begin[s]);
        cnt[t] = __popc(region_bits(bm, w, lo, hi, kind == 0));
    }
}

__device__ __forceinline__ unsigned long long scan_at(const unsigned long long* off, uint64_t i, uint64_t n,
                                                      const unsigned long long* total) {
    return i < n ? off[i] : *total;
}

// F: free slots below n (set-local positions), in order; only the first N are needed
__global__ void k_free_list(const uint32_t* __restrict__ bm, const RemapDesc* __restrict__ sets, uint32_t nsets,
                            const uint64_t* __restrict__ zbegin, const unsigned long long* __restrict__ zoff,
                            uint64_t* __restrict__ F) {
    const uint64_t total = zbegin[nsets];
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t s = find_set(zbegin, nsets, t);
        const RemapDesc d = sets[s];
        const uint64_t w = (d.g0 >> 5) + (t - zbegin[s]);
        uint32_t z = region_bits(bm, w, d.g0, d.g0 + d.n, true);
        unsigned long long r = zoff[t] - zoff[zbegin[s]];
        const uint64_t cap = d.M - d.n;
        while (z && r < cap) {
            const uint32_t b = __ffs(z) - 1;
            z &= z - 1;
            F[d.f_base + r++] = w * 32 + b - d.g0;
        }
    }
}

// fs[q - n] for q in [n, M) of every set (flattened: entry f_base + i of set s)
__global__ void k_fill_fs(const uint32_t* __restrict__ bm, const RemapDesc* __restrict__ sets, uint32_t nsets,
                          const uint64_t* __restrict__ fbegin, const uint64_t* __restrict__ tbegin,
                          const unsigned long long* __restrict__ toff, const unsigned long long* __restrict__ ttotal,
                          const uint64_t* __restrict__ F, uint64_t* __restrict__ fs) {
    const uint64_t total = fbegin[nsets];
    const uint64_t tw_total = tbegin[nsets];
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t s = find_set(fbegin, nsets, t);
        const RemapDesc d = sets[s];
        const uint64_t q = d.n + (t - d.f_base);  // set-local slot
        const uint64_t gb = d.g0 + q;             // global bit
        const uint64_t w = gb >> 5;
        const uint64_t lo = d.g0 + d.n;
        const uint64_t widx = tbegin[s] + (w - (lo >> 5));
        const unsigned long long base = scan_at(toff, tbegin[s], tw_total, ttotal);
        const unsigned long long nF = scan_at(toff, tbegin[s + 1], tw_total, ttotal) - base;
        const unsigned long long r = toff[widx] - base + __popc(region_bits(bm, w, lo, gb, false));
        fs[t] = nF ? F[d.f_base + (r < nF ? r : nF - 1)] : 0;
    }
}

__global__ void k_ef_low(const RemapDesc* __restrict__ sets, uint32_t nsets, const uint64_t* __restrict__ lbegin,
                         const uint64_t* __restrict__ fs, uint64_t* __restrict__ arena) {
    const uint64_t total = lbegin[nsets];
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t s = find_set(lbegin, nsets, t);
        const RemapDesc d = sets[s];
        const uint64_t k = t - lbegin[s];
        const uint32_t l = d.l;
        const uint64_t N = d.M - d.n;
        uint64_t acc = 0;
        if (l) {
            const uint64_t lmask = (1ull << l) - 1;
            const uint64_t wlo = k * 64, whi = wlo + 64, end = N * l;
            if (wlo < end) {
                const uint64_t hi = whi < end ? whi : end;
                const uint64_t i0 = wlo / l, i1 = (hi - 1) / l;
                for (uint64_t i = i0; i <= i1; i++) {
                    const uint64_t v = fs[d.f_base + i] & lmask, o = i * l;
                    acc |= o >= wlo ? (v << (o - wlo)) : (v >> (wlo - o));
                }
                const uint64_t b = hi - wlo;
                if (b < 64) acc &= (1ull << b) - 1;
            }
        }
        arena[d.low_dst + k] = acc;
    }
}

__global__ void k_ef_high(const RemapDesc* __restrict__ sets, uint32_t nsets, const uint64_t* __restrict__ fbegin,
                          const uint64_t* __restrict__ fs, uint64_t* __restrict__ arena) {
    const uint64_t total = fbegin[nsets];
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t s = find_set(fbegin, nsets, t);
        const RemapDesc d = sets[s];
        const uint64_t i = t - d.f_base;
        const uint64_t pos = (fs[t] >> d.l) + i;
        atomicOr((unsigned long long*)(arena + d.high_dst + (pos >> 6)), 1ull << (pos & 63));
        if ((i & 63) == 0) arena[d.samp_dst + (i >> 6)] = pos;
    }
}

unsigned grid_for(uint64_t work, unsigned threads) {
    uint64_t g = (work + threads - 1) / threads;
    if (g > 65535ull * 4) g = 65535ull * 4;
    return (unsigned)(g ? g : 1);
}

}  // namespace

size_t remap_scratch_bytes(uint64_t zwords, uint64_t twords, uint64_t ntotal) {
    size_t s = 0;
    s += (zwords + twords) * 4 + 32;  // counts
    s += (zwords + twords) * 8 + 32;  // scans
    s += scan_tiles_bytes(zwords) + scan_tiles_bytes(twords) + 32;
    s += (ntotal + 1) * 8;            // F
    s += (ntotal + 1) * 8;            // fs
    return s + 256;
}

cudaError_t launch_remap(const uint32_t* bm, const RemapDesc* d_sets, uint32_t nsets, const uint64_t* d_zbegin,
                         uint64_t zwords, const uint64_t* d_tbegin, uint64_t twords, const uint64_t* d_fbegin,
                         uint64_t ntotal, const uint64_t* d_lbegin, uint64_t lwords, uint64_t* arena, void* scratch,
                         cudaStream_t st) {
    unsigned char* p = static_cast<unsigned char*>(scratch);
    auto take = [&](size_t bytes) {
        void* r = p;
        p += (bytes + 15) & ~size_t(15);
        return r;
    };
    uint32_t* zc = (uint32_t*)take(zwords * 4 + 4);
    uint32_t* tc = (uint32_t*)take(twords * 4 + 4);
    unsigned long long* zoff = (unsigned long long*)take(zwords * 8 + 8);
    unsigned long long* toff = (unsigned long long*)take(twords * 8 + 8);
    unsigned long long* ztiles = (unsigned long long*)take(scan_tiles_bytes(zwords));
    unsigned long long* ttiles = (unsigned long long*)take(scan_tiles_bytes(twords));
    uint64_t* F = (uint64_t*)take((ntotal + 1) * 8);
    uint64_t* fs = (uint64_t*)take((ntotal + 1) * 8);

    k_count_words<0><<<grid_for(zwords, 256), 256, 0, st>>>(bm, d_sets, nsets, d_zbegin, zc);
    note_launches(1);
    k_count_words<1><<<grid_for(twords, 256), 256, 0, st>>>(bm, d_sets, nsets, d_tbegin, tc);
    note_launches(1);
    cudaError_t e;
    if ((e = exclusive_scan_u32(zc, zwords, zoff, ztiles, st)) != cudaSuccess) return e;
    if ((e = exclusive_scan_u32(tc, twords, toff, ttiles, st)) != cudaSuccess) return e;
    k_free_list<<<grid_for(zwords, 256), 256, 0, st>>>(bm, d_sets, nsets, d_zbegin, zoff, F);
    note_launches(1);
    k_fill_fs<<<grid_for(ntotal, 256), 256, 0, st>>>(bm, d_sets, nsets, d_fbegin, d_tbegin, toff,
                                                     scan_total(ttiles, twords), F, fs);
    note_launches(1);
    k_ef_low<<<grid_for(lwords, 256), 256, 0, st>>>(d_sets, nsets, d_lbegin, fs, arena);
    note_launches(1);
    k_ef_high<<<grid_for(ntotal, 256), 256, 0, st>>>(d_sets, nsets, d_fbegin, fs, arena);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace phobic
