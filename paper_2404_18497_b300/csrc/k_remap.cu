// K7: remap of slots >= n onto free slots < n (alpha < 1).
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
// Device steps: popcounts per 32-bit word of the occupancy bitmap, exclusive
// scans (three-phase: block sums, scan of the sums, block scan with carry),
// then compaction of F and the per-slot gather of fs.  The Elias-Fano words
// are built last.
#include "phobic_dev.cuh"
#include "phobic_kernels.cuh"

namespace phobic {

namespace {

constexpr uint64_t kScanTile = kScanTileItems;

// count of bits in word w of the region [lo, hi) of a u32 bitmap; `want_zero`
// counts free slots instead of occupied ones
__device__ __forceinline__ uint32_t region_bits(const uint32_t* bm, uint64_t w, uint64_t lo, uint64_t hi, bool want_zero) {
    uint32_t v = bm[w];
    if (want_zero) v = ~v;
    uint64_t b0 = w * 32;
    uint32_t mask = 0xFFFFFFFFu;
    if (b0 < lo) mask &= 0xFFFFFFFFu << (uint32_t)(lo - b0);
    if (b0 + 32 > hi) mask &= (hi - b0 >= 32) ? 0xFFFFFFFFu : ((1u << (uint32_t)(hi - b0)) - 1);
    return v & mask;
}

__global__ void __launch_bounds__(256) k_count_words(const uint32_t* __restrict__ bm, uint64_t w0, uint64_t nw,
                                                              uint64_t lo, uint64_t hi, int want_zero,
                                                              uint32_t* __restrict__ cnt) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nw; i += (uint64_t)gridDim.x * blockDim.x)
        cnt[i] = __popc(region_bits(bm, w0 + i, lo, hi, want_zero != 0));
}

// F: free slots below n, in order (only the first cap entries are needed)
__global__ void k_free_list(const uint32_t* __restrict__ bm, uint64_t nw, uint64_t n,
                            const unsigned long long* __restrict__ zoff, uint64_t* __restrict__ F, uint64_t cap) {
    for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < nw; w += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t z = region_bits(bm, w, 0, n, true);
        unsigned long long r = zoff[w];
        while (z && r < cap) {
            uint32_t b = __ffs(z) - 1;
            z &= z - 1;
            F[r++] = w * 32 + b;
        }
    }
}

// fs[q - n] for q in [n, M)
__global__ void k_fill_fs(const uint32_t* __restrict__ bm, uint64_t n, uint64_t M, uint64_t w0,
                          const unsigned long long* __restrict__ toff, const unsigned long long* __restrict__ ttotal,
                          const uint64_t* __restrict__ F, uint64_t* __restrict__ fs) {
    const unsigned long long nF = *ttotal;
    for (uint64_t q = n + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < M; q += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t w = q >> 5;
        uint32_t below = region_bits(bm, w, n, q, false);
        unsigned long long r = toff[w - w0] + __popc(below);
        fs[q - n] = nF ? F[r < nF ? r : nF - 1] : 0;
    }
}

__global__ void k_ef_low(const uint64_t* __restrict__ fs, uint64_t N, uint32_t l, uint64_t* __restrict__ low,
                         uint64_t nwords) {
    const uint64_t lmask = l ? ((1ull << l) - 1) : 0;
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < nwords; k += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t acc = 0;
        if (l) {
            uint64_t wlo = k * 64, whi = wlo + 64, end = N * l;
            if (wlo < end) {
                uint64_t hi = whi < end ? whi : end;
                uint64_t i0 = wlo / l, i1 = (hi - 1) / l;
                for (uint64_t i = i0; i <= i1; i++) {
                    uint64_t v = fs[i] & lmask, o = i * l;
                    acc |= o >= wlo ? (v << (o - wlo)) : (v >> (wlo - o));
                }
                uint64_t b = hi - wlo;
                if (b < 64) acc &= (1ull << b) - 1;
            }
        }
        low[k] = acc;
    }
}

__global__ void k_ef_high(const uint64_t* __restrict__ fs, uint64_t N, uint32_t l, uint64_t* __restrict__ high,
                          uint64_t* __restrict__ samples) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t pos = (fs[i] >> l) + i;
        atomicOr((unsigned long long*)(high + (pos >> 6)), 1ull << (pos & 63));
        if ((i & 63) == 0) samples[i >> 6] = pos;
    }
}

unsigned grid_for(uint64_t work, unsigned threads) {
    uint64_t g = (work + threads - 1) / threads;
    if (g > 65535ull * 4) g = 65535ull * 4;
    return (unsigned)(g ? g : 1);
}

}  // namespace

size_t remap_scratch_bytes(uint64_t n, uint64_t M) {
    uint64_t nw0 = (n + 31) / 32;                       // words of [0, n)
    uint64_t w0 = n >> 5, nw1 = ((M - 1) >> 5) - w0 + 1; // words of [n, M)
    uint64_t N = M - n;
    size_t s = 0;
    s += (nw0 + nw1) * 4 + 16;                          // counts
    s += (nw0 + nw1) * 8 + 16;                          // scans
    s += 2 * ((nw0 + kScanTile - 1) / kScanTile + (nw1 + kScanTile - 1) / kScanTile + 4) * 8; // tile sums
    s += (N + 1) * 8;                                   // F
    return s + 256;
}

cudaError_t launch_remap(const uint32_t* taken_bits, uint64_t n, uint64_t M, uint32_t l, uint64_t* fs,
                         uint64_t* ef_low, uint64_t low_nwords, uint64_t* ef_high, uint64_t high_nwords,
                         uint64_t* ef_samples, void* scratch, cudaStream_t st) {
    const uint64_t N = M - n;
    const uint64_t nw0 = (n + 31) / 32;
    const uint64_t w0 = n >> 5, nw1 = ((M - 1) >> 5) - w0 + 1;
    unsigned char* p = static_cast<unsigned char*>(scratch);
    auto take = [&](size_t bytes) {
        void* r = p;
        p += (bytes + 15) & ~size_t(15);
        return r;
    };
    uint32_t* zc = (uint32_t*)take(nw0 * 4);
    uint32_t* tc = (uint32_t*)take(nw1 * 4);
    unsigned long long* zoff = (unsigned long long*)take(nw0 * 8);
    unsigned long long* toff = (unsigned long long*)take(nw1 * 8);
    unsigned long long* ztiles = (unsigned long long*)take(((nw0 + kScanTile - 1) / kScanTile + 2) * 8);
    unsigned long long* ttiles = (unsigned long long*)take(((nw1 + kScanTile - 1) / kScanTile + 2) * 8);
    uint64_t* F = (uint64_t*)take((N + 1) * 8);

    k_count_words<<<grid_for(nw0, 256), 256, 0, st>>>(taken_bits, 0, nw0, 0, n, 1, zc);
    note_launches(1);
    k_count_words<<<grid_for(nw1, 256), 256, 0, st>>>(taken_bits, w0, nw1, n, M, 0, tc);
    note_launches(1);
    cudaError_t e;
    if ((e = exclusive_scan_u32(zc, nw0, zoff, ztiles, st)) != cudaSuccess) return e;
    if ((e = exclusive_scan_u32(tc, nw1, toff, ttiles, st)) != cudaSuccess) return e;
    k_free_list<<<grid_for(nw0, 256), 256, 0, st>>>(taken_bits, nw0, n, zoff, F, N);
    note_launches(1);
    k_fill_fs<<<grid_for(N, 256), 256, 0, st>>>(taken_bits, n, M, w0, toff, scan_total(ttiles, nw1), F, fs);
    note_launches(1);
    if ((e = cudaMemsetAsync(ef_high, 0, high_nwords * 8, st)) != cudaSuccess) return e;
    k_ef_low<<<grid_for(low_nwords, 256), 256, 0, st>>>(fs, N, l, ef_low, low_nwords);
    note_launches(1);
    k_ef_high<<<grid_for(N, 256), 256, 0, st>>>(fs, N, l, ef_high, ef_samples);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace phobic
