// K5 + K6: partition offsets and interleaved pilot encoders.
//
// Offsets (Section 4, "Encoding the offsets of the partitions"): partition
// sizes are implicit as differences of consecutive offsets T_j, and each T_j is
// stored as its difference to the expectation E_j = floor(j Q / 2^32), with
// Q = floor(M 2^32 / N_P).  The differences are shifted by their minimum and
// bit-packed at a common width.
//
// Interleaved coding (Section 4.1): encoder b stores the pilot of bucket b of
// every partition.  The pilot matrix is already column-major, so column b is
// one contiguous run of N_P values.
//   IC-C (Compact): width = bit length of the column's largest pilot.
//   IC-D (Dictionary): the column's sorted distinct pilots, bit-packed at the
//   bit length of the largest, plus each partition's rank in that dictionary,
//   bit-packed at the bit length of (#distinct - 1).  The distinct values are
//   found by marking a presence bitmap over [0, max]; a rank is a prefix
//   popcount over that bitmap.
// Packing is a gather: each thread assembles one 64-bit output word from the
// values that overlap it.  Words shared by two columns use atomicOr.
#include "phobic_dev.cuh"
#include "phobic_kernels.cuh"

namespace phobic {

namespace {

constexpr uint64_t kMeta = (1ull << 56) - 1;

__device__ __forceinline__ uint64_t expectation(uint64_t j, uint64_t Q) {
    uint64_t lo = j * Q, hi = __umul64hi(j, Q);
    return (hi << 32) | (lo >> 32);
}

__global__ void __launch_bounds__(1024) k_offset_minmax(const uint64_t* __restrict__ T, uint64_t np, uint64_t Q,
                                                        long long* mm) {
    __shared__ long long smin[32], smax[32];
    long long lo = LLONG_MAX, hi = LLONG_MIN;
    for (uint64_t j = threadIdx.x; j <= np; j += blockDim.x) {
        long long d = (long long)(T[j] - expectation(j, Q));
        lo = min(lo, d);
        hi = max(hi, d);
    }
    for (int o = 16; o; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xFFFFFFFFu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xFFFFFFFFu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        smin[threadIdx.x >> 5] = lo;
        smax[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) {
            lo = min(lo, smin[w]);
            hi = max(hi, smax[w]);
        }
        lo = min(lo, smin[0]);
        hi = max(hi, smax[0]);
        mm[0] = lo;
        mm[1] = hi;
    }
}

// Assemble output word `word` (absolute word index) from values i in [0, count)
// placed at bit base + i*w; value(i) supplies the value.  Only bits of this
// column are produced; the caller combines columns.
template <class F>
__device__ __forceinline__ uint64_t gather_word(uint64_t word, uint64_t base, uint32_t w, uint64_t count, F value) {
    if (w == 0 || count == 0) return 0;
    const uint64_t wlo = word * 64, whi = wlo + 64;  // [wlo, whi)
    const uint64_t cend = base + count * w;
    uint64_t lo = wlo > base ? wlo : base;
    uint64_t hi = whi < cend ? whi : cend;
    if (lo >= hi) return 0;
    uint64_t i0 = (lo - base) / w, i1 = (hi - 1 - base) / w;
    uint64_t acc = 0;
    const uint64_t vmask = w == 64 ? ~0ull : ((1ull << w) - 1);
    for (uint64_t i = i0; i <= i1; i++) {
        uint64_t v = value(i) & vmask;
        uint64_t o = base + i * w;  // first bit of value i
        if (o >= wlo) {
            uint64_t sh = o - wlo;
            acc |= v << sh;  // sh < 64
        } else {
            uint64_t sh = wlo - o;  // 0 < sh < w <= 64
            acc |= v >> sh;
        }
    }
    // keep only the bits of [lo, hi)
    uint64_t a = lo - wlo, b = hi - wlo;  // 0 <= a < b <= 64
    uint64_t keep = (b == 64 ? ~0ull : ((1ull << b) - 1)) & ~((1ull << a) - 1);
    return acc & keep;
}

__global__ void k_offset_pack(const uint64_t* __restrict__ T, uint64_t np, uint64_t Q, int64_t dmin, uint32_t w,
                              uint64_t* __restrict__ words, uint64_t nwords) {
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < nwords; k += (uint64_t)gridDim.x * blockDim.x) {
        words[k] = gather_word(k, 0, w, np + 1, [&](uint64_t j) {
            return (uint64_t)((long long)(T[j] - expectation(j, Q)) - dmin);
        });
    }
}

__global__ void __launch_bounds__(256) k_column_max(const uint32_t* __restrict__ pilots, uint64_t np,
                                                    uint32_t* __restrict__ colmax) {
    __shared__ uint32_t sm[8];
    const uint32_t* col = pilots + (uint64_t)blockIdx.x * np;
    uint32_t mx = 0;
    for (uint64_t j = threadIdx.x; j < np; j += blockDim.x) mx = max(mx, __ldg(col + j));
    mx = __reduce_max_sync(0xFFFFFFFFu, mx);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < 8; i++) mx = max(mx, sm[i]);
        colmax[blockIdx.x] = mx;
    }
}

// column of flat thread index t: col_word_begin is a prefix sum over columns of
// the number of output words each column touches
__device__ __forceinline__ uint32_t find_column(const uint64_t* __restrict__ begin, uint32_t ncols, uint64_t t) {
    uint32_t lo = 0, hi = ncols;  // answer in [0, ncols)
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (__ldg(begin + mid) <= t) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void k_compact_pack(const uint32_t* __restrict__ pilots, uint64_t np, uint32_t B,
                               const uint64_t* __restrict__ col_meta, const uint64_t* __restrict__ col_word_begin,
                               uint64_t* __restrict__ words) {
    const uint64_t total = col_word_begin[B];
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total; t += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t b = find_column(col_word_begin, B, t);
        uint64_t meta = __ldg(col_meta + b);
        uint64_t base = meta & kMeta;
        uint32_t w = (uint32_t)(meta >> 56);
        uint64_t word = (base >> 6) + (t - col_word_begin[b]);
        const uint32_t* col = pilots + (uint64_t)b * np;
        uint64_t v = gather_word(word, base, w, np, [&](uint64_t j) { return (uint64_t)__ldg(col + j); });
        uint64_t cend = base + np * w;
        bool interior = word * 64 >= base && word * 64 + 64 <= cend;
        if (interior) words[word] = v;
        else if (v) atomicOr((unsigned long long*)(words + word), (unsigned long long)v);
    }
}

__global__ void k_dict_mark(const uint32_t* __restrict__ pilots, uint64_t np, uint32_t B,
                            const uint64_t* __restrict__ bm_base, uint64_t* __restrict__ bitmaps) {
    const uint64_t total = np * B;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total; t += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t b = (uint32_t)(t / np);
        uint32_t v = __ldg(pilots + t);
        atomicOr((unsigned long long*)(bitmaps + bm_base[b] + (v >> 6)), 1ull << (v & 63));
    }
}

// one block per column: exclusive popcount prefix of its bitmap words
__global__ void __launch_bounds__(1024) k_dict_rank(const uint64_t* __restrict__ bm_base,
                                                    uint64_t* __restrict__ bitmaps_rank,
                                                    const uint64_t* __restrict__ bitmaps, uint64_t* __restrict__ K) {
    __shared__ uint32_t warp_sums[32];
    __shared__ unsigned long long carry_s;
    const uint32_t b = blockIdx.x;
    const uint64_t w0 = bm_base[b], w1 = bm_base[b + 1];
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry_s = 0;
    __syncthreads();
    for (uint64_t c = w0; c < w1; c += 1024) {
        uint64_t i = c + tid;
        uint32_t v = i < w1 ? __popcll(bitmaps[i]) : 0;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= (uint32_t)o) x += y;
        }
        if (lane == 31) warp_sums[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t s = warp_sums[lane], z = s;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xFFFFFFFFu, z, o);
                if (lane >= (uint32_t)o) z += y;
            }
            warp_sums[lane] = z - s;
        }
        __syncthreads();
        unsigned long long carry = carry_s;
        if (i < w1) bitmaps_rank[i] = carry + warp_sums[warp] + x - v;
        __syncthreads();
        if (tid == 1023) carry_s = carry + warp_sums[31] + x;
        __syncthreads();
    }
    if (tid == 0) K[b] = carry_s;
}

__device__ __forceinline__ uint64_t dict_rank_of(uint32_t v, uint64_t wbase, const uint64_t* __restrict__ bitmaps,
                                                 const uint64_t* __restrict__ bitmaps_rank) {
    uint64_t wi = wbase + (v >> 6);
    uint64_t below = (v & 63) ? (__ldg(bitmaps + wi) & ((1ull << (v & 63)) - 1)) : 0;
    return __ldg(bitmaps_rank + wi) + __popcll(below);
}

__global__ void k_dict_pack_ranks(const uint32_t* __restrict__ pilots, uint64_t np, uint32_t B,
                                  const uint64_t* __restrict__ bm_base, const uint64_t* __restrict__ bitmaps,
                                  const uint64_t* __restrict__ bitmaps_rank, const uint64_t* __restrict__ col_meta,
                                  const uint64_t* __restrict__ word_begin, uint64_t* __restrict__ words) {
    const uint64_t total = word_begin[B];
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total; t += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t b = find_column(word_begin, B, t);
        uint64_t meta = __ldg(col_meta + 2 * b);
        uint64_t base = meta & kMeta;
        uint32_t w = (uint32_t)(meta >> 56);
        uint64_t word = (base >> 6) + (t - word_begin[b]);
        const uint32_t* col = pilots + (uint64_t)b * np;
        const uint64_t wb = bm_base[b];
        uint64_t v = gather_word(word, base, w, np,
                                 [&](uint64_t j) { return dict_rank_of(__ldg(col + j), wb, bitmaps, bitmaps_rank); });
        uint64_t cend = base + np * w;
        bool interior = word * 64 >= base && word * 64 + 64 <= cend;
        if (interior) words[word] = v;
        else if (v) atomicOr((unsigned long long*)(words + word), (unsigned long long)v);
    }
}

// dictionary entries: thread per bitmap word; each set bit v with rank r writes
// v at bit dbase + r * dw
__global__ void k_dict_pack_values(uint32_t B, const uint64_t* __restrict__ bm_base,
                                   const uint64_t* __restrict__ bitmaps, const uint64_t* __restrict__ bitmaps_rank,
                                   const uint64_t* __restrict__ col_meta, uint64_t* __restrict__ words) {
    const uint64_t total = bm_base[B];
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total; t += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t bits = bitmaps[t];
        if (!bits) continue;
        uint32_t b = find_column(bm_base, B, t);
        uint64_t meta = __ldg(col_meta + 2 * b + 1);
        uint64_t base = meta & kMeta;
        uint32_t w = (uint32_t)(meta >> 56);
        uint64_t r = bitmaps_rank[t];
        uint64_t v0 = (t - bm_base[b]) * 64;
        while (bits) {
            uint32_t bit = __ffsll((long long)bits) - 1;
            bits &= bits - 1;
            uint64_t v = v0 + bit;
            if (w) {
                uint64_t o = base + r * w;
                uint64_t wi = o >> 6;
                uint32_t sh = (uint32_t)(o & 63);
                atomicOr((unsigned long long*)(words + wi), (unsigned long long)(v << sh));
                if (sh + w > 64) atomicOr((unsigned long long*)(words + wi + 1), (unsigned long long)(v >> (64 - sh)));
            }
            r++;
        }
    }
}

unsigned grid_for(uint64_t work, unsigned threads) {
    uint64_t g = (work + threads - 1) / threads;
    if (g > 65535ull * 4) g = 65535ull * 4;
    return (unsigned)(g ? g : 1);
}

}  // namespace

cudaError_t launch_offset_minmax(const uint64_t* T, uint64_t np, uint64_t Q, long long* mm, cudaStream_t stream) {
    k_offset_minmax<<<1, 1024, 0, stream>>>(T, np, Q, mm);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_offset_pack(const uint64_t* T, uint64_t np, uint64_t Q, int64_t dmin, uint32_t w, uint64_t* words,
                               uint64_t nwords, cudaStream_t stream) {
    k_offset_pack<<<grid_for(nwords, 256), 256, 0, stream>>>(T, np, Q, dmin, w, words, nwords);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_column_max(const uint32_t* pilots, uint64_t np, uint32_t B, uint32_t* colmax, cudaStream_t stream) {
    k_column_max<<<B, 256, 0, stream>>>(pilots, np, colmax);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_compact_pack(const uint32_t* pilots, uint64_t np, uint32_t B, const uint64_t* col_meta,
                                const uint64_t* col_word_begin, uint64_t* words, uint64_t total_colwords,
                                cudaStream_t stream) {
    k_compact_pack<<<grid_for(total_colwords, 256), 256, 0, stream>>>(pilots, np, B, col_meta, col_word_begin, words);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_dict_mark(const uint32_t* pilots, uint64_t np, uint32_t B, const uint64_t* bm_base,
                             uint64_t* bitmaps, cudaStream_t stream) {
    k_dict_mark<<<grid_for(np * B, 256), 256, 0, stream>>>(pilots, np, B, bm_base, bitmaps);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_dict_rank(const uint64_t* bm_base, uint32_t B, uint64_t* bitmaps_rank, const uint64_t* bitmaps,
                             uint64_t* K, cudaStream_t stream) {
    k_dict_rank<<<B, 1024, 0, stream>>>(bm_base, bitmaps_rank, bitmaps, K);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_dict_pack(const uint32_t* pilots, uint64_t np, uint32_t B, const uint64_t* bm_base,
                             const uint64_t* bitmaps, const uint64_t* bitmaps_rank, const uint64_t* col_meta,
                             const uint64_t* rank_word_begin, uint64_t* rank_words, uint64_t rank_colwords,
                             const uint64_t* /*dict_word_begin*/, uint64_t* dict_words, uint64_t bitmap_words,
                             cudaStream_t stream) {
    k_dict_pack_ranks<<<grid_for(rank_colwords, 256), 256, 0, stream>>>(pilots, np, B, bm_base, bitmaps, bitmaps_rank,
                                                                        col_meta, rank_word_begin, rank_words);
    note_launches(1);
    k_dict_pack_values<<<grid_for(bitmap_words, 256), 256, 0, stream>>>(B, bm_base, bitmaps, bitmaps_rank, col_meta,
                                                                        dict_words);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace phobic
