// K5 + K6: partition offsets and interleaved pilot encoders, for every key set
// of a build in one launch per step.
//
// Offsets (Section 4, "Encoding the offsets of the partitions"): partition
// sizes are implicit as differences of consecutive offsets T_j, and each T_j is
// stored as its difference to the expectation E_j = floor(j Q / 2^32), with
// Q = floor(M 2^32 / N_P).  The differences are shifted by their minimum and
// bit-packed at a common width.
//
// Interleaved coding (Section 4.1): encoder b stores the pilot of bucket b of
// every partition.  The pilot matrix of a set is column-major, so column b is
// one contiguous run of N_P values.
//   IC-C (Compact): width = bit length of the column's largest pilot.
//   IC-D (Dictionary): the column's sorted distinct pilots, bit-packed at the
//   bit length of the largest, plus each partition's rank in that dictionary,
//   bit-packed at the bit length of (#distinct - 1).  The distinct values are
//   found by marking a presence bitmap over [0, max]; a rank is a prefix
//   popcount over that bitmap.
//   IC-R (Golomb-Rice, parameter l by Kiely's rule from the column mean): the
//   low l bits of each pilot packed at width l (the IC-C packer with width l);
//   the rest in unary, the pilot of partition j setting bit
//   j + sum_{i <= j} (v_i >> l) of the column's unary bits; and that position
//   for every 64th partition as a select sample.
//   IC-EF (Elias-Fano over each column's prefix sums E_j, l = floor(log2((E_last
//   + 1) / N_P)) low bits): the low bits of E_j packed at width l, bit
//   j + (E_j >> l) set in the high part, and the same select samples.
// Columns of all sets are described by ColDesc records; packing is a gather in
// which each thread assembles one 64-bit output word from the values that
// overlap it (atomicOr where two columns share a word).
#include "phobic_dev.cuh"
#include "phobic_kernels.cuh"

namespace phobic {

namespace {

// Assemble output word `word` (index inside the array) from values i in
// [0, count) placed at bit base + i*w; value(i) supplies the value.  Only this
// column's bits are produced.
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
        if (o >= wlo)
            acc |= v << (o - wlo);  // shift < 64
        else
            acc |= v >> (wlo - o);  // 0 < shift < w <= 64
    }
    uint64_t a = lo - wlo, b = hi - wlo;  // 0 <= a < b <= 64
    uint64_t keep = (b == 64 ? ~0ull : ((1ull << b) - 1)) & ~((1ull << a) - 1);
    return acc & keep;
}

// largest index c in [0, n) with begin[c] <= t (begin non-decreasing, begin[0] = 0)
__device__ __forceinline__ uint32_t find_item(const uint64_t* __restrict__ begin, uint32_t n, uint64_t t) {
    uint32_t lo = 0, hi = n;
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (__ldg(begin + mid) <= t) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ void put_word(uint64_t* words, uint64_t word, uint64_t v, bool interior) {
    if (interior)
        words[word] = v;
    else if (v)
        atomicOr((unsigned long long*)(words + word), (unsigned long long)v);
}

// ---------------------------------------------------------------- offsets ---
__global__ void k_minmax_init(long long* __restrict__ mm, uint32_t nsets) {
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < nsets) {
        mm[2 * s] = LLONG_MAX;
        mm[2 * s + 1] = LLONG_MIN;
    }
}

// min and max over j of D_j = T_j - T_0 - floor(j Q / 2^32) for every set.  The
// blocks serve the sets round-robin (block b takes set b mod nsets), so that a
// single large set is spread over the whole grid; partial results meet in mm
// through 64-bit atomics (set up by k_minmax_init).
__global__ void __launch_bounds__(256) k_offset_minmax(const uint64_t* __restrict__ T,
                                                       const OffDesc* __restrict__ sets, uint32_t nsets,
                                                       long long* __restrict__ mm) {
    __shared__ long long smin[8], smax[8];
    const uint32_t s = blockIdx.x % nsets;
    const uint32_t part = blockIdx.x / nsets;
    const uint32_t nparts = (gridDim.x - s + nsets - 1) / nsets;  // blocks that serve set s
    const OffDesc d = sets[s];
    const uint64_t T0 = T[d.part_base];
    long long lo = LLONG_MAX, hi = LLONG_MIN;
    for (uint64_t j = (uint64_t)part * blockDim.x + threadIdx.x; j <= d.np; j += (uint64_t)nparts * blockDim.x) {
        const long long v = (long long)(T[d.part_base + j] - T0 - offset_expectation(j, d.Q));
        lo = min(lo, v);
        hi = max(hi, v);
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
        for (int w = 1; w < 8; w++) {
            lo = min(lo, smin[w]);
            hi = max(hi, smax[w]);
        }
        atomicMin(mm + 2 * s, lo);
        atomicMax(mm + 2 * s + 1, hi);
    }
}

__global__ void k_offset_pack(const uint64_t* __restrict__ T, const OffDesc* __restrict__ sets, uint32_t nsets,
                              const uint64_t* __restrict__ word_begin, uint64_t* __restrict__ arena) {
    const uint64_t total = word_begin[nsets];
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t s = find_item(word_begin, nsets, t);
        const OffDesc d = sets[s];
        const uint64_t word = t - word_begin[s];
        const uint64_t T0 = T[d.part_base];
        arena[d.dst_word + word] = gather_word(word, 0, d.width, d.np + 1, [&](uint64_t j) {
            return (uint64_t)((long long)(T[d.part_base + j] - T0 - offset_expectation(j, d.Q)) - d.dmin);
        });
    }
}

// ---------------------------------------------------------------- columns ---
// Largest pilot (and sum) of every column.  A column is split into chunks of
// kColChunk values, one block per (column, chunk), so that a few long columns
// still fill the GPU; chunks meet in colmax / colsum through atomics (both
// cleared before the launch).
constexpr uint32_t kColChunk = 8192;
__global__ void __launch_bounds__(256) k_column_max(const uint32_t* __restrict__ pilots,
                                                    const ColDesc* __restrict__ cols, uint32_t ncols,
                                                    uint32_t chunks, uint32_t* __restrict__ colmax,
                                                    unsigned long long* __restrict__ colsum) {
    __shared__ uint32_t sm[8];
    __shared__ unsigned long long ss[8];
    const uint64_t items = (uint64_t)ncols * chunks;
    for (uint64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const uint32_t c = (uint32_t)(it / chunks);
        const uint64_t j0 = (it % chunks) * (uint64_t)kColChunk;
        const ColDesc d = cols[c];
        if (j0 >= d.count) continue;  // the same for the whole block
        const uint64_t j1 = d.count - j0 < kColChunk ? d.count : j0 + kColChunk;
        uint32_t mx = 0;
        unsigned long long sum = 0;
        for (uint64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
            const uint32_t v = __ldg(pilots + d.src + j);
            mx = max(mx, v);
            sum += v;
        }
        mx = __reduce_max_sync(0xFFFFFFFFu, mx);
        for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
        if ((threadIdx.x & 31) == 0) {
            sm[threadIdx.x >> 5] = mx;
            ss[threadIdx.x >> 5] = sum;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int i = 1; i < 8; i++) {
                mx = max(mx, sm[i]);
                sum += ss[i];
            }
            atomicMax(colmax + c, mx);
            if (colsum) atomicAdd(colsum + c, sum);
        }
        __syncthreads();
    }
}

// IC-R: per column, the sum of (pilot >> l)
__global__ void __launch_bounds__(256) k_rice_unary_len(const uint32_t* __restrict__ pilots,
                                                        const ColDesc* __restrict__ cols, uint32_t ncols,
                                                        uint64_t* __restrict__ hlen) {
    __shared__ unsigned long long ss[8];
    for (uint32_t c = blockIdx.x; c < ncols; c += gridDim.x) {
        const ColDesc d = cols[c];
        unsigned long long sum = 0;
        for (uint64_t j = threadIdx.x; j < d.count; j += blockDim.x) sum += __ldg(pilots + d.src + j) >> d.width;
        for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
        if ((threadIdx.x & 31) == 0) ss[threadIdx.x >> 5] = sum;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int i = 1; i < 8; i++) sum += ss[i];
            hlen[c] = sum;
        }
        __syncthreads();
    }
}

// IC-R and IC-EF: one block per column, an inclusive block scan over the
// column's partitions, chunk by chunk with a carry.
//   IC-R (kEF = false): scan of q_j = pilot >> l; value j sets bit
//   j + sum_{i <= j} q_i of the unary bits (its low part is packed separately).
//   IC-EF (kEF = true): scan of the pilots themselves, E_j = sum_{i <= j} v_i;
//   value j writes the low l bits of E_j at bit base + j l of the low array and
//   sets bit j + (E_j >> l) of the high bits.
// Bits go in with atomicOr (neighbours share words); every 64th set bit's
// position becomes a select sample.  A mono encoder's column continues its
// set's single sequence from value index idx0 with the scan carried in at sum0,
// so value i = idx0 + j sets bit i + (sum0 + incl) (Rice) or i + ((sum0 + incl)
// >> l) (Elias-Fano), and samples go by the global index i.
template <bool kEF>
__global__ void __launch_bounds__(1024) k_column_unary(const uint32_t* __restrict__ pilots,
                                                       const ColDesc* __restrict__ cols, uint32_t ncols,
                                                       uint64_t* __restrict__ arena) {
    __shared__ unsigned long long warp_sums[32];
    __shared__ unsigned long long carry_s;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (uint32_t c = blockIdx.x; c < ncols; c += gridDim.x) {
        const ColDesc d = cols[c];
        if (d.samp_dst_word == ~0ull) continue;  // a Compact column of a mixture
        uint64_t* high = arena + d.hi_dst_word;
        uint64_t* low = arena + d.dst_word;
        uint32_t* samples = reinterpret_cast<uint32_t*>(arena + d.samp_dst_word) + d.samp_base;
        if (tid == 0) carry_s = 0;
        __syncthreads();
        for (uint64_t j0 = 0; j0 < d.count; j0 += 1024) {
            const uint64_t j = j0 + tid;
            const uint32_t v = j < d.count ? __ldg(pilots + d.src + j) : 0u;
            const unsigned long long q = kEF ? (unsigned long long)v : (unsigned long long)(v >> d.width);
            unsigned long long x = q;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
                if (lane >= (uint32_t)o) x += y;
            }
            if (lane == 31) warp_sums[warp] = x;
            __syncthreads();
            if (warp == 0) {
                const unsigned long long s = warp_sums[lane];
                unsigned long long z = s;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, z, o);
                    if (lane >= (uint32_t)o) z += y;
                }
                warp_sums[lane] = z - s;  // exclusive prefix of the warp totals
            }
            __syncthreads();
            const unsigned long long carry = carry_s;
            if (j < d.count) {
                const uint64_t incl = d.sum0 + carry + warp_sums[warp] + x;  // inclusive sum
                const uint64_t i = d.idx0 + j;
                uint64_t pos;
                if (kEF) {
                    pos = i + (incl >> d.width);
                    if (d.width) {
                        const uint64_t lv = incl & ((1ull << d.width) - 1);
                        const uint64_t o = d.base + j * d.width;
                        const uint32_t sh = (uint32_t)(o & 63);
                        atomicOr((unsigned long long*)(low + (o >> 6)), (unsigned long long)(lv << sh));
                        if (sh + d.width > 64)
                            atomicOr((unsigned long long*)(low + (o >> 6) + 1), (unsigned long long)(lv >> (64 - sh)));
                    }
                } else {
                    pos = i + incl;
                }
                const uint64_t bit = d.hi_base + pos;
                atomicOr((unsigned long long*)(high + (bit >> 6)), 1ull << (bit & 63));
                if ((i & 63) == 0) samples[i >> 6] = (uint32_t)pos;
            }
            __syncthreads();
            if (tid == 1023) carry_s = carry + warp_sums[31] + x;
            __syncthreads();
        }
    }
}

__device__ __forceinline__ uint64_t dict_rank_of(uint32_t v, uint64_t wbase, const uint64_t* __restrict__ bitmaps,
                                                 const uint64_t* __restrict__ bitmaps_rank) {
    const uint64_t wi = wbase + (v >> 6);
    const uint64_t below = (v & 63) ? (__ldg(bitmaps + wi) & ((1ull << (v & 63)) - 1)) : 0;
    return __ldg(bitmaps_rank + wi) + __popcll(below);
}

// IC-C data (kRanks = false) or IC-D ranks (kRanks = true) of every column
template <bool kRanks>
__global__ void k_pack_columns(const uint32_t* __restrict__ pilots, const ColDesc* __restrict__ cols, uint32_t ncols,
                               const uint64_t* __restrict__ word_begin, const uint64_t* __restrict__ bitmaps,
                               const uint64_t* __restrict__ bitmaps_rank, uint64_t* __restrict__ arena) {
    const uint64_t total = word_begin[ncols];
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t c = find_item(word_begin, ncols, t);
        const ColDesc d = cols[c];
        const uint64_t word = (d.base >> 6) + (t - word_begin[c]);
        const uint32_t* col = pilots + d.src;
        uint64_t v;
        if (kRanks)
            v = gather_word(word, d.base, d.width, d.count,
                            [&](uint64_t j) { return dict_rank_of(__ldg(col + j), d.bm_base, bitmaps, bitmaps_rank); });
        else
            v = gather_word(word, d.base, d.width, d.count, [&](uint64_t j) { return (uint64_t)__ldg(col + j); });
        const uint64_t cend = d.base + d.count * d.width;
        put_word(arena + d.dst_word, word, v, word * 64 >= d.base && word * 64 + 64 <= cend);
    }
}

// IC-D presence bitmaps: bit v of column c's bitmap is set when v occurs.  The
// low kMarkWords words of the column's bitmap are gathered in shared memory
// first (small pilots are by far the most frequent, and a mono dictionary's
// columns all mark one bitmap) and OR-ed into it once per non-zero word.
constexpr uint32_t kMarkWords = 2048;  // 64-bit words: pilots < 131072
__global__ void __launch_bounds__(256) k_dict_mark(const uint32_t* __restrict__ pilots,
                                                   const ColDesc* __restrict__ cols, uint32_t ncols,
                                                   uint64_t* __restrict__ bitmaps) {
    __shared__ uint32_t sbm[2 * kMarkWords];
    for (uint32_t c = blockIdx.x; c < ncols; c += gridDim.x) {
        const ColDesc d = cols[c];
        const uint32_t sw = d.bm_words < kMarkWords ? (uint32_t)d.bm_words : kMarkWords;  // staged words
        for (uint32_t i = threadIdx.x; i < 2 * sw; i += blockDim.x) sbm[i] = 0;
        __syncthreads();
        for (uint64_t j = threadIdx.x; j < d.count; j += blockDim.x) {
            const uint32_t v = __ldg(pilots + d.src + j);
            if ((v >> 6) < sw)
                atomicOr(&sbm[v >> 5], 1u << (v & 31));
            else
                atomicOr((unsigned long long*)(bitmaps + d.bm_base + (v >> 6)), 1ull << (v & 63));
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < sw; i += blockDim.x) {
            const uint64_t w = (uint64_t)sbm[2 * i] | ((uint64_t)sbm[2 * i + 1] << 32);
            if (w) atomicOr((unsigned long long*)(bitmaps + d.bm_base + i), (unsigned long long)w);
        }
        __syncthreads();
    }
}

// one block per column: exclusive popcount prefix of its bitmap words, and the
// number of distinct values K
__global__ void __launch_bounds__(1024) k_dict_rank(const ColDesc* __restrict__ cols, uint32_t ncols,
                                                    uint64_t* __restrict__ bitmaps_rank,
                                                    const uint64_t* __restrict__ bitmaps, uint64_t* __restrict__ K) {
    __shared__ uint32_t warp_sums[32];
    __shared__ unsigned long long carry_s;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (uint32_t c = blockIdx.x; c < ncols; c += gridDim.x) {
        const uint64_t w0 = cols[c].bm_base, w1 = w0 + cols[c].bm_words;
        if (tid == 0) carry_s = 0;
        __syncthreads();
        for (uint64_t cc = w0; cc < w1; cc += 1024) {
            uint64_t i = cc + tid;
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
        if (tid == 0) K[c] = carry_s;
        __syncthreads();
    }
}

// IC-D dictionaries: thread per bitmap word; each set bit v with rank r writes
// v at bit dict_base + r * dict_width of its set's dictionary array
__global__ void k_dict_pack_values(const ColDesc* __restrict__ cols, uint32_t ncols,
                                   const uint64_t* __restrict__ bm_begin, const uint64_t* __restrict__ bitmaps,
                                   const uint64_t* __restrict__ bitmaps_rank, uint64_t* __restrict__ arena) {
    const uint64_t total = bm_begin[ncols];
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total; t += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t bits = bitmaps[t];
        if (!bits) continue;
        const uint32_t c = find_item(bm_begin, ncols, t);
        const ColDesc d = cols[c];
        const uint32_t w = d.dict_width;
        uint64_t* words = arena + d.dict_dst_word;
        uint64_t r = bitmaps_rank[t];
        const uint64_t v0 = (t - d.bm_base) * 64;
        while (bits) {
            const uint32_t bit = __ffsll((long long)bits) - 1;
            bits &= bits - 1;
            const uint64_t v = v0 + bit;
            if (w) {
                const uint64_t o = d.dict_base + r * w;
                const uint64_t wi = o >> 6;
                const uint32_t sh = (uint32_t)(o & 63);
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

unsigned grid_items(uint64_t items) { return (unsigned)(items < 65535ull * 4 ? (items ? items : 1) : 65535ull * 4); }

}  // namespace

cudaError_t launch_offset_minmax(const uint64_t* T, const OffDesc* sets, uint32_t nsets, long long* mm,
                                 cudaStream_t stream) {
    if (nsets == 0) return cudaSuccess;
    k_minmax_init<<<(nsets + 255) / 256, 256, 0, stream>>>(mm, nsets);
    const uint32_t grid = nsets > 1024 ? nsets : 1024;  // at least one block per set
    k_offset_minmax<<<grid, 256, 0, stream>>>(T, sets, nsets, mm);
    note_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_offset_pack(const uint64_t* T, const OffDesc* sets, uint32_t nsets, const uint64_t* word_begin,
                               uint64_t total_words, uint64_t* arena, cudaStream_t stream) {
    k_offset_pack<<<grid_for(total_words, 256), 256, 0, stream>>>(T, sets, nsets, word_begin, arena);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_column_max(const uint32_t* pilots, const ColDesc* cols, uint32_t ncols, uint64_t max_count,
                              uint32_t* colmax, uint64_t* colsum, cudaStream_t stream) {
    if (ncols == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(colmax, 0, (size_t)ncols * 4, stream);
    if (e == cudaSuccess && colsum) e = cudaMemsetAsync(colsum, 0, (size_t)ncols * 8, stream);
    if (e != cudaSuccess) return e;
    const uint32_t chunks = (uint32_t)((max_count + kColChunk - 1) / kColChunk > 0 ? (max_count + kColChunk - 1) / kColChunk : 1);
    k_column_max<<<grid_items((uint64_t)ncols * chunks), 256, 0, stream>>>(
        pilots, cols, ncols, chunks, colmax, reinterpret_cast<unsigned long long*>(colsum));
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_rice_unary_len(const uint32_t* pilots, const ColDesc* cols, uint32_t ncols, uint64_t* hlen,
                                  cudaStream_t stream) {
    k_rice_unary_len<<<grid_items(ncols), 256, 0, stream>>>(pilots, cols, ncols, hlen);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_rice_unary(const uint32_t* pilots, const ColDesc* cols, uint32_t ncols, uint64_t* arena,
                              cudaStream_t stream) {
    k_column_unary<false><<<grid_items(ncols), 1024, 0, stream>>>(pilots, cols, ncols, arena);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_ef_columns(const uint32_t* pilots, const ColDesc* cols, uint32_t ncols, uint64_t* arena,
                              cudaStream_t stream) {
    k_column_unary<true><<<grid_items(ncols), 1024, 0, stream>>>(pilots, cols, ncols, arena);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_pack_columns(const uint32_t* pilots, const ColDesc* cols, uint32_t ncols, const uint64_t* word_begin,
                                uint64_t total_words, bool ranks, const uint64_t* bitmaps,
                                const uint64_t* bitmaps_rank, uint64_t* arena, cudaStream_t stream) {
    if (ranks)
        k_pack_columns<true><<<grid_for(total_words, 256), 256, 0, stream>>>(pilots, cols, ncols, word_begin, bitmaps,
                                                                             bitmaps_rank, arena);
    else
        k_pack_columns<false><<<grid_for(total_words, 256), 256, 0, stream>>>(pilots, cols, ncols, word_begin,
                                                                              bitmaps, bitmaps_rank, arena);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_dict_mark(const uint32_t* pilots, const ColDesc* cols, uint32_t ncols, uint64_t* bitmaps,
                             cudaStream_t stream) {
    k_dict_mark<<<grid_items(ncols), 256, 0, stream>>>(pilots, cols, ncols, bitmaps);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_dict_rank(const ColDesc* cols, uint32_t ncols, uint64_t* bitmaps_rank, const uint64_t* bitmaps,
                             uint64_t* K, cudaStream_t stream) {
    k_dict_rank<<<grid_items(ncols), 1024, 0, stream>>>(cols, ncols, bitmaps_rank, bitmaps, K);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_dict_pack_values(const ColDesc* cols, uint32_t ncols, const uint64_t* bm_begin,
                                    uint64_t total_bm_words, const uint64_t* bitmaps, const uint64_t* bitmaps_rank,
                                    uint64_t* arena, cudaStream_t stream) {
    k_dict_pack_values<<<grid_for(total_bm_words, 256), 256, 0, stream>>>(cols, ncols, bm_begin, bitmaps, bitmaps_rank,
                                                                          arena);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace phobic
