// K1 + K2: master hashing fused into an LSD onesweep radix sort by partition id.
//
// Section 4 splits the keys into partitions of expected size P.  Partition
// j = floor(hk * N_P / 2^64) is a monotone function of the 64-bit master hash
// hk.  Sorting by j therefore needs only ceil(log2 N_P) bits.  The sort is a
// least-significant-digit radix sort in the onesweep style (Adinets & Merrill
// 2022): one upfront pass computes every digit histogram, then each digit pass
// ranks a tile in shared memory.  It finds the tile's global offset by decoupled
// look-back over its predecessors and writes the tile out in digit order.  When
// the input is raw 64-bit keys, the upfront pass hashes them and writes the
// master hashes out (8 B per key more than the method needs), so that no digit
// pass hashes again.
//
// Segments: the input may hold several independent key sets back to back (a
// batched build).  Each set is a segment with its own partition count; tiles
// never cross segments, digit offsets are per segment and the look-back stops
// at the segment's first tile, so every set comes out grouped by its own
// partition ids in place.  A single build is one segment.
#include "phobic_dev.cuh"
#include "phobic_kernels.cuh"

namespace phobic {

namespace {

constexpr int kThreads = 384;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;  // keys per tile
static_assert(kTile == (int)kSortTileKeys, "tile size");
constexpr int kWarps = kThreads / 32;
constexpr uint64_t kFlagAgg = 1ull << 62;
constexpr uint64_t kFlagPre = 2ull << 62;
constexpr uint64_t kValMask = (1ull << 62) - 1;
constexpr uint32_t kSpinLimit = 1u << 22;
constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr uint32_t kLookWin = 2;    // predecessors' states read per look-back poll
constexpr uint64_t kStatusPad = 2;  // unused tile rows before the states (a poll's window may start at tile -1)

// The digit of each pass: bits [shift[p], shift[p] + bits[p]) of the partition
// id.  ceil(log2 N_P) bits split into as few passes of at most 9 bits as
// possible; when they do not split evenly, the first passes take one bit less
// (17 bits: 8 + 9, where equal widths would run two 512-digit passes, one of
// them with half its digits empty).  Histogram rows, digit bases and look-back
// states keep the widest pass's stride.
constexpr uint32_t kMaxPasses = 8;
struct DigitPlan {
    uint32_t passes, max_bits;
    uint32_t bits[kMaxPasses], shift[kMaxPasses];
    __device__ __forceinline__ uint32_t digit(uint64_t j, uint32_t p) const {
        return (uint32_t)(j >> shift[p]) & ((1u << bits[p]) - 1);
    }
};

DigitPlan make_digit_plan(uint64_t np) {
    DigitPlan d{};
    uint32_t bits_max = 0;
    sort_plan(np, &d.passes, &bits_max);
    d.max_bits = bits_max;
    const uint32_t total = np > 1 ? bitlen64(np - 1) : 0;
    if (d.passes) {
        const uint32_t base = total / d.passes, extra = total % d.passes;
        uint32_t sh = 0;
        for (uint32_t p = 0; p < d.passes; p++) {
            d.bits[p] = base + (p >= d.passes - extra ? 1u : 0u);
            d.shift[p] = sh;
            sh += d.bits[p];
        }
    }
    return d;
}

__device__ __forceinline__ uint64_t load_hk(const uint64_t* in, uint64_t i, uint64_t kseed, int hash_input) {
    uint64_t v = __ldg(in + i);
    return hash_input ? key_hash(v, kseed) : v;
}

// Digit histograms of every pass in one read of the input, per segment.  Each
// block walks a contiguous range of tiles; each warp counts into its own
// sub-histogram, which is flushed to the segment's global histogram when the
// segment changes and at the end.  When the input needs hashing, the master
// hashes are also written out (hashed_out, with streaming stores: the first
// pass reads them only after the whole input), so that no pass hashes again.
__device__ __forceinline__ uint32_t seg_of_tile(const SortSeg* __restrict__ segs, uint32_t nseg, uint64_t t) {
    uint32_t lo = 0, hi = nseg;  // largest s with first_tile[s] <= t
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (segs[mid].first_tile <= t) lo = mid; else hi = mid;
    }
    return lo;
}

// kPasses = dp.passes, so that the per-key loop over the passes unrolls exactly.
template <uint32_t kPasses>
__global__ void __launch_bounds__(256) k_sort_hist(const uint64_t* __restrict__ in, const SortSeg* __restrict__ segs,
                                                   uint32_t nseg, uint64_t tiles, uint64_t kseed, int hash_input,
                                                   DigitPlan dp, unsigned long long* __restrict__ hist,
                                                   uint64_t* __restrict__ hashed_out) {
    extern __shared__ uint32_t sh_hist[];  // [kWarpsH][passes * R], R = 2^(widest digit)
    constexpr int kWarpsH = 8;
    constexpr uint32_t passes = kPasses;
    const uint32_t R = 1u << dp.max_bits, PR = passes * R;
    const uint64_t per = (tiles + gridDim.x - 1) / gridDim.x;
    const uint64_t t0 = (uint64_t)blockIdx.x * per;
    const uint64_t t1 = t0 + per < tiles ? t0 + per : tiles;
    if (t0 >= t1) return;
    for (uint32_t i = threadIdx.x; i < kWarpsH * PR; i += blockDim.x) sh_hist[i] = 0;
    __syncthreads();
    uint32_t* mine = sh_hist + (threadIdx.x >> 5) * PR;
    uint32_t sg = seg_of_tile(segs, nseg, t0);
    uint64_t t = t0;
    while (t < t1) {
        const SortSeg S = segs[sg];
        const uint64_t tend = S.first_tile + (S.n + kTile - 1) / kTile;  // this segment's tiles
        const uint64_t ta = t, tb = tend < t1 ? tend : t1;
        const uint64_t k0 = S.key_base + (ta - S.first_tile) * kTile;
        uint64_t k1 = S.key_base + (tb - S.first_tile) * kTile;
        if (k1 > S.key_base + S.n) k1 = S.key_base + S.n;
        // four keys per thread per step, so that four loads are in flight
        uint64_t i = k0 + threadIdx.x;
        for (; i + 3ull * blockDim.x < k1; i += 4ull * blockDim.x) {
            uint64_t v[4];
#pragma unroll
            for (int u = 0; u < 4; u++) v[u] = __ldg(in + i + (uint64_t)u * blockDim.x);
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const uint64_t hk = hash_input ? key_hash(v[u], kseed) : v[u];
                if (hashed_out) __stcs(hashed_out + i + (uint64_t)u * blockDim.x, hk);  // read again only by the first pass
                const uint64_t j = partition_of(hk, S.np);
#pragma unroll
                for (uint32_t p = 0; p < passes; p++) atomicAdd(&mine[p * R + dp.digit(j, p)], 1u);
            }
        }
        for (; i < k1; i += blockDim.x) {
            const uint64_t v = __ldg(in + i);
            const uint64_t hk = hash_input ? key_hash(v, kseed) : v;
            if (hashed_out) __stcs(hashed_out + i, hk);
            const uint64_t j = partition_of(hk, S.np);
#pragma unroll
            for (uint32_t p = 0; p < passes; p++) atomicAdd(&mine[p * R + dp.digit(j, p)], 1u);
        }
        __syncthreads();
        unsigned long long* gh = hist + (uint64_t)sg * PR;
        for (uint32_t i = threadIdx.x; i < PR; i += blockDim.x) {
            uint32_t c = 0;
            for (int w = 0; w < kWarpsH; w++) {
                c += sh_hist[w * PR + i];
                sh_hist[w * PR + i] = 0;
            }
            if (c) atomicAdd(gh + i, (unsigned long long)c);
        }
        __syncthreads();
        t = tb;
        sg++;
    }
}

// exclusive scan of each (segment, pass) digit histogram, plus the segment's
// first key index (one block of 512 threads each)
__global__ void __launch_bounds__(512) k_sort_hist_scan(unsigned long long* hist, const SortSeg* __restrict__ segs,
                                                        uint32_t passes, uint32_t bits) {
    __shared__ unsigned long long ws[16];
    const uint32_t R = 1u << bits, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t sg = blockIdx.x / passes;
    unsigned long long* h = hist + (uint64_t)blockIdx.x * R;
    const unsigned long long v = tid < R ? h[tid] : 0;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(kFull, x, o);
        if (lane >= (uint32_t)o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    unsigned long long off = segs[sg].key_base;
    for (uint32_t w = 0; w < warp; w++) off += ws[w];
    if (tid < R) h[tid] = off + x - v;
}

struct PassArgs {
    const uint64_t* in;
    uint64_t* out;
    const SortSeg* segs;
    uint32_t nseg, passes, pass;
    uint64_t kseed;
    int hash_input;
    uint32_t shift, bits;   // this pass's digit: bits [shift, shift + bits) of the partition id
    uint32_t bits0;         // the first pass's digit width
    uint32_t rstride;       // digits per (segment, pass) row of digit_base: 2^(widest digit)
    const unsigned long long* digit_base; // [seg][pass][rstride]: exclusive scans of the histograms
    unsigned long long* status;            // [kStatusPad + tiles][R]: flag | value
    uint32_t* tile_counter;
    uint32_t* error;
    uint32_t spin_limit;  // polls of an unpublished predecessor before the wait gives up
    uint64_t mute_tile;   // self-test: this tile never publishes its state (~0: none)
};

// One digit pass.  Tile = kTile consecutive keys.  Warp w ranks its 32 x kItems
// keys (order: item, lane): the lanes with equal digits are found as the AND,
// over the digit's bits, of the ballots of the lanes that agree on that bit;
// the leader of each group adds the group size to the warp's counter with one
// shared atomicAdd and hands the old value to its peers, so ranks are stable.
// The first of several passes need not be stable (every later pass is, and
// keeps its digit order; the order inside a partition is left unspecified): it
// ranks each key with one shared atomicAdd on its digit's counter.  The last
// of two passes ranks the same way when its tile holds at most two first-pass
// digits, with each digit's keys in two bins by that digit.  Then per digit:
// prefix over warps and publication of the tile's counts, a block scan for
// the tile-local digit starts, a shared-memory reorder, decoupled look-back
// for the tile's global offset, and a coalesced write-out.
__global__ void __launch_bounds__(kThreads, 2) k_sort_pass(PassArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t R = 1u << a.bits, mask = R - 1;
    uint64_t* keys_s = reinterpret_cast<uint64_t*>(smem);                      // kTile
    // per warp 2R counters: a digit's keys of the tile split by the previous
    // pass's digit when the last pass ranks without ballots (below)
    const uint32_t WS = 2 * R;
    uint32_t* wh = reinterpret_cast<uint32_t*>(keys_s + kTile);                // kWarps x 2R
    uint32_t* tile_start = wh + kWarps * WS;                                   // R
    uint32_t* sub1 = tile_start + R;                                           // R
    unsigned long long* gbase = reinterpret_cast<unsigned long long*>(sub1 + R);  // R
    __shared__ uint32_t tile_s;
    __shared__ uint32_t warp_tot[kWarps];

    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) tile_s = atomicAdd(a.tile_counter, 1u);
    for (uint32_t i = tid; i < kWarps * WS; i += kThreads) wh[i] = 0;
    __syncthreads();
    const uint64_t tile = tile_s;
    const uint32_t sg = seg_of_tile(a.segs, a.nseg, tile);
    const SortSeg S = a.segs[sg];
    const uint64_t first = S.first_tile;
    const uint64_t seg_end = S.key_base + S.n;
    const uint64_t base = S.key_base + (tile - first) * kTile;
    const uint64_t wbase = base + (uint64_t)warp * 32 * kItems;

    uint64_t k[kItems];
#pragma unroll
    for (int i = 0; i < kItems; i++) {
        uint64_t idx = wbase + (uint64_t)i * 32 + lane;
        k[i] = idx < seg_end ? load_hk(a.in, idx, a.kseed, a.hash_input) : 0;
    }
    uint32_t dr[kItems];  // digit (or bin) << 16 | rank within the warp's digit (bin) group
    const uint32_t lt = (1u << lane) - 1;
    uint32_t* myh = wh + warp * WS;
    // The last of two passes must keep, inside each digit, the order of the
    // first pass's digit.  Its input is grouped by that digit, so a tile holds a
    // run of consecutive first-pass digits: when the run has at most two, the
    // keys of digit d go to bin 2 d + (first-pass digit != the tile's first),
    // and ranking within a bin needs no order (one shared atomic per key); the
    // two bins of a digit are laid out one after the other.  Wider runs (few
    // keys per digit) keep the stable ballot ranking.
    bool split = false;
    uint32_t lo_first = 0;
    if (a.pass == 1 && a.passes == 2) {
        // the run of first-pass digits: those of the tile's first and last keys
        const uint64_t last = (seg_end - base < (uint64_t)kTile ? seg_end : base + kTile) - 1;
        const uint32_t m0 = (1u << a.bits0) - 1;
        lo_first = (uint32_t)partition_of(load_hk(a.in, base, a.kseed, a.hash_input), S.np) & m0;
        const uint32_t ll = (uint32_t)partition_of(load_hk(a.in, last, a.kseed, a.hash_input), S.np) & m0;
        split = ll - lo_first <= 1;
    }
    if (split) {
        const uint64_t lomask = (1ull << a.bits0) - 1;
#pragma unroll
        for (int i = 0; i < kItems; i++) {
            const bool valid = wbase + (uint64_t)i * 32 + lane < seg_end;
            const uint64_t j = partition_of(k[i], S.np);
            const uint32_t dg = (uint32_t)((j >> a.shift) & mask);
            const uint32_t bin = valid ? 2 * dg + ((uint32_t)(j & lomask) != lo_first ? 1u : 0u) : WS;
            const uint32_t rank = valid ? atomicAdd(&myh[bin], 1u) : 0u;
            dr[i] = (bin << 16) | rank;
        }
    } else if (a.pass == 0 && a.passes > 1) {
        // the first of several passes need not be stable (the later ones keep its
        // digit order): a key's rank is one shared atomic on its warp's counter
#pragma unroll
        for (int i = 0; i < kItems; i++) {
            const bool valid = wbase + (uint64_t)i * 32 + lane < seg_end;
            const uint32_t dg = valid ? (uint32_t)((partition_of(k[i], S.np) >> a.shift) & mask) : R;
            const uint32_t rank = valid ? atomicAdd(&myh[dg], 1u) : 0u;
            dr[i] = (dg << 16) | rank;
        }
    } else
#pragma unroll
    for (int i = 0; i < kItems; i++) {
        const bool valid = wbase + (uint64_t)i * 32 + lane < seg_end;
        const uint32_t dg = valid ? (uint32_t)((partition_of(k[i], S.np) >> a.shift) & mask) : R;
        uint32_t peers = __ballot_sync(kFull, valid);
        for (uint32_t bb = 0; bb < a.bits; bb++) {
            const uint32_t bit = (dg >> bb) & 1u;
            const uint32_t bal = __ballot_sync(kFull, bit);
            peers &= bit ? bal : ~bal;
        }
        const uint32_t leader = __ffs(peers) - 1;
        uint32_t old = 0;
        if (lane == leader && dg < R) old = atomicAdd(&myh[dg], (uint32_t)__popc(peers));
        old = __shfl_sync(kFull, old, leader);
        dr[i] = (dg << 16) | (old + __popc(peers & lt));
    }
    __syncthreads();
    // per digit (per bin when split): exclusive prefix over warps; tile count into tile_start
    if (split) {
        for (uint32_t d = tid; d < R; d += kThreads) {
            uint32_t run0 = 0, run1 = 0;
#pragma unroll
            for (int w = 0; w < kWarps; w++) {
                const uint32_t c0 = wh[w * WS + 2 * d], c1 = wh[w * WS + 2 * d + 1];
                wh[w * WS + 2 * d] = run0;
                wh[w * WS + 2 * d + 1] = run1;
                run0 += c0;
                run1 += c1;
            }
            sub1[d] = run0;  // the second bin of digit d starts after the first
            tile_start[d] = run0 + run1;
        }
    } else {
        for (uint32_t d = tid; d < R; d += kThreads) {
            uint32_t run = 0;
#pragma unroll
            for (int w = 0; w < kWarps; w++) {
                uint32_t c = wh[w * WS + d];
                wh[w * WS + d] = run;
                run += c;
            }
            tile_start[d] = run;
        }
    }
    __syncthreads();
    // Publish the tile's digit counts at once (the aggregate; the inclusive
    // prefix for a segment's first tile), so that successors can sum past this
    // tile while it scans and reorders.  Thread tid owns digits tid and
    // tid + kThreads (R <= 512 < 2 kThreads) and keeps their counts for its
    // look-back below.
    volatile unsigned long long* st = a.status;
    const bool publish = tile != a.mute_tile;
    uint32_t cnt_own[2] = {0, 0};
#pragma unroll
    for (int u = 0; u < 2; u++) {
        const uint32_t d = tid + u * kThreads;
        if (d < R) {
            cnt_own[u] = tile_start[d];
            if (publish) st[(tile + kStatusPad) * R + d] = (tile == first ? kFlagPre : kFlagAgg) | cnt_own[u];
        }
    }
    // block-wide exclusive scan of the tile counts over digits: each thread
    // owns R / kThreads consecutive digits (1 or 2)
    {
        const uint32_t per = (R + kThreads - 1) / kThreads;
        uint32_t c[2] = {0, 0}, sum = 0;
        for (uint32_t u = 0; u < per; u++) {
            uint32_t d = tid * per + u;
            c[u] = d < R ? tile_start[d] : 0;
            sum += c[u];
        }
        uint32_t x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(kFull, x, o);
            if (lane >= (uint32_t)o) x += y;
        }
        if (lane == 31) warp_tot[warp] = x;
        __syncthreads();
        uint32_t woff = 0;
#pragma unroll
        for (int w = 0; w < kWarps; w++) woff += (w < (int)warp) ? warp_tot[w] : 0;
        uint32_t run = woff + x - sum;
        for (uint32_t u = 0; u < per; u++) {
            uint32_t d = tid * per + u;
            if (d < R) tile_start[d] = run;
            run += c[u];
        }
    }
    __syncthreads();
    // reorder in shared memory by digit (tile-local offsets only)
    if (split) {
#pragma unroll
        for (int i = 0; i < kItems; i++) {
            const uint32_t bin = dr[i] >> 16;
            if (bin < WS) {
                const uint32_t d = bin >> 1;
                keys_s[tile_start[d] + ((bin & 1u) ? sub1[d] : 0u) + wh[warp * WS + bin] + (dr[i] & 0xFFFFu)] = k[i];
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < kItems; i++) {
            uint32_t d = dr[i] >> 16;
            if (d < R) keys_s[tile_start[d] + wh[warp * WS + d] + (dr[i] & 0xFFFFu)] = k[i];
        }
    }
    // Decoupled look-back per digit, after the reorder: the predecessors have
    // had that much longer to publish.  Each poll reads the states of two
    // predecessors; reading more per poll was measured slower, because the
    // polls of all tiles share the L2 lines that the tiles publish to.
#pragma unroll
    for (int u = 0; u < 2; u++) {
        const uint32_t d = tid + u * kThreads;
        if (d >= R) continue;
        uint64_t excl = 0;
        if (tile != first) {
            // states of tile x for digit d at (x + kStatusPad) R + d; the tile rows
            // start 256-byte aligned
            const volatile unsigned long long* col = st + kStatusPad * R + d;
            int64_t e = (int64_t)tile;  // predecessors [first, e) are not accounted yet
            const int64_t lo = (int64_t)first;
            uint32_t spins = 0;
            bool done = false;
            while (!done) {
                const int64_t s0 = e - (int64_t)kLookWin;  // >= -1, inside the padding
                unsigned long long v[kLookWin];
#pragma unroll
                for (int q = 0; q < (int)kLookWin; q++) v[q] = col[(s0 + q) * (int64_t)R];
                const int64_t e0 = e;
                bool stop = false;
#pragma unroll
                for (int q = (int)kLookWin - 1; q >= 0; q--) {
                    const int64_t x = s0 + q;  // nearest first
                    if (stop) continue;
                    if (x < lo) {  // past the segment's first tile: everything is accounted
                        done = stop = true;
                        continue;
                    }
                    const uint64_t flag = v[q] & ~kValMask;
                    if (flag == 0) {  // not published yet: poll again from here
                        stop = true;
                        continue;
                    }
                    excl += v[q] & kValMask;
                    e = x;
                    if (flag == kFlagPre) done = stop = true;
                }
                if (done) break;
                if (e == e0) {
                    if (++spins > a.spin_limit) {
                        atomicMax(a.error, kDevTimeout);
                        break;
                    }
                    if (spins > 32) __nanosleep(64);
                }
            }
            if (publish) st[(tile + kStatusPad) * R + d] = kFlagPre | (excl + cnt_own[u]);
        }
        gbase[d] = a.digit_base[((uint64_t)sg * a.passes + a.pass) * a.rstride + d] + excl - tile_start[d];
    }
    __syncthreads();
    // coalesced write-out: consecutive slots of one digit go to consecutive addresses
    const uint64_t valid = seg_end - base < (uint64_t)kTile ? seg_end - base : (uint64_t)kTile;
#pragma unroll 4
    for (uint32_t i = tid; i < valid; i += kThreads) {
        uint64_t v = keys_s[i];
        uint32_t d = (uint32_t)((partition_of(v, S.np) >> a.shift) & mask);
        uint64_t dst = gbase[d] + i;
        if (dst >= S.key_base && dst < seg_end) a.out[dst] = v;  // only a timed-out look-back could leave the range
    }
}

// master hashes (or a copy) of n keys: 16-byte loads and stores of key pairs
// when both arrays are 16-byte aligned, streaming past the caches
__global__ void k_hash_copy(const uint64_t* __restrict__ in, uint64_t* __restrict__ out, uint64_t n, uint64_t kseed,
                            int hash_input) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t t0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15) == 0) {
        const ulonglong2* in2 = reinterpret_cast<const ulonglong2*>(in);
        ulonglong2* out2 = reinterpret_cast<ulonglong2*>(out);
        for (uint64_t i = t0; i < n / 2; i += stride) {
            ulonglong2 v = __ldcs(in2 + i);
            if (hash_input) {
                v.x = key_hash(v.x, kseed);
                v.y = key_hash(v.y, kseed);
            }
            __stcs(out2 + i, v);
        }
        if ((n & 1) && t0 == 0) out[n - 1] = load_hk(in, n - 1, kseed, hash_input);
    } else {
        for (uint64_t i = t0; i < n; i += stride) out[i] = load_hk(in, i, kseed, hash_input);
    }
}

// start[part_base_s + j] = first index of partition j of segment s in the
// sorted array (binary search inside the segment); start[total partitions] = n
__global__ void k_partition_starts(const uint64_t* __restrict__ sorted, const SortSeg* __restrict__ segs, uint32_t nseg,
                                   uint64_t total_parts, uint64_t* __restrict__ start) {
    const uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (g > total_parts) return;
    uint32_t lo_s = 0, hi_s = nseg;  // segment: largest s with part_base <= g (ignoring empty ones at the end)
    while (hi_s - lo_s > 1) {
        uint32_t mid = (lo_s + hi_s) >> 1;
        if (segs[mid].part_base <= g) lo_s = mid; else hi_s = mid;
    }
    const SortSeg S = segs[lo_s];
    const uint64_t j = g - S.part_base;
    uint64_t lo = S.key_base, hi = S.key_base + S.n;
    if (j >= S.np) {
        start[g] = hi;
        return;
    }
    while (lo < hi) {
        uint64_t mid = (lo + hi) >> 1;
        if (partition_of(__ldg(sorted + mid), S.np) < j)
            lo = mid + 1;
        else
            hi = mid;
    }
    start[g] = lo;
}

}  // namespace

size_t sort_pass_smem(uint32_t bits) {
    uint32_t R = 1u << bits;
    return (size_t)kTile * 8 + (size_t)kWarps * 2 * R * 4 + (size_t)2 * R * 4 + (size_t)R * 8;
}

void sort_plan(uint64_t np, uint32_t* passes, uint32_t* bits) {
    uint32_t total = np > 1 ? bitlen64(np - 1) : 0;
    uint32_t p = (total + 8) / 9;  // at most 9 bits (512 digits) per pass
    *passes = p;
    *bits = p ? (total + p - 1) / p : 0;
}

uint64_t sort_tiles(uint64_t n) { return (n + kTile - 1) / kTile; }

size_t sort_seg_scratch_bytes(uint64_t n_total, uint64_t tiles, uint32_t nseg, uint64_t max_np) {
    uint32_t passes, bits;
    sort_plan(max_np, &passes, &bits);
    const uint64_t R = 1ull << bits;
    size_t s = 0;
    s += (size_t)n_total * 8;                          // ping-pong buffer
    s += (size_t)nseg * (passes ? passes : 1) * R * 8 + 64;  // histograms / digit bases
    s += 256 + (size_t)(tiles + kStatusPad) * R * 8 + 64;  // look-back states, 256-byte aligned
    s += 64 * 4;                                       // tile counters
    return s;
}

size_t sort_scratch_bytes(uint64_t n, uint64_t np) {
    return sort_seg_scratch_bytes(n, sort_tiles(n), 1, np) + 64;  // + one segment record
}

cudaError_t launch_partition_sort_segs(const uint64_t* in, int hash_input, uint64_t kseed, const SortSeg* d_segs,
                                       uint32_t nseg, uint64_t n_total, uint64_t tiles, uint64_t max_np,
                                       uint64_t total_parts, uint64_t* sorted, uint64_t* start, void* scratch,
                                       uint32_t* d_error, cudaStream_t stream, const SortWaitTest* wait_test) {
    const DigitPlan dp = make_digit_plan(max_np);
    const uint32_t passes = dp.passes, bits = dp.max_bits;
    const uint32_t R = 1u << bits;
    unsigned char* p = static_cast<unsigned char*>(scratch);
    uint64_t* alt = reinterpret_cast<uint64_t*>(p);
    p += (size_t)n_total * 8;
    unsigned long long* hist = reinterpret_cast<unsigned long long*>(p);
    p += (size_t)nseg * (passes ? passes : 1) * R * 8 + 64;
    p = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(p) + 255) & ~uintptr_t(255));
    unsigned long long* status = reinterpret_cast<unsigned long long*>(p);
    const size_t status_bytes = (size_t)(tiles + kStatusPad) * R * 8;
    p += status_bytes + 64;
    uint32_t* counters = reinterpret_cast<uint32_t*>(p);
    cudaError_t e;

    if (passes == 0) {  // every segment is a single partition: hash (or copy) only
        if (n_total) {
            k_hash_copy<<<(unsigned)((n_total + 255) / 256 < 8192 ? (n_total + 255) / 256 : 8192), 256, 0,
                          stream>>>(in, sorted, n_total, kseed, hash_input);
            note_launches(1);
        }
    } else {
        if ((e = cudaMemsetAsync(hist, 0, (size_t)nseg * passes * R * 8, stream)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(counters, 0, 64 * 4, stream)) != cudaSuccess) return e;
        int dev = 0, sms = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        uint64_t hblocks = tiles < (uint64_t)sms * 8 ? tiles : (uint64_t)sms * 8;
        if (hblocks == 0) hblocks = 1;
        using HistKernel = void (*)(const uint64_t*, const SortSeg*, uint32_t, uint64_t, uint64_t, int, DigitPlan,
                                    unsigned long long*, uint64_t*);
        static const HistKernel hist_kernels[kMaxPasses] = {k_sort_hist<1>, k_sort_hist<2>, k_sort_hist<3>,
                                                            k_sort_hist<4>, k_sort_hist<5>, k_sort_hist<6>,
                                                            k_sort_hist<7>, k_sort_hist<8>};
        if (passes > kMaxPasses) return cudaErrorInvalidValue;
        const HistKernel hk = hist_kernels[passes - 1];
        if ((e = allow_max_dynamic_smem(reinterpret_cast<const void*>(hk))) != cudaSuccess) return e;
        // with hashing: the histogram pass also writes the master hashes, into the
        // buffer that the first pass does not write, and the passes read those
        uint64_t* hashed = hash_input ? ((passes & 1) ? alt : sorted) : nullptr;
        hk<<<(unsigned)hblocks, 256, 8 * passes * R * 4, stream>>>(in, d_segs, nseg, tiles, kseed, hash_input, dp,
                                                                   hist, hashed);
        note_launches(1);
        k_sort_hist_scan<<<nseg * passes, 512, 0, stream>>>(hist, d_segs, passes, bits);
        note_launches(1);
        if ((e = allow_max_dynamic_smem(reinterpret_cast<const void*>(k_sort_pass))) != cudaSuccess) return e;
        const uint64_t* src = hashed ? hashed : in;
        int hash_now = 0;
        // ping-pong so that the last pass lands in `sorted`
        uint64_t* dst = (passes & 1) ? sorted : alt;
        for (uint32_t ps = 0; ps < passes; ps++) {
            if ((e = cudaMemsetAsync(status, 0, status_bytes, stream)) != cudaSuccess) return e;
            PassArgs a;
            a.in = src;
            a.out = dst;
            a.segs = d_segs;
            a.nseg = nseg;
            a.passes = passes;
            a.pass = ps;
            a.kseed = kseed;
            a.hash_input = hash_now;
            a.shift = dp.shift[ps];
            a.bits = dp.bits[ps];
            a.bits0 = dp.bits[0];
            a.rstride = R;
            a.digit_base = hist;
            a.status = status;
            a.tile_counter = counters + ps;
            a.error = d_error;
            a.spin_limit = wait_test ? wait_test->spin_limit : kSpinLimit;
            a.mute_tile = wait_test ? wait_test->mute_tile : ~0ull;
            k_sort_pass<<<(unsigned)tiles, kThreads, sort_pass_smem(dp.bits[ps]), stream>>>(a);
            note_launches(1);
            src = dst;
            hash_now = 0;
            dst = (dst == sorted) ? alt : sorted;
        }
    }
    k_partition_starts<<<(unsigned)((total_parts + 1 + 255) / 256), 256, 0, stream>>>(sorted, d_segs, nseg,
                                                                                      total_parts, start);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_partition_sort(const uint64_t* in, int hash_input, uint64_t kseed, uint64_t n, uint64_t np,
                                  uint64_t* sorted, uint64_t* start, void* scratch, uint32_t* d_error,
                                  cudaStream_t stream, const SortWaitTest* wait_test) {
    // one segment; its record sits at the end of the scratch region
    const uint64_t tiles = sort_tiles(n);
    SortSeg* d_seg = reinterpret_cast<SortSeg*>(static_cast<unsigned char*>(scratch) +
                                                sort_seg_scratch_bytes(n, tiles, 1, np));
    SortSeg hs;
    hs.key_base = 0;
    hs.n = n;
    hs.np = np;
    hs.part_base = 0;
    hs.first_tile = 0;
    cudaError_t e = cudaMemcpyAsync(d_seg, &hs, sizeof(SortSeg), cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return e;
    return launch_partition_sort_segs(in, hash_input, kseed, d_seg, 1, n, tiles, np, np, sorted, start, scratch,
                                      d_error, stream, wait_test);
}

cudaError_t launch_hash_u64(const uint64_t* keys, uint64_t n, uint64_t kseed, uint64_t* out, cudaStream_t stream) {
    uint64_t blocks = (n + 255) / 256;
    if (blocks > 16384) blocks = 16384;
    if (blocks == 0) return cudaSuccess;
    k_hash_copy<<<(unsigned)blocks, 256, 0, stream>>>(keys, out, n, kseed, 1);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace phobic
