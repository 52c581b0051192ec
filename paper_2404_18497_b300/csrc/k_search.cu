// K3 + K4: per-partition bucketing, bucket ordering and pilot search.
//
// One warp owns one partition (Section 4.2: one workgroup per partition; the
// search runs in shared memory).  For each partition:
//   1. Load the partition's master hashes.  Compute every key's bucket with the
//      tabulated gamma (Section 3.1, Appendix C), and counting-sort the keys by
//      bucket in shared memory.
//   2. Order the non-empty buckets by size descending, then by index descending.
//      Index descending means increasing expected size (Section 1; Section 5,
//      "Further Remarks").  Equal sizes are split with __match_any_sync, so the
//      order is deterministic.
//   3. Place the buckets one after another.  Each bucket takes the smallest pilot
//      that puts its keys on distinct free slots (Section 4.2: "smallest working
//      seed").
//      ADDITIVE mode (Section 4, "Hash Function"): p = s m + d.  For each s the
//      warp computes h(x, s) once per key.  Equal values among the keys rule
//      out this s (a shift by d moves them together).  Otherwise d is found by
//      scanning windows of 64 (or 32) displacements of the free-slot bitmap.
//      The bitmap is stored twice in a row, so (h + d) mod m reads linearly.  A
//      window is the AND, over the bucket's keys, of the free bits starting at
//      h + 64w.  Lanes split into groups: each group covers one window and its
//      lanes cover the keys.  A ballot picks the first window with a set bit,
//      and __ffs picks its smallest d.  That is the smallest valid d, so p
//      matches a sequential scan exactly.
//      XOR mode (PTHash): groups of lanes test consecutive pilots p, one key
//      per lane.  A slot must be free and unshared within its group.
//   4. Write the pilots (column-major, i.e. interleaved order) and, when a
//      global occupancy bitmap is requested (alpha < 1), the partition's taken
//      slots at bit offset T_j.
// Bounded work: a bucket that needs s >= min(s_max, floor((2^32 - 1) / m)) (the
// largest s whose pilots fit 32 bits), or holds more than 1023 keys,
// stops its partition with SEARCH_LIMIT.  Equal master hashes inside a bucket
// (duplicate keys) are detected and reported as DUP_HASH.
#include "phobic_dev.cuh"
#include "phobic_kernels.cuh"

namespace phobic {

namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr int kSizeHist = 1024;  // bucket sizes 1..1023
constexpr int kBigRegs = 4;      // keys per lane kept in registers for buckets of 33..128 keys

struct SmemLayout {
    uint32_t off_hk, off_bend, off_order, off_fw, off_scr, off_aux, off_ctl, total;
    uint32_t fw_words, scr_words;
};

// Shared memory of one partition's CTA: keys (optional), bucket ends, bucket
// order, the doubled free bitmap, then per warp a collision scratch bitmap and a
// u16[1024] buffer of h values (warp 0's also serves as the size histogram),
// then the control words through which the warps of a CTA agree on a result.
__host__ __device__ inline SmemLayout smem_layout(uint32_t cap_n, uint32_t cap_m, uint32_t B, bool keys_in_smem,
                                                  uint32_t warps) {
    SmemLayout L;
    uint32_t o = 0;
    L.off_hk = o;
    if (keys_in_smem) o += ((cap_n + 1) & ~1u) * 8;
    L.off_bend = o;
    o += (B + 1) * 4;
    L.off_order = o;
    o += B * 4;
    L.fw_words = (2 * cap_m + 128) / 32 + 3;
    L.off_fw = o;
    o += L.fw_words * 4;
    L.scr_words = (cap_m + 31) / 32 + 1;
    L.off_scr = o;
    o += warps * L.scr_words * 4;
    o = (o + 7) & ~7u;
    L.off_aux = o;
    o += warps * kSizeHist * 2;
    L.off_ctl = o;
    o += (warps > 1 ? 4 * warps + 4 : 0) * 4;
    L.total = (o + 15) & ~15u;
    return L;
}

template <int kWarps>
__device__ __forceinline__ void cta_sync() {
    if constexpr (kWarps == 1)
        __syncwarp();
    else
        __syncthreads();
}

// 32 free bits starting at bit q of the doubled free bitmap
__device__ __forceinline__ uint32_t window32(const uint32_t* fw, uint32_t q) {
    return __funnelshift_r(fw[q >> 5], fw[(q >> 5) + 1], q & 31);
}

// W free bits (W = 32 or 64 displacements) starting at bit q, with the mask of
// displacements d = W w .. W w + W - 1 that lie below m, and helpers on them.
template <int W>
struct Win;
template <>
struct Win<32> {
    using T = uint32_t;
    static __device__ __forceinline__ T load(const uint32_t* fw, uint32_t q) { return window32(fw, q); }
    static __device__ __forceinline__ T valid(uint32_t w, uint32_t m) {
        return (32 * w + 32 <= m) ? 0xFFFFFFFFu : ((1u << (m - 32 * w)) - 1);
    }
    static __device__ __forceinline__ uint32_t first(T x) { return __ffs(x) - 1; }
    static __device__ __forceinline__ T shfl(T x, uint32_t l) { return __shfl_sync(0xFFFFFFFFu, x, l); }
    static __device__ __forceinline__ T shfl_xor(T x, uint32_t o) { return __shfl_xor_sync(0xFFFFFFFFu, x, o); }
};
template <>
struct Win<64> {
    using T = uint64_t;
    static __device__ __forceinline__ T load(const uint32_t* fw, uint32_t q) {
        const uint32_t i = q >> 5, sh = q & 31;
        const uint32_t a = fw[i], b = fw[i + 1], c = fw[i + 2];
        return (uint64_t)__funnelshift_r(a, b, sh) | ((uint64_t)__funnelshift_r(b, c, sh) << 32);
    }
    static __device__ __forceinline__ T valid(uint32_t w, uint32_t m) {
        return (64 * w + 64 <= m) ? ~0ull : ((1ull << (m - 64 * w)) - 1);
    }
    static __device__ __forceinline__ uint32_t first(T x) { return __ffsll((long long)x) - 1; }
    static __device__ __forceinline__ T shfl(T x, uint32_t l) { return __shfl_sync(0xFFFFFFFFu, x, l); }
    static __device__ __forceinline__ T shfl_xor(T x, uint32_t o) { return __shfl_xor_sync(0xFFFFFFFFu, x, o); }
};

__device__ __forceinline__ void take_slot(uint32_t* fw, uint32_t pos, uint32_t m) {
    atomicAnd(&fw[pos >> 5], ~(1u << (pos & 31)));
    uint32_t q = pos + m;
    atomicAnd(&fw[q >> 5], ~(1u << (q & 31)));
}

// Lanes per window for a bucket of k keys when `free_slots` of m are free.
// A displacement is valid with probability about q^k (q = free fraction), so
// about C = q^-k candidates are scanned.  With L lanes per window one warp step
// covers 32 W / L candidates (W displacements per window); while C L <= 32 W one
// step suffices and a larger L splits the k keys over more lanes, so take the
// largest such L (at most pow2ceil(k)); otherwise L = 1 (every lane scans its
// own window).  The
// choice only changes speed: every L finds the smallest valid displacement.
template <int W>
__device__ __forceinline__ uint32_t choose_lanes_log2(uint32_t k, uint32_t free_slots, uint32_t m) {
    const uint32_t lk = k <= 1 ? 0u : 32u - __clz(k - 1);  // log2 pow2ceil(k)
    const float q = __fdividef((float)free_slots, (float)m);
    const float lc = (float)k * -__log2f(q);                // log2 C
    const float lg = (W == 64 ? 11.0f : 10.0f) - lc;        // log2(32 W) - log2 C
    const uint32_t l = lg <= 0.0f ? 0u : (uint32_t)lg;
    return min(l, min(lk, 5u));
}

// One sweep over the displacement windows for the current s with 2^LG lanes
// per window (32 >> LG windows per warp step): lane rr of group g ANDs the
// windows of keys rr, rr + 2^LG, ... for window w0 + g, the group reduces by
// AND, and a ballot over the group leaders takes the first window that still
// has a set bit; its lowest bit is the smallest valid displacement.  With one
// lane per window and 2048 < m <= 3072, the lanes take 96-bit windows instead,
// so that one step covers all m displacements.
template <int W, int LG>
__device__ __forceinline__ bool scan_windows(const uint32_t* fw, const uint16_t* hb, uint32_t k, uint32_t m,
                                             uint32_t nw, uint32_t lane, uint32_t& d, unsigned long long& steps) {
    using Wn = Win<W>;
    using WT = typename Wn::T;
    constexpr uint32_t Lw = 1u << LG, G = 32u >> LG;
    const uint32_t g = lane >> LG, rr = lane & (Lw - 1);
    if constexpr (W == 64 && LG == 0) {
        if (nw > 32 && m <= 96 * 32) {
            // 2048 < m <= 3072 (a partition of about 2500 keys): 64-bit windows
            // would take two steps, the second with most lanes idle.  One step of
            // 96-bit windows (lane g: displacements 96 g .. 96 g + 95; four loads
            // and three funnel shifts per key) covers every displacement instead.
            // Four keys at a time, so that their loads are in flight together: a
            // warp here waits mostly on its own loads, not for issue slots.
            steps++;
            const uint32_t base = 96 * lane;
            uint32_t a0 = 0, a1 = 0, a2 = 0;
            if (base < m) {
                const uint32_t rem = m - base;
                a0 = rem >= 32 ? kFull : (1u << rem) - 1;
                a1 = rem >= 64 ? kFull : rem <= 32 ? 0u : (1u << (rem - 32)) - 1;
                a2 = rem >= 96 ? kFull : rem <= 64 ? 0u : (1u << (rem - 64)) - 1;
                uint32_t i = 0;
                for (; i + 3 < k && (a0 | a1 | a2); i += 4) {
                    const uint32_t q = (uint32_t)hb[i] + base, r = (uint32_t)hb[i + 1] + base;
                    const uint32_t u = (uint32_t)hb[i + 2] + base, v = (uint32_t)hb[i + 3] + base;
                    const uint32_t* x = fw + (q >> 5);
                    const uint32_t* y = fw + (r >> 5);
                    const uint32_t* z = fw + (u >> 5);
                    const uint32_t* t = fw + (v >> 5);
                    const uint32_t sq = q & 31, sr = r & 31, su = u & 31, sv = v & 31;
                    a0 &= __funnelshift_r(x[0], x[1], sq) & __funnelshift_r(y[0], y[1], sr) &
                          __funnelshift_r(z[0], z[1], su) & __funnelshift_r(t[0], t[1], sv);
                    a1 &= __funnelshift_r(x[1], x[2], sq) & __funnelshift_r(y[1], y[2], sr) &
                          __funnelshift_r(z[1], z[2], su) & __funnelshift_r(t[1], t[2], sv);
                    a2 &= __funnelshift_r(x[2], x[3], sq) & __funnelshift_r(y[2], y[3], sr) &
                          __funnelshift_r(z[2], z[3], su) & __funnelshift_r(t[2], t[3], sv);
                }
                for (; i + 1 < k && (a0 | a1 | a2); i += 2) {
                    const uint32_t q = (uint32_t)hb[i] + base, r = (uint32_t)hb[i + 1] + base;
                    const uint32_t* x = fw + (q >> 5);
                    const uint32_t* y = fw + (r >> 5);
                    const uint32_t sq = q & 31, sr = r & 31;
                    const uint32_t x0 = x[0], x1 = x[1], x2 = x[2], x3 = x[3];
                    const uint32_t y0 = y[0], y1 = y[1], y2 = y[2], y3 = y[3];
                    a0 &= __funnelshift_r(x0, x1, sq) & __funnelshift_r(y0, y1, sr);
                    a1 &= __funnelshift_r(x1, x2, sq) & __funnelshift_r(y1, y2, sr);
                    a2 &= __funnelshift_r(x2, x3, sq) & __funnelshift_r(y2, y3, sr);
                }
                if (i < k && (a0 | a1 | a2)) {
                    const uint32_t q = (uint32_t)hb[i] + base;
                    const uint32_t* x = fw + (q >> 5);
                    const uint32_t sq = q & 31;
                    const uint32_t x0 = x[0], x1 = x[1], x2 = x[2], x3 = x[3];
                    a0 &= __funnelshift_r(x0, x1, sq);
                    a1 &= __funnelshift_r(x1, x2, sq);
                    a2 &= __funnelshift_r(x2, x3, sq);
                }
            }
            const uint32_t win = __ballot_sync(kFull, (a0 | a1 | a2) != 0);
            if (!win) return false;
            const uint32_t fl = __ffs(win) - 1;
            const uint32_t b0 = __shfl_sync(kFull, a0, fl), b1 = __shfl_sync(kFull, a1, fl),
                           b2 = __shfl_sync(kFull, a2, fl);
            d = 96 * fl + (b0 ? __ffs(b0) - 1 : b1 ? 31 + __ffs(b1) : 63 + __ffs(b2));
            return true;
        }
    }
    for (uint32_t w0 = 0; w0 < nw; w0 += G) {
        steps++;
        const uint32_t w = w0 + g;
        WT acc = 0;
        if (w < nw) {
            acc = Wn::valid(w, m);
            const uint32_t q0 = W * w;
            uint32_t i = rr;
            for (; i + Lw < k && acc; i += 2 * Lw) {
                const WT x0 = Wn::load(fw, (uint32_t)hb[i] + q0);
                const WT x1 = Wn::load(fw, (uint32_t)hb[i + Lw] + q0);
                acc &= x0 & x1;
            }
            if (i < k && acc) acc &= Wn::load(fw, (uint32_t)hb[i] + q0);
        }
        if constexpr (LG == 5 && W == 32) {
            acc = __reduce_and_sync(kFull, acc);
        } else {
#pragma unroll
            for (uint32_t o = 1; o < Lw; o <<= 1) acc &= Wn::shfl_xor(acc, o);
        }
        const uint32_t win = __ballot_sync(kFull, acc != 0 && rr == 0);
        if (win) {
            const uint32_t fl = __ffs(win) - 1;
            d = W * (w0 + (fl >> LG)) + Wn::first(Wn::shfl(acc, fl));
            return true;
        }
    }
    return false;
}

// any two equal master hashes among keys[0..k)?
__device__ bool bucket_has_dup(const uint64_t* keys, uint32_t k, uint32_t lane) {
    bool dup = false;
    for (uint32_t i = lane; i < k && !dup; i += 32) {
        uint64_t x = keys[i];
        for (uint32_t i2 = i + 1; i2 < k; i2++)
            if (keys[i2] == x) {
                dup = true;
                break;
            }
    }
    return __any_sync(kFull, dup);
}

// Outcomes of one candidate range (one s, or one run of XOR pilots) for one warp;
// the first range, in enumeration order, with a nonzero outcome decides.
constexpr uint32_t kOutNone = 0, kOutFound = 1, kOutDup = 2, kOutLimit = 3;

// Agreement among the warps of a CTA after each of them tested its own
// candidate range: publish (outcome, value), wait, and return the first warp in
// enumeration order whose outcome is final (or kWarps when none is).  The slots
// alternate between two banks so that the next round never overwrites a bank
// that another warp may still be reading.
template <int kWarps>
__device__ __forceinline__ uint32_t first_final(uint32_t* ctl, uint32_t& bank, uint32_t warp, uint32_t lane,
                                                uint32_t out, uint32_t val, uint32_t& w_out, uint32_t& w_val) {
    uint32_t* slot = ctl + bank * 2 * kWarps;
    if (lane == 0) {
        slot[2 * warp] = out;
        slot[2 * warp + 1] = val;
    }
    __syncthreads();
    uint32_t w = kWarps;
#pragma unroll
    for (int i = kWarps - 1; i >= 0; i--)
        if (slot[2 * i] != kOutNone) w = (uint32_t)i;
    if (w < kWarps) {
        w_out = slot[2 * w];
        w_val = slot[2 * w + 1];
    }
    bank ^= 1u;
    return w;
}

// kKeysInSmem: the partition's bucket-sorted master hashes live in shared
// memory (fewest latency, ~8 B/key of shared memory per partition); otherwise
// they are written to a global scratch region (the same index range as the
// sorted input, L2-resident while the partition is active).  Each bucket's keys
// are prefetched into registers one bucket ahead, and shared memory shrinks to
// the bitmaps and counters, so several times more partitions fit on an SM.
//
// kWarps > 1 warps share one partition.  Bucketing and ordering are split over
// the CTA (scans by warp 0).  In the placement of a bucket, warp w tests the
// (w+1)-th next candidate range: s = s0 + w in ADDITIVE mode, pilots
// p0 + w G .. p0 + w G + G - 1 in XOR mode.  The CTA then takes the first range
// in enumeration order with a final outcome (placed, duplicate or limit), which
// is the outcome a single sequential search reaches first.  The singleton
// buckets come last in the order and are placed by warp 0 alone.
template <bool kKeysInSmem, int kW, int kMode, int kWarps>
__device__ __forceinline__ void search_partition(const SearchLaunch& a, const SearchSet& S, const uint64_t gid,
                                                 const uint64_t j, unsigned char* smem, const SmemLayout& L) {
    using Wn = Win<kW>;
    using WT = typename Wn::T;
    constexpr uint32_t NT = 32 * kWarps;
    uint32_t* bend = reinterpret_cast<uint32_t*>(smem + L.off_bend);
    uint32_t* order = reinterpret_cast<uint32_t*>(smem + L.off_order);
    uint32_t* fw = reinterpret_cast<uint32_t*>(smem + L.off_fw);
    uint16_t* aux = reinterpret_cast<uint16_t*>(smem + L.off_aux);
    uint32_t* ctl = reinterpret_cast<uint32_t*>(smem + L.off_ctl);  // kWarps > 1 only

    const uint32_t tid = threadIdx.x;
    const uint32_t lane = tid & 31, warp = kWarps == 1 ? 0u : tid >> 5;
    uint32_t* scr = reinterpret_cast<uint32_t*>(smem + L.off_scr) + warp * L.scr_words;
    uint16_t* hb = aux + warp * kSizeHist;  // this warp's h values of the bucket's keys
    const uint64_t s0 = a.start[gid];
    const uint32_t nj = (uint32_t)(a.start[gid + 1] - s0);
    const uint64_t Tj = a.T[gid];
    const uint32_t m = (uint32_t)(a.T[gid + 1] - Tj);
    const uint32_t B = S.B;
    const uint64_t* const table = S.table;
    uint32_t* const pil = a.pilots + S.pilot_base + j;  // pilot of bucket b at pil[b * S.np]
    if (nj == 0) return;
    uint64_t* hk = kKeysInSmem ? reinterpret_cast<uint64_t*>(smem + L.off_hk) : a.bkeys + s0;

    // ---- init: counts, doubled free bitmap, scratch, size histogram
    for (uint32_t b = tid; b <= B; b += NT) bend[b] = 0;
    const uint32_t fwn = (2 * m + 128) / 32 + 3;
    for (uint32_t w = tid; w < fwn; w += NT) {
        uint32_t lo = w * 32, v;
        if (lo + 32 <= 2 * m)
            v = kFull;
        else if (lo >= 2 * m)
            v = 0;
        else
            v = (1u << (2 * m - lo)) - 1;
        fw[w] = v;
    }
    {
        uint32_t* scr0 = reinterpret_cast<uint32_t*>(smem + L.off_scr);
        const uint32_t sw = (m + 31) / 32 + 1;
        for (uint32_t w = tid; w < kWarps * L.scr_words; w += NT)
            if (w % L.scr_words < sw) scr0[w] = 0;
    }
    for (uint32_t i = tid; i < kSizeHist; i += NT) aux[i] = 0;
    cta_sync<kWarps>();

    // ---- 1. bucket counts, then counting sort of the keys by bucket
    for (uint32_t i = tid; i < nj; i += NT) {
        uint64_t x = __ldg(a.sorted + s0 + i);
        atomicAdd(&bend[bucket_of(bucket_hash(x), table, B)], 1u);
    }
    cta_sync<kWarps>();
    uint32_t local_err = kDevOk;
    if (warp == 0) {
        uint32_t carry = 0;
        for (uint32_t b0 = 0; b0 < B; b0 += 32) {
            uint32_t b = b0 + lane;
            uint32_t c = b < B ? bend[b] : 0;
            if (c > kMaxBucket) local_err = kDevSearchLimit;
            uint32_t x = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(kFull, x, o);
                if (lane >= (uint32_t)o) x += y;
            }
            if (b < B) bend[b] = carry + x - c;  // start of bucket b (cursor)
            carry += __shfl_sync(kFull, x, 31);
        }
        local_err = __reduce_max_sync(kFull, local_err);
    }
    cta_sync<kWarps>();
    for (uint32_t i = tid; i < nj; i += NT) {
        uint64_t x = __ldg(a.sorted + s0 + i);
        uint32_t b = bucket_of(bucket_hash(x), table, B);
        hk[atomicAdd(&bend[b], 1u)] = x;
    }
    cta_sync<kWarps>();
    // now bend[b] = end of bucket b; start of b = b ? bend[b-1] : 0

    // ---- 2. bucket order: size descending, index descending (warp 0)
    uint32_t nb = 0;
    if (warp == 0 && local_err == kDevOk) {
        for (uint32_t b = lane; b < B; b += 32) {
            uint32_t sz = bend[b] - (b ? bend[b - 1] : 0);
            if (sz) atomicAdd(reinterpret_cast<unsigned int*>(aux + (sz & ~1u)), 1u << ((sz & 1) * 16));
        }
        __syncwarp();
        // cum[s] = number of buckets larger than s, computed from the top
        {
            uint32_t carry = 0;
            for (int s0i = kSizeHist - 32; s0i >= 0; s0i -= 32) {
                uint32_t s = (uint32_t)s0i + (31 - lane);  // lane 0 takes the largest size of the chunk
                uint32_t c = aux[s];
                uint32_t x = c;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    uint32_t y = __shfl_up_sync(kFull, x, o);
                    if (lane >= (uint32_t)o) x += y;
                }
                __syncwarp();
                aux[s] = (uint16_t)(carry + x - c);
                carry += __shfl_sync(kFull, x, 31);
            }
        }
        __syncwarp();
        for (uint32_t c0 = 0; c0 < B; c0 += 32) {
            uint32_t idx = c0 + lane;
            uint32_t b = idx < B ? B - 1 - idx : 0;
            uint32_t sz = idx < B ? bend[b] - (b ? bend[b - 1] : 0) : 0;
            uint32_t peers = __match_any_sync(kFull, sz);
            if (sz) {
                uint32_t base = aux[sz];
                uint32_t r = __popc(peers & ((1u << lane) - 1));
                order[base + r] = b;
            }
            __syncwarp();
            if (sz && lane == (uint32_t)(__ffs(peers) - 1)) aux[sz] = (uint16_t)(aux[sz] + __popc(peers));
            nb += __popc(__ballot_sync(kFull, sz != 0));
            __syncwarp();
        }
    }
    if constexpr (kWarps > 1) {
        if (tid == 0) {
            ctl[4 * kWarps] = nb;
            ctl[4 * kWarps + 1] = local_err;
        }
        __syncthreads();
        nb = ctl[4 * kWarps];
        local_err = ctl[4 * kWarps + 1];
    }
    uint32_t bank = 0;  // kWarps > 1: control bank of the next agreement round

    // ---- 3. placement
    unsigned long long s_tries = 0, steps = 0;
    const uint32_t nw = (m + kW - 1) / kW;  // windows of kW displacements
    uint32_t placed = 0;  // keys placed so far in this partition
    // pilot seeds mix64(s ^ C) for s < 32, one per lane (most buckets need s < 32)
    const uint64_t ps_lane = pilot_seed(lane);
    // one key per lane of the next bucket, loaded a bucket ahead
    uint64_t pre = 0;
    if (nb) {
        const uint32_t b = order[0], bs = b ? bend[b - 1] : 0;
        if (lane < bend[b] - bs) pre = hk[bs + lane];
    }
    for (uint32_t r = 0; r < nb && local_err == kDevOk; r++) {
        const uint32_t b = order[r];
        const uint32_t bs = b ? bend[b - 1] : 0;
        const uint32_t k = bend[b] - bs;
        const uint64_t* keys = hk + bs;
        const uint64_t mykey = pre;
        if (r + 1 < nb) {
            const uint32_t bn = order[r + 1], bsn = bn ? bend[bn - 1] : 0;
            pre = lane < bend[bn] - bsn ? hk[bsn + lane] : 0;
        }
        uint32_t p = 0;
        if (kMode == 0) {
            // ===== additive displacement =====
            if (k == 1) {
                // Every bucket from here on holds one key (buckets come in size
                // order): s = 0 always succeeds, and d is the distance from h to
                // the next free slot.  Warp 0 hashes 32 of these keys at a time,
                // one per lane, then places them one after another.
                if (kWarps > 1 && warp != 0) break;
                const uint64_t ps0 = __shfl_sync(kFull, ps_lane, 0);
                for (uint32_t r1 = r; r1 < nb && local_err == kDevOk; r1 += 32) {
                    const uint32_t cnt = min(32u, nb - r1);
                    uint32_t bl = 0, hl = 0, dl = 0;
                    if (lane < cnt) {
                        bl = order[r1 + lane];
                        hl = position_hash(hk[bend[bl] - 1], ps0, m);
                    }
                    for (uint32_t i = 0; i < cnt; i++) {
                        const uint32_t h1 = __shfl_sync(kFull, hl, i);
                        s_tries++;
                        bool got = false;
                        uint32_t d1 = 0;
                        for (uint32_t w0 = 0; w0 < nw; w0 += 32) {
                            steps++;
                            const uint32_t w = w0 + lane;
                            WT acc = 0;
                            if (w < nw) acc = Wn::valid(w, m) & Wn::load(fw, h1 + kW * w);
                            const uint32_t win = __ballot_sync(kFull, acc != 0);
                            if (win) {
                                const uint32_t fl = __ffs(win) - 1;
                                d1 = kW * (w0 + fl) + Wn::first(Wn::shfl(acc, fl));
                                got = true;
                                break;
                            }
                        }
                        if (!got) {  // unreachable while the counts are consistent
                            local_err = kDevSearchLimit;
                            break;
                        }
                        if (lane == i) dl = d1;
                        if (lane == 0) {
                            uint32_t pos = h1 + d1;
                            if (pos >= m) pos -= m;
                            take_slot(fw, pos, m);
                        }
                        __syncwarp();
                    }
                    if (local_err == kDevOk && lane < cnt) pil[(uint64_t)bl * S.np] = dl;
                    placed += cnt;
                }
                break;
            }
            uint32_t d = 0;
            uint32_t sb = 0;           // first s of this round
            uint32_t winner = 0;       // warp whose s decided
            uint32_t outcome = kOutNone;
            // lanes per window: chosen once per bucket from the current load
            const uint32_t lg = choose_lanes_log2<kW>(k, m - placed, m);  // lanes per window: 2^lg
            uint64_t bigkey[kBigRegs];
            if (k > 32) {
#pragma unroll
                for (int t = 0; t < kBigRegs; t++) {
                    const uint32_t i = lane + 32 * t;
                    bigkey[t] = i < k ? keys[i] : 0;
                }
            }
            for (;; sb += kWarps) {
                const uint32_t s = sb + warp;
                uint32_t my = kOutNone, myd = 0;
                // seeds s < min(s_max, floor((2^32 - 1) / m)): the requested limit, and
                // never past the largest s whose pilots s m + d all fit 32 bits
                // (s >= floor(X / m) exactly when (s + 1) m > X).  Below s_fast, the
                // same bound for the launch's largest m, neither can hold.
                bool at_limit = false;
                if (__builtin_expect(s >= a.s_fast, 0)) at_limit = s >= a.s_max || (uint64_t)(s + 1) * m > 0xFFFFFFFFull;
                if (at_limit) {
                    my = kOutLimit;
                } else {
                    uint64_t ps;
                    if (s < 32)  // warp-uniform branch: never evaluate both sides
                        ps = __shfl_sync(kFull, ps_lane, s);
                    else
                        ps = pilot_seed(s);
                    bool coll = false;
                    if (k <= 32) {
                        const uint32_t h = lane < k ? position_hash(mykey, ps, m) : 0u;
                        if (lane < k) hb[lane] = (uint16_t)h;
                        // two keys on one slot: mark each slot in the warp's
                        // scratch bitmap and look at the bit's old value
                        bool c = false;
                        if (lane < k) {
                            const uint32_t bit = 1u << (h & 31);
                            c = (atomicOr(&scr[h >> 5], bit) & bit) != 0;
                        }
                        coll = __any_sync(kFull, c);
                        if (lane < k) scr[h >> 5] = 0;
                    } else {
                        // large bucket: up to kBigRegs keys per lane stay in registers
                        // across s values; the rest are re-read from the key store
                        bool c = false;
                        uint32_t hv[kBigRegs];
#pragma unroll
                        for (int t = 0; t < kBigRegs; t++) {
                            const uint32_t i = lane + 32 * t;
                            hv[t] = i < k ? position_hash(bigkey[t], ps, m) : 0;
                        }
#pragma unroll
                        for (int t = 0; t < kBigRegs; t++) {
                            const uint32_t i = lane + 32 * t;
                            if (i < k) {
                                hb[i] = (uint16_t)hv[t];
                                const uint32_t bit = 1u << (hv[t] & 31);
                                if (atomicOr(&scr[hv[t] >> 5], bit) & bit) c = true;
                            }
                        }
                        for (uint32_t i = lane + 32 * kBigRegs; i < k; i += 32) {
                            uint32_t hi = position_hash(keys[i], ps, m);
                            hb[i] = (uint16_t)hi;
                            uint32_t bit = 1u << (hi & 31);
                            if (atomicOr(&scr[hi >> 5], bit) & bit) c = true;
                        }
                        coll = __any_sync(kFull, c);
                        for (uint32_t i = lane; i < k; i += 32) scr[hb[i] >> 5] = 0;
                    }
                    __syncwarp();
                    if (coll) {
                        if (s == 8 && bucket_has_dup(keys, k, lane)) my = kOutDup;
                    } else {
                        bool f;
                        switch (lg) {
                            case 0: f = scan_windows<kW, 0>(fw, hb, k, m, nw, lane, myd, steps); break;
                            case 1: f = scan_windows<kW, 1>(fw, hb, k, m, nw, lane, myd, steps); break;
                            case 2: f = scan_windows<kW, 2>(fw, hb, k, m, nw, lane, myd, steps); break;
                            case 3: f = scan_windows<kW, 3>(fw, hb, k, m, nw, lane, myd, steps); break;
                            case 4: f = scan_windows<kW, 4>(fw, hb, k, m, nw, lane, myd, steps); break;
                            default: f = scan_windows<kW, 5>(fw, hb, k, m, nw, lane, myd, steps); break;
                        }
                        if (f) my = kOutFound;
                    }
                }
                if constexpr (kWarps == 1) {
                    if (my != kOutLimit) s_tries++;
                    if (my != kOutNone) {
                        outcome = my;
                        d = myd;
                        break;
                    }
                } else {
                    uint32_t wo = kOutNone, wv = 0;
                    const uint32_t w = first_final<kWarps>(ctl, bank, warp, lane, my, myd, wo, wv);
                    if (w < kWarps) {
                        outcome = wo;
                        d = wv;
                        winner = w;
                        s_tries += w + (wo == kOutLimit ? 0 : 1);
                        break;
                    }
                    s_tries += kWarps;
                }
            }
            if (outcome != kOutFound) {
                local_err = outcome == kOutDup ? kDevDupHash : kDevSearchLimit;
                break;
            }
            p = (sb + winner) * m + d;
            if (warp == winner) {
                for (uint32_t i = lane; i < k; i += 32) {
                    uint32_t pos = (uint32_t)hb[i] + d;
                    if (pos >= m) pos -= m;
                    take_slot(fw, pos, m);
                }
            }
            placed += k;
        } else {
            // ===== PTHash XOR form: p = 0, 1, 2, ... =====
            const uint64_t limit = (uint64_t)min(a.s_max, 0xFFFFFFFFu / m) * m;  // pilots < 2^32
            uint32_t outcome = kOutNone, winner = 0;
            // Expected candidates about q^-k (q the free fraction).  When they exceed
            // what one step of the grouped scan below covers (floor(32 / k) pilots),
            // the filter cascade takes the bucket instead.
            const float xq = __fdividef((float)(m - placed), (float)m);
            const bool cascade = k <= 32 && (float)k * -__log2f(xq) > __log2f((float)(32u / k));
            if (cascade) {
                // Filter cascade over windows of 32 consecutive pilots, one pilot per
                // lane: every lane tests the bucket's key 0 under its pilot, then the
                // lanes whose slot was free test key 1, and so on, while any lane's
                // pilot still has all of its slots free.  On a filling table most
                // pilots fail on their first keys, so a window costs about 1 / (1 - q)
                // slot tests per pilot instead of k.  The surviving pilots are then
                // checked for pairwise distinct slots in increasing order, so the first
                // that passes is the smallest valid pilot of the window.
                const uint64_t kv = lane < k ? keys[lane] : 0;  // key r on lane r
                uint32_t mypos = 0;
                for (uint64_t pb = 0;; pb += (uint64_t)kWarps * 32) {
                    const uint64_t p0 = pb + (uint64_t)warp * 32;
                    uint32_t my = kOutNone, myp = 0;
                    if (p0 >= limit) {
                        my = kOutLimit;
                    } else if (p0 <= 8ull * m && 8ull * m < p0 + 32 && bucket_has_dup(keys, k, lane)) {
                        my = kOutDup;  // the window holding pilot 8 m checks for duplicates
                    } else {
                        steps++;
                        const uint64_t pc = p0 + lane;
                        const uint64_t ps = pilot_seed(pc);
                        bool alive = pc < limit;
                        for (uint32_t r = 0; r < k; r++) {
                            const uint64_t kr = __shfl_sync(kFull, kv, r);
                            if (alive) {
                                const uint32_t pos = position_hash(kr, ps, m);
                                alive = (fw[pos >> 5] >> (pos & 31)) & 1;
                            }
                            if (!__any_sync(kFull, alive)) break;
                        }
                        uint32_t cand = __ballot_sync(kFull, alive);
                        while (cand) {
                            const uint32_t l = __ffs(cand) - 1;
                            cand &= cand - 1;
                            const uint32_t pos = position_hash(kv, __shfl_sync(kFull, ps, l), m);
                            if (k > 1) {
                                // pairwise distinct slots: mark them in the warp's scratch bitmap
                                bool c = false;
                                if (lane < k) {
                                    const uint32_t bit = 1u << (pos & 31);
                                    c = (atomicOr(&scr[pos >> 5], bit) & bit) != 0;
                                }
                                const bool coll = __any_sync(kFull, c);
                                if (lane < k) scr[pos >> 5] = 0;
                                __syncwarp();
                                if (coll) continue;
                            }
                            my = kOutFound;
                            myp = (uint32_t)(p0 + l);
                            mypos = pos;
                            break;
                        }
                    }
                    if constexpr (kWarps == 1) {
                        if (my != kOutNone) {
                            outcome = my;
                            p = myp;
                            break;
                        }
                    } else {
                        uint32_t wo = kOutNone, wv = 0;
                        const uint32_t w = first_final<kWarps>(ctl, bank, warp, lane, my, myp, wo, wv);
                        if (w < kWarps) {
                            outcome = wo;
                            p = wv;
                            winner = w;
                            break;
                        }
                    }
                }
                if (outcome != kOutFound) {
                    local_err = outcome == kOutDup ? kDevDupHash : kDevSearchLimit;
                    break;
                }
                if (warp == winner && lane < k) take_slot(fw, mypos, m);
                placed += k;
            } else if (k <= 32) {
                // groups of k lanes test G = floor(32 / k) consecutive pilots per warp
                // step (lanes g >= G idle): lane rr of group g hashes key rr with pilot
                // p0 + g.  A group wins when its k slots are free and pairwise
                // distinct; distinctness is looked at only in steps where some group
                // has all its slots free
                const uint32_t G = 32u / k;
                const uint32_t g = lane / k, rr = lane - g * k;
                const bool act = g < G;
                const uint64_t gkey = act ? keys[rr] : 0;
                const uint32_t gmask = k == 32 ? kFull : ((1u << k) - 1);
                uint32_t mypos = 0;
                // pilot seeds of 32 consecutive pilots from cb on, one per lane (one
                // warp per partition, G < 32)
                uint64_t cb = 0, ps_cache = pilot_seed(lane);
                for (uint64_t pb = 0;; pb += (uint64_t)kWarps * G) {
                    const uint64_t p0 = pb + (uint64_t)warp * G;
                    uint32_t my = kOutNone, myp = 0, pos = 0;
                    if (p0 >= limit) {
                        my = kOutLimit;
                    } else if (p0 >= 8ull * m && p0 < 8ull * m + G && bucket_has_dup(keys, k, lane)) {
                        my = kOutDup;  // the first step at or past 8 m checks for duplicates
                    } else {
                        steps++;
                        const uint64_t pc = p0 + g;
                        bool free_slot = false;  // idle lanes and pilots past the limit count as taken
                        uint64_t ps;
                        if (G == 32 || kWarps > 1) {
                            // singletons need a new seed in every lane at every step, and
                            // several warps per partition jump past the cache every round
                            ps = pilot_seed(pc);
                        } else {
                            if (p0 + G > cb + 32) {  // warp-uniform: refill the seed cache from p0
                                cb = p0;
                                ps_cache = pilot_seed(cb + lane);
                            }
                            ps = __shfl_sync(kFull, ps_cache, (uint32_t)(p0 - cb) + (act ? g : 0u));
                        }
                        if (act && pc < limit) {
                            pos = position_hash(gkey, ps, m);
                            free_slot = (fw[pos >> 5] >> (pos & 31)) & 1;
                        }
                        const uint32_t taken = __ballot_sync(kFull, !free_slot);
                        const bool gfree = act && ((taken >> (g * k)) & gmask) == 0;
                        if (__ballot_sync(kFull, gfree && rr == 0)) {
                            const uint32_t key = gfree ? ((g << 20) | pos) : (0xFFFFFFFFu - lane);  // filler never a slot
                            const uint32_t peers = __match_any_sync(kFull, key);
                            const uint32_t dup = __ballot_sync(kFull, gfree && __popc(peers) > 1);
                            const bool gok = gfree && ((dup >> (g * k)) & gmask) == 0;
                            const uint32_t win = __ballot_sync(kFull, gok && rr == 0);
                            if (win) {
                                const uint32_t fl = __ffs(win) - 1;  // first lane of the winning group
                                my = kOutFound;
                                myp = (uint32_t)(p0 + fl / k);
                                mypos = __shfl_sync(kFull, pos, fl + (lane < k ? lane : 0u));
                            }
                        }
                    }
                    if constexpr (kWarps == 1) {
                        if (my != kOutNone) {
                            outcome = my;
                            p = myp;
                            break;
                        }
                    } else {
                        uint32_t wo = kOutNone, wv = 0;
                        const uint32_t w = first_final<kWarps>(ctl, bank, warp, lane, my, myp, wo, wv);
                        if (w < kWarps) {
                            outcome = wo;
                            p = wv;
                            winner = w;
                            break;
                        }
                    }
                }
                if (outcome != kOutFound) {
                    local_err = outcome == kOutDup ? kDevDupHash : kDevSearchLimit;
                    break;
                }
                if (warp == winner && lane < k) take_slot(fw, mypos, m);
                placed += k;
            } else {
                for (uint64_t pb = 0;; pb += kWarps) {
                    const uint64_t pc = pb + warp;
                    uint32_t my = kOutNone;
                    if (pc >= limit) {
                        my = kOutLimit;
                    } else if (pc == 8ull * m && bucket_has_dup(keys, k, lane)) {
                        my = kOutDup;
                    } else {
                        steps++;
                        const uint64_t ps = pilot_seed(pc);
                        bool bad = false;
                        for (uint32_t i = lane; i < k; i += 32) {
                            uint32_t pos = position_hash(keys[i], ps, m);
                            hb[i] = (uint16_t)pos;
                            uint32_t bit = 1u << (pos & 31);
                            if (!((fw[pos >> 5] >> (pos & 31)) & 1)) bad = true;
                            if (atomicOr(&scr[pos >> 5], bit) & bit) bad = true;
                        }
                        bool anybad = __any_sync(kFull, bad);
                        for (uint32_t i = lane; i < k; i += 32) scr[hb[i] >> 5] = 0;
                        __syncwarp();
                        if (!anybad) my = kOutFound;
                    }
                    if constexpr (kWarps == 1) {
                        if (my != kOutNone) {
                            outcome = my;
                            p = (uint32_t)pc;
                            break;
                        }
                    } else {
                        uint32_t wo = kOutNone, wv = 0;
                        const uint32_t w = first_final<kWarps>(ctl, bank, warp, lane, my, (uint32_t)pc, wo, wv);
                        if (w < kWarps) {
                            outcome = wo;
                            p = wv;
                            winner = w;
                            break;
                        }
                    }
                }
                if (outcome != kOutFound) {
                    local_err = outcome == kOutDup ? kDevDupHash : kDevSearchLimit;
                    break;
                }
                if (warp == winner)
                    for (uint32_t i = lane; i < k; i += 32) take_slot(fw, hb[i], m);
                placed += k;
            }
        }
        cta_sync<kWarps>();
        if (tid == 0) pil[(uint64_t)b * S.np] = p;
    }

    if constexpr (kWarps > 1) {
        // warp 0 alone may have run on (singletons): its error word decides
        __syncthreads();
        if (tid == 0) ctl[4 * kWarps + 1] = local_err;
        __syncthreads();
        local_err = ctl[4 * kWarps + 1];
    }
    if (local_err != kDevOk) {
        if (warp == 0) {
            // a duplicate anywhere in the partition takes precedence over other errors
            if (local_err != kDevDupHash) {
                for (uint32_t b = 0; b < B; b++) {
                    uint32_t bs = b ? bend[b - 1] : 0, k = bend[b] - bs;
                    if (k > 1 && bucket_has_dup(hk + bs, k, lane)) {
                        local_err = kDevDupHash;
                        break;
                    }
                }
            }
            if (lane == 0) atomicMax(a.status, local_err);
        }
        return;
    }
    if (a.work && lane == 0) {
        if (warp == 0) atomicAdd(a.work, s_tries);
        atomicAdd(a.work + 1, steps);
    }

    // ---- 4. taken slots into the global occupancy bitmap at bit offset T_j
    if (a.taken_bits && m) {
        const uint64_t o0 = Tj >> 5, o1 = (Tj + m - 1) >> 5;
        for (uint64_t o = o0 + tid; o <= o1; o += NT) {
            int64_t t0 = (int64_t)(o * 32) - (int64_t)Tj;
            uint32_t v;
            if (t0 >= 0) {
                uint32_t tt = (uint32_t)t0;
                v = ~window32(fw, tt);
                if (tt + 32 > m) v &= (m - tt >= 32) ? kFull : ((1u << (m - tt)) - 1);
            } else {
                uint32_t sh = (uint32_t)(-t0);
                v = ~(fw[0] << sh) & ~((1u << sh) - 1);
                if (m + sh < 32) v &= (1u << (m + sh)) - 1;
            }
            if (v) atomicOr(a.taken_bits + o, v);
        }
    }
}

// kWarps warps per CTA, one partition per CTA at a time.  kQueue = true:
// persistent kernel, every CTA takes the next partition (a global partition id
// over every key set of the launch) from a device work queue until none are
// left.  kQueue = false: CTA g processes partition g.  Neither the order in which
// partitions are processed nor the number of warps changes any result.
template <bool kKeysInSmem, int kW, int kMode, bool kQueue, int kWarps>
__global__ void __launch_bounds__(32 * kWarps, 32 / kWarps) k_search(SearchLaunch a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const SmemLayout L = smem_layout(a.cap_n, a.cap_m, a.cap_B, kKeysInSmem, kWarps);
    unsigned long long gid = blockIdx.x;
    for (;;) {
        if (kQueue) {
            if constexpr (kWarps == 1) {
                if (threadIdx.x == 0) gid = atomicAdd(a.queue, 1ull);
                gid = __shfl_sync(kFull, gid, 0);
            } else {
                unsigned long long* slot = reinterpret_cast<unsigned long long*>(smem + L.total);
                if (threadIdx.x == 0) *slot = atomicAdd(a.queue, 1ull);
                __syncthreads();
                gid = *slot;
            }
            if (gid >= a.total_parts) break;
        }
        uint32_t lo = 0, hi = a.nsets;  // key set: largest s with part_base <= gid
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (a.sets[mid].part_base <= gid) lo = mid; else hi = mid;
        }
        const SearchSet S = a.sets[lo];
        search_partition<kKeysInSmem, kW, kMode, kWarps>(a, S, gid, gid - S.part_base, smem, L);
        if (!kQueue) break;
        cta_sync<kWarps>();
    }
}

// m_j from the partition starts (alpha = 1: m_j = n_j; else ceil(n_j / alpha) in
// IEEE double), plus the largest n_j and m_j
__global__ void __launch_bounds__(256) k_table_sizes(const uint64_t* __restrict__ start, uint64_t np, double alpha,
                                                     uint32_t* __restrict__ m_out,
                                                     unsigned long long* __restrict__ maxima) {
    unsigned long long mn = 0, mm = 0;
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < np; j += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t nj = start[j + 1] - start[j], mj;
        if (alpha == 1.0) {
            mj = nj;
        } else {
            mj = (uint64_t)ceil((double)nj / alpha);
            if (mj < nj) mj = nj;
        }
        m_out[j] = (uint32_t)(mj < 0xFFFFFFFFull ? mj : 0xFFFFFFFFull);
        mn = max(mn, (unsigned long long)nj);
        mm = max(mm, (unsigned long long)mj);
    }
    for (int o = 16; o; o >>= 1) {
        mn = max(mn, __shfl_xor_sync(kFull, mn, o));
        mm = max(mm, __shfl_xor_sync(kFull, mm, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(maxima, mn);
        atomicMax(maxima + 1, mm);
    }
}

__global__ void k_gather_u64(const uint64_t* __restrict__ src, const uint64_t* __restrict__ idx,
                             uint64_t* __restrict__ out, uint64_t count) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = src[idx[i]];
}

}  // namespace

cudaError_t launch_gather_u64(const uint64_t* src, const uint64_t* idx, uint64_t* out, uint64_t count,
                              cudaStream_t stream) {
    if (count == 0) return cudaSuccess;
    uint64_t blocks = (count + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_gather_u64<<<(unsigned)blocks, 256, 0, stream>>>(src, idx, out, count);
    note_launches(1);
    return cudaGetLastError();
}

size_t search_smem_bytes(uint32_t cap_n, uint32_t cap_m, uint32_t B, bool keys_in_smem, uint32_t warps) {
    // plus one 8-byte slot for the queue's partition id when several warps share a CTA
    return smem_layout(cap_n, cap_m, B, keys_in_smem, warps).total + (warps > 1 ? 16 : 0);
}

size_t search_smem_limit() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return (size_t)v;
}

namespace {
using SearchKernel = void (*)(SearchLaunch);

template <bool SM, int W, int MD, int WP>
SearchKernel pick_queue(bool q) {
    return q ? k_search<SM, W, MD, true, WP> : k_search<SM, W, MD, false, WP>;
}

template <int WP>
SearchKernel pick_kernel(const SearchLaunch& a) {
    const bool in_smem = a.keys_in_smem != 0, q = a.use_queue != 0;
    if (a.mode != 0)  // PTHash XOR pilots: the window width does not apply
        return in_smem ? pick_queue<true, 32, 1, WP>(q) : pick_queue<false, 32, 1, WP>(q);
    if (a.window_bits == 64)
        return in_smem ? pick_queue<true, 64, 0, WP>(q) : pick_queue<false, 64, 0, WP>(q);
    return in_smem ? pick_queue<true, 32, 0, WP>(q) : pick_queue<false, 32, 0, WP>(q);
}
}  // namespace

cudaError_t launch_search(const SearchLaunch& a, cudaStream_t stream) {
    const uint32_t wp = a.warps;
    if (wp != 1 && wp != 2 && wp != 4 && wp != 8) return cudaErrorInvalidValue;
    const size_t smem = search_smem_bytes(a.cap_n, a.cap_m, a.cap_B, a.keys_in_smem != 0, wp);
    const SearchKernel kern = wp == 1   ? pick_kernel<1>(a)
                              : wp == 2 ? pick_kernel<2>(a)
                              : wp == 4 ? pick_kernel<4>(a)
                                        : pick_kernel<8>(a);
    const bool q = a.use_queue != 0;
    cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void*>(kern));
    if (e != cudaSuccess) return e;
    uint64_t grid = a.total_parts;
    if (q) {
        int dev = 0, sms = 148, per_sm = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * wp, smem)) != cudaSuccess)
            return e;
        if (per_sm < 1) per_sm = 1;
        grid = (uint64_t)sms * per_sm;  // persistent: every CTA resident, work from the queue
        if (grid > a.total_parts) grid = a.total_parts;
        if ((e = cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), stream)) != cudaSuccess) return e;
    }
    if (grid == 0) return cudaSuccess;
    if (grid > 0x7FFFFFFFull) return cudaErrorInvalidValue;
    kern<<<(unsigned)grid, 32 * wp, smem, stream>>>(a);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_sizes(const uint64_t* start, uint64_t np, double alpha, uint64_t* T, uint64_t* stats,
                         void* scratch, cudaStream_t stream) {
    // scratch: m_j (u32, np) | scan tile sums; stats[0] = M, stats[1] = max n_j, stats[2] = max m_j
    uint32_t* m = static_cast<uint32_t*>(scratch);
    unsigned long long* tiles = reinterpret_cast<unsigned long long*>(
        static_cast<unsigned char*>(scratch) + ((np * 4 + 15) & ~uint64_t(15)));
    cudaError_t e = cudaMemsetAsync(stats, 0, 3 * sizeof(uint64_t), stream);
    if (e != cudaSuccess) return e;
    uint64_t blocks = (np + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_table_sizes<<<(unsigned)blocks, 256, 0, stream>>>(start, np, alpha, m,
                                                        reinterpret_cast<unsigned long long*>(stats + 1));
    note_launches(1);
    e = exclusive_scan_u32(m, np, reinterpret_cast<unsigned long long*>(T), tiles, stream);
    if (e != cudaSuccess) return e;
    // T[np] = M = grand total; stats[0] = M
    e = cudaMemcpyAsync(T + np, scan_total(tiles, np), sizeof(uint64_t), cudaMemcpyDeviceToDevice, stream);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(stats, T + np, sizeof(uint64_t), cudaMemcpyDeviceToDevice, stream);
}

size_t sizes_scratch_bytes(uint64_t np) { return ((np * 4 + 15) & ~uint64_t(15)) + scan_tiles_bytes(np); }

}  // namespace phobic
