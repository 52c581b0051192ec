// K8: query.  For each key (Section 4, "Hash Function", and Section 4.1):
//   hk = master hash; j = partition; T_j and T_{j+1} decoded from the offsets
//   stored as differences to their expectation; m = T_{j+1} - T_j;
//   b = bucket of hk; p = pilot of bucket b in partition j (interleaved
//   Compact or Dictionary column b, entry j);
//   additive: local = (h(x, floor(p/m)) + p) mod m;  XOR: local = h(x xor h(p));
//   g = T_j + local, remapped through Elias-Fano when g >= n.
// Keys are read and results written coalesced (two keys per thread through
// 16-byte accesses when aligned); the structure (offsets, column metadata,
// packed pilots, remap) is a few tens of MB and stays L2-resident, read through
// the read-only path.
#include "phobic_dev.cuh"
#include "phobic_kernels.cuh"
#include "phobic_xxh64.cuh"

namespace phobic {

namespace {

constexpr uint64_t kMeta = (1ull << 56) - 1;

// T_j and T_{j+1}: the two stored differences are adjacent (2w <= 62 bits), so
// one 128-bit window of the packed words holds both.  kNarrow: read the second
// word only when the pair runs into it.
template <bool kNarrow>
__device__ __forceinline__ void offsets_of(const QueryView& v, uint64_t j, uint64_t* Tj, uint64_t* Tj1) {
    const uint32_t w = v.off_w;
    uint64_t d0 = 0, d1 = 0;
    if (w) {
        const uint64_t o = j * w;
        const uint64_t i = o >> 6;
        const uint32_t sh = (uint32_t)(o & 63);
        uint64_t x;
        if (kNarrow) {
            x = __ldg(v.off_words + i) >> sh;
            if (sh + 2 * w > 64) x |= __ldg(v.off_words + i + 1) << (64 - sh);  // sh > 0 here
        } else {
            const uint64_t lo = __ldg(v.off_words + i);
            x = sh ? (lo >> sh) | (__ldg(v.off_words + i + 1) << (64 - sh)) : lo;
        }
        const uint64_t mask = (1ull << w) - 1;
        d0 = x & mask;
        d1 = (x >> w) & mask;
    }
    *Tj = offset_expectation(j, v.off_Q) + (uint64_t)v.off_dmin + d0;
    *Tj1 = offset_expectation(j + 1, v.off_Q) + (uint64_t)v.off_dmin + d1;
}

__device__ __forceinline__ uint64_t offset_of(const QueryView& v, uint64_t j) {
    return offset_expectation(j, v.off_Q) + (uint64_t)v.off_dmin + read_bits(v.off_words, j * v.off_w, v.off_w);
}

// read_bits32 for narrow fields: the 64-bit word holding bit o, and the next
// word only when the field runs into it (for random o, with probability about
// w/64), which spares the cache the second access of most random reads
__device__ __forceinline__ uint32_t read_bits32_narrow(const uint64_t* __restrict__ words, uint32_t o, uint32_t w) {
    const uint32_t i = o >> 6, sh = o & 63;
    uint64_t x = __ldg(words + i) >> sh;
    if (sh + w > 64) x |= __ldg(words + i + 1) << (64 - sh);  // sh > 0 here
    return w >= 32 ? (uint32_t)x : ((uint32_t)x & ((1u << w) - 1));
}

// floor(p / m) for m >= 1 through a float reciprocal and an exact integer
// correction.  The float estimate has a relative error below 2^-21 (two
// conversions and two round-toward-zero operations) plus the truncation, so the
// loops run at most p / m 2^-21 + 2 times: once or twice for the pilots a build
// makes, whose s stays far below 2^21.
__device__ __forceinline__ uint32_t div_u32(uint32_t p, uint32_t m) {
    uint32_t q = __float2uint_rz(__fmul_rz((float)p, __frcp_rz((float)m)));
    int64_t r = (int64_t)p - (int64_t)q * m;
    while (r < 0) {
        q--;
        r += m;
    }
    while (r >= (int64_t)m) {
        q++;
        r -= m;
    }
    return q;
}

// floor(p / m) and p mod m for 1 <= m < 2^30, as div_u32 in 32-bit arithmetic:
// |p - q m| <= p 2^-21 + m < 2^31 for the estimate q, so the remainder is exact
// as a signed 32-bit value
__device__ __forceinline__ uint32_t div_small(uint32_t p, uint32_t m, uint32_t& rem) {
    uint32_t q = __float2uint_rz(__fmul_rz((float)p, __frcp_rz((float)m)));
    int32_t r = (int32_t)(p - q * m);
    while (r < 0) {
        q--;
        r += (int32_t)m;
    }
    while (r >= (int32_t)m) {
        q++;
        r -= (int32_t)m;
    }
    rem = (uint32_t)r;
    return q;
}

// Position of the r-th (0-based) set bit of w, which has more than r set bits:
// a binary search over halves, quarters, ... by popcount, in six fixed steps
// (no loop whose length depends on r, so the lanes of a warp stay together)
__device__ __forceinline__ uint32_t select_in_word(uint64_t w, uint32_t r) {
    uint32_t pos = 0, c;
    c = __popc((uint32_t)w);
    if (r >= c) { r -= c; w >>= 32; pos += 32; }
    c = __popc((uint32_t)w & 0xFFFFu);
    if (r >= c) { r -= c; w >>= 16; pos += 16; }
    c = __popc((uint32_t)w & 0xFFu);
    if (r >= c) { r -= c; w >>= 8; pos += 8; }
    c = __popc((uint32_t)w & 0xFu);
    if (r >= c) { r -= c; w >>= 4; pos += 4; }
    c = __popc((uint32_t)w & 0x3u);
    if (r >= c) { r -= c; w >>= 2; pos += 2; }
    if (r >= ((uint32_t)w & 1u)) pos += 1;
    return pos;
}

// i-th value of the Elias-Fano sequence
__device__ __forceinline__ uint64_t ef_access(const QueryView& v, uint64_t i) {
    uint64_t pos = __ldg(v.ef_samples + (i >> 6));
    uint32_t need = (uint32_t)(i & 63);  // ones to pass after the sampled one
    uint64_t wi = pos >> 6;
    uint64_t w = __ldg(v.ef_high + wi) & (~0ull << (pos & 63));
    for (;;) {
        uint32_t c = __popcll(w);
        if (need < c) break;
        need -= c;
        w = __ldg(v.ef_high + ++wi);
    }
    uint64_t one = wi * 64 + select_in_word(w, need);
    uint64_t low = read_bits(v.ef_low, i * v.ef_l, v.ef_l);
    return ((one - i) << v.ef_l) | low;
}

// first one at or after bit g of `words` (one exists)
__device__ __forceinline__ uint64_t next_one(const uint64_t* __restrict__ words, uint64_t g) {
    uint64_t wi = g >> 6;
    uint64_t w = __ldg(words + wi) & (~0ull << (g & 63));
    while (!w) w = __ldg(words + ++wi);
    return wi * 64 + (uint64_t)(__ffsll((long long)w) - 1);
}

// last one strictly before bit g of `words` (one exists)
__device__ __forceinline__ uint64_t prev_one(const uint64_t* __restrict__ words, uint64_t g) {
    uint64_t wi = g >> 6;
    uint64_t w = (g & 63) ? (__ldg(words + wi) & ((1ull << (g & 63)) - 1)) : 0;
    while (!w) w = __ldg(words + --wi);
    return wi * 64 + 63 - (uint64_t)__clzll((long long)w);
}

// Bits of the ones of partitions j - 1 and j in column b's select-sampled
// unary part (a = hb - 1 for j = 0): from the column's sample for partition
// 64 floor(j / 64), skipping ones with popcounts.  hb: the column's first bit.
__device__ __forceinline__ void unary_pair(const QueryView& v, uint32_t sc, uint64_t j, uint64_t hb, uint64_t* a_out,
                                           uint64_t* c_out) {
    // sc: the column's select-sample column (IC-CR: b - mix_c)
    const uint32_t* samples = reinterpret_cast<const uint32_t*>(v.dict_words) + (uint64_t)sc * v.rice_ns;
    const uint64_t* high = v.rice_high;
    const uint64_t s = hb + __ldg(samples + (j >> 6));  // bit of the one of partition 64 floor(j / 64)
    uint64_t a, c;
    if ((j & 63) == 0) {
        c = s;
        a = j ? prev_one(high, c) : hb - 1;
    } else {
        uint32_t need = (uint32_t)(j & 63) - 1;  // further ones after the sample's, up to partition j - 1
        a = s;
        if (need) {
            uint64_t wi = (s + 1) >> 6;
            uint64_t w = __ldg(high + wi) & (~0ull << ((s + 1) & 63));
            for (;;) {
                const uint32_t cnt = (uint32_t)__popcll(w);
                if (need <= cnt) break;
                need -= cnt;
                w = __ldg(high + ++wi);
            }
            a = wi * 64 + select_in_word(w, need - 1);
        }
        c = next_one(high, a + 1);
    }
    *a_out = a;
    *c_out = c;
}

// IC-R pilot of partition j in column b: the low part at width l, plus the
// unary part (the distance between the ones of partitions j-1 and j, minus one)
__device__ __forceinline__ uint32_t rice_pilot(const QueryView& v, uint32_t b, uint64_t j) {
    const uint64_t m0 = __ldg(v.col_meta + 2 * b), hb = __ldg(v.col_meta + 2 * b + 1);
    const uint32_t l = (uint32_t)(m0 >> 56);
    uint64_t a, c;
    unary_pair(v, b - v.mix_c, j, hb, &a, &c);
    const uint64_t q = c - a - 1;
    return (uint32_t)((q << l) | read_bits(v.pil_words, (m0 & kMeta) + j * l, l));
}

// IC-EF pilot of partition j in column b: E_j - E_{j-1}, each prefix sum from
// the position of its one (high part: position - index) and its low l bits
__device__ __forceinline__ uint32_t ef_column_pilot(const QueryView& v, uint32_t b, uint64_t j) {
    const uint64_t m0 = __ldg(v.col_meta + 2 * b), hb = __ldg(v.col_meta + 2 * b + 1);
    const uint32_t l = (uint32_t)(m0 >> 56);
    const uint64_t lb = m0 & kMeta;
    uint64_t a, c;
    unary_pair(v, b, j, hb, &a, &c);
    const uint64_t ej = ((c - hb - j) << l) | read_bits(v.pil_words, lb + j * l, l);
    const uint64_t ep = j ? (((a - hb - (j - 1)) << l) | read_bits(v.pil_words, lb + (j - 1) * l, l)) : 0;
    return (uint32_t)(ej - ep);
}

// A mono encoder (5..8: Compact, Dictionary, Rice, Elias-Fano over one column of
// all pilots): value i = b N_P + j of column 0
__device__ __forceinline__ uint32_t mono_pilot(const QueryView& v, uint64_t i) {
    const uint64_t m0 = __ldg(v.col_meta);
    const uint32_t w = (uint32_t)(m0 >> 56);
    switch (v.encoder) {
        case 5:
            return (uint32_t)read_bits(v.pil_words, (m0 & kMeta) + i * w, w);
        case 6: {
            const uint64_t dm = __ldg(v.col_meta + 1);
            const uint32_t dw = (uint32_t)(dm >> 56);
            const uint64_t r = read_bits(v.pil_words, (m0 & kMeta) + i * w, w);
            return (uint32_t)read_bits(v.dict_words, (dm & kMeta) + r * dw, dw);
        }
        case 7:
            return rice_pilot(v, 0, i);
        default:
            return ef_column_pilot(v, 0, i);
    }
}

constexpr int kSeedTable = 64;  // pilot seeds mix64(s ^ C) for s < 64, per block

// Kinds of query kernel, one instantiation each, so that no encoder's code is
// shaped by another's:
//   kQInterleaved: the interleaved encoders (0..4), chosen at run time;
//   kQMono: a mono encoder (5..8);
//   kQDict: IC-D.  Its two dependent narrow reads (rank, then dictionary entry)
//     leave the query bound by L1 accesses, so it reads a field's second word
//     only when the field runs into it (about w/64 of random offsets).  The other
//     encoders are bound by issue and keep the branch-free two-word reads.
constexpr int kQInterleaved = 0, kQMono = 1, kQDict = 2;

__host__ __forceinline__ int query_kind(const QueryView& v) {
    return v.encoder >= 5 ? kQMono : v.encoder == 1 ? kQDict : kQInterleaved;
}

// Structures whose partition arithmetic fits 32 bits (every structure of up to
// about 10^12 keys at the default partition size) take a second instantiation,
// k32, with no 64-bit multiplies outside the hashes:
//   - j = floor(hk N_P / 2^64) is fastrange onto N_P < 2^32 - 1;
//   - the offsets' bit positions (N_P + 1) w stay below 2^32;
//   - with Q = Qh 2^32 + Ql, the expectation floor(j Q / 2^32) is
//     j Qh + floor(j Ql / 2^32) for j < 2^32: one wide multiply-add and one high
//     multiply;
//   - floor(p / m) and p mod m take 32-bit arithmetic (div_small): every
//     m_j is below 2^16, since a build refuses larger partition tables and an
//     import checks the decoded offsets for it;
//   - the packed pilot arrays hold fewer than 2^32 bits (small_bits).
// The instantiation is chosen once per launch, so no key takes a branch for it.
__host__ __forceinline__ bool query_fast32(const QueryView& v) {
    if (v.NP >= 0xFFFFFFFFull || v.off_w > 31 || !v.small_bits) return false;
    return (v.NP + 1) * (uint64_t)v.off_w < (1ull << 32);
}

template <int kKind, bool k32>
__device__ __forceinline__ uint64_t query_hashed(const QueryView& v, uint64_t hk, const uint64_t* seeds);

template <int kKind, bool k32>
__device__ __forceinline__ uint64_t query_one(const QueryView& v, uint64_t key, const uint64_t* seeds) {
    return query_hashed<kKind, k32>(v, key_hash(key, v.kseed), seeds);
}

template <int kKind, bool k32>
__device__ __forceinline__ uint64_t query_hashed(const QueryView& v, uint64_t hk, const uint64_t* seeds) {
    constexpr bool kMono = kKind == kQMono, kNarrow = kKind == kQDict;
    uint64_t j, Tj;
    uint32_t m;
    if constexpr (k32) {
        const uint32_t j32 = fastrange32(hk, (uint32_t)v.NP);
        const uint32_t w = v.off_w;
        uint32_t d0 = 0, d1 = 0;
        if (w) {
            const uint32_t o = j32 * w, i = o >> 6, sh = o & 63;
            uint64_t x;
            if (kNarrow) {
                x = __ldg(v.off_words + i) >> sh;
                if (sh + 2 * w > 64) x |= __ldg(v.off_words + i + 1) << (64 - sh);  // sh > 0 here
            } else {
                const uint64_t lo = __ldg(v.off_words + i);
                x = sh ? (lo >> sh) | (__ldg(v.off_words + i + 1) << (64 - sh)) : lo;
            }
            const uint32_t mask = (1u << w) - 1;
            d0 = (uint32_t)x & mask;
            d1 = (uint32_t)(x >> w) & mask;
        }
        const uint32_t Qh = (uint32_t)(v.off_Q >> 32), Ql = (uint32_t)v.off_Q;
        const uint64_t e0 = (uint64_t)j32 * Qh + __umulhi(j32, Ql);
        const uint32_t e1 = (j32 + 1) * Qh + __umulhi(j32 + 1, Ql);  // low 32 bits of E(j + 1)
        Tj = e0 + (uint64_t)v.off_dmin + d0;
        m = e1 - (uint32_t)e0 + d1 - d0;
        j = j32;
    } else {
        j = partition_of(hk, v.NP);
        uint64_t Tj1;
        if (v.off_w <= 31) {
            offsets_of<kNarrow>(v, j, &Tj, &Tj1);
        } else {
            Tj = offset_of(v, j);
            Tj1 = offset_of(v, j + 1);
        }
        m = (uint32_t)(Tj1 - Tj);
    }
    if (m == 0) return 0;  // only a key outside the set can land in an empty partition
    const uint32_t b = bucket_of(bucket_hash(hk), v.table, v.B);
    uint32_t p;
    if (kMono) {
        p = mono_pilot(v, (uint64_t)b * v.NP + j);
    } else if (v.encoder == 2) {
        p = rice_pilot(v, b, j);
    } else if (v.encoder == 3) {
        p = ef_column_pilot(v, b, j);
    } else if (v.encoder == 4) {  // IC-CR: Compact below mix_c, Rice from there on
        if (b < v.mix_c) {
            const uint64_t meta = __ldg(v.col_meta + 2 * b);
            const uint32_t w = (uint32_t)(meta >> 56);
            p = (uint32_t)read_bits(v.pil_words, (meta & kMeta) + j * w, w);
        } else {
            p = rice_pilot(v, b, j);
        }
    } else if (k32 || v.small_bits) {
        const uint32_t jj = (uint32_t)j;
        if (v.encoder == 0) {
            const uint64_t meta = __ldg(v.col_meta + b);
            const uint32_t w = (uint32_t)(meta >> 56);
            p = read_bits32(v.pil_words, (uint32_t)meta + jj * w, w);
        } else {
            const uint64_t rm = __ldg(v.col_meta + 2 * b), dm = __ldg(v.col_meta + 2 * b + 1);
            const uint32_t rw = (uint32_t)(rm >> 56), dw = (uint32_t)(dm >> 56);
            uint32_t r;
            if (kNarrow) {
                r = read_bits32_narrow(v.pil_words, (uint32_t)rm + jj * rw, rw);
                p = read_bits32_narrow(v.dict_words, (uint32_t)dm + r * dw, dw);
            } else {
                r = read_bits32(v.pil_words, (uint32_t)rm + jj * rw, rw);
                p = read_bits32(v.dict_words, (uint32_t)dm + r * dw, dw);
            }
        }
    } else if (v.encoder == 0) {
        uint64_t meta = __ldg(v.col_meta + b);
        uint32_t w = (uint32_t)(meta >> 56);
        p = (uint32_t)read_bits(v.pil_words, (meta & kMeta) + j * w, w);
    } else {
        uint64_t rm = __ldg(v.col_meta + 2 * b), dm = __ldg(v.col_meta + 2 * b + 1);
        uint32_t rw = (uint32_t)(rm >> 56), dw = (uint32_t)(dm >> 56);
        uint64_t r = read_bits(v.pil_words, (rm & kMeta) + j * rw, rw);
        p = (uint32_t)read_bits(v.dict_words, (dm & kMeta) + r * dw, dw);
    }
    uint32_t local;
    if (v.pilot_mode == 0) {
        uint32_t s, d;
        if constexpr (k32) {
            s = div_small(p, m, d);
        } else {
            s = div_u32(p, m);
            d = p - s * m;
        }
        const uint64_t ps = s < kSeedTable ? seeds[s] : pilot_seed(s);
        local = position_hash(hk, ps, m) + d;
        if (local >= m) local -= m;
    } else {
        const uint64_t ps = p < kSeedTable ? seeds[p] : pilot_seed(p);
        local = position_hash(hk, ps, m);
    }
    uint64_t g = Tj + local;
    if (g >= v.n) g = ef_access(v, g - v.n);
    return g;
}

template <int kKind, bool k32>
__global__ void __launch_bounds__(256) k_query(const QueryView v, const uint64_t* __restrict__ keys,
                                               uint64_t* __restrict__ out, uint64_t m) {
    __shared__ uint64_t seeds[kSeedTable];
    if (threadIdx.x < kSeedTable) seeds[threadIdx.x] = pilot_seed(threadIdx.x);
    __syncthreads();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const bool vec = ((reinterpret_cast<uintptr_t>(keys) | reinterpret_cast<uintptr_t>(out)) & 15) == 0;
    if (vec) {
        const uint64_t pairs = m >> 1;
        const ulonglong2* k2 = reinterpret_cast<const ulonglong2*>(keys);
        ulonglong2* o2 = reinterpret_cast<ulonglong2*>(out);
        for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < pairs; i += stride) {
            ulonglong2 k = __ldcs(k2 + i);
            ulonglong2 r;
            r.x = query_one<kKind, k32>(v, k.x, seeds);
            r.y = query_one<kKind, k32>(v, k.y, seeds);
            __stcs(o2 + i, r);
        }
        if ((m & 1) && blockIdx.x == 0 && threadIdx.x == 0) out[m - 1] = query_one<kKind, k32>(v, keys[m - 1], seeds);
    } else {
        for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += stride)
            out[i] = query_one<kKind, k32>(v, keys[i], seeds);
    }
}

// string keys: XXH64 master hash of each string (Section 5), then the same query
template <int kKind, bool k32>
__global__ void __launch_bounds__(256) k_query_strings(const QueryView v, const uint8_t* __restrict__ bytes,
                                                       const uint64_t* __restrict__ offsets, uint64_t* __restrict__ out,
                                                       uint64_t m) {
    __shared__ uint64_t seeds[kSeedTable];
    if (threadIdx.x < kSeedTable) seeds[threadIdx.x] = pilot_seed(threadIdx.x);
    __syncthreads();
    const uint64_t total = __ldg(offsets + m);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = query_hashed<kKind, k32>(v, string_master_hash(bytes, offsets, total, i, v.string_seed), seeds);
}

// Several query batches against different structures in one launch.  The
// batches are concatenated into one index space: request r covers indexes
// [reqs[r].begin, reqs[r + 1].begin).  A block takes chunks of kChunk
// consecutive indexes; thread 0 finds the request of the chunk's first index by
// binary search and every thread advances from there (a chunk rarely spans more
// than two requests).  Loads and stores stay coalesced inside each request.
constexpr uint32_t kChunk = 1024;

__global__ void __launch_bounds__(256) k_query_multi(const MultiQuery* __restrict__ reqs, uint32_t nreq,
                                                     uint64_t total) {
    __shared__ uint64_t seeds[kSeedTable];
    __shared__ uint32_t r_first[2];
    if (threadIdx.x < kSeedTable) seeds[threadIdx.x] = pilot_seed(threadIdx.x);
    uint32_t bank = 0;
    for (uint64_t c0 = blockIdx.x * (uint64_t)kChunk; c0 < total; c0 += (uint64_t)gridDim.x * kChunk) {
        if (threadIdx.x == 0) {
            uint32_t lo = 0, hi = nreq;  // largest r with begin <= c0
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (reqs[mid].begin <= c0) lo = mid; else hi = mid;
            }
            r_first[bank] = lo;
        }
        __syncthreads();  // (two banks: the next chunk's write never meets this chunk's reads)
        uint32_t r = r_first[bank];
        bank ^= 1;
        for (uint32_t k = 0; k < kChunk / 256; k++) {
            const uint64_t i = c0 + k * 256 + threadIdx.x;
            if (i >= total) break;
            while (r + 1 < nreq && reqs[r + 1].begin <= i) r++;
            const MultiQuery* q = reqs + r;
            const uint64_t x = __ldcs(q->keys + (i - q->begin));
            // a handle's encoder is uniform over its request
            const uint32_t enc = q->v.encoder;
            const uint64_t y = enc >= 5   ? query_one<kQMono, false>(q->v, x, seeds)
                               : enc == 1 ? query_one<kQDict, false>(q->v, x, seeds)
                                          : query_one<kQInterleaved, false>(q->v, x, seeds);
            __stcs(q->out + (i - q->begin), y);
        }
    }
}

}  // namespace

cudaError_t launch_query_multi(const MultiQuery* d_reqs, uint32_t nreq, uint64_t total, cudaStream_t stream) {
    if (total == 0 || nreq == 0) return cudaSuccess;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint64_t want = (total + kChunk - 1) / kChunk;
    uint64_t cap = (uint64_t)sms * 8;
    unsigned grid = (unsigned)(want < cap ? want : cap);
    k_query_multi<<<grid, 256, 0, stream>>>(d_reqs, nreq, total);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_query_strings(const QueryView& v, const uint8_t* bytes, const uint64_t* offsets, uint64_t* out,
                                 uint64_t m, cudaStream_t stream) {
    if (m == 0) return cudaSuccess;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint64_t want = (m + 255) / 256;
    uint64_t cap = (uint64_t)sms * 8;
    unsigned grid = (unsigned)(want < cap ? (want ? want : 1) : cap);
    const bool f32 = query_fast32(v);
    switch (query_kind(v)) {
        case kQMono: k_query_strings<kQMono, false><<<grid, 256, 0, stream>>>(v, bytes, offsets, out, m); break;
        case kQDict:
            if (f32)
                k_query_strings<kQDict, true><<<grid, 256, 0, stream>>>(v, bytes, offsets, out, m);
            else
                k_query_strings<kQDict, false><<<grid, 256, 0, stream>>>(v, bytes, offsets, out, m);
            break;
        default:
            if (f32)
                k_query_strings<kQInterleaved, true><<<grid, 256, 0, stream>>>(v, bytes, offsets, out, m);
            else
                k_query_strings<kQInterleaved, false><<<grid, 256, 0, stream>>>(v, bytes, offsets, out, m);
            break;
    }
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_query(const QueryView& v, const uint64_t* keys, uint64_t* out, uint64_t m, cudaStream_t stream) {
    if (m == 0) return cudaSuccess;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint64_t want = (m / 2 + 255) / 256;
    uint64_t cap = (uint64_t)sms * 8;  // 8 resident blocks of 256 threads per SM
    unsigned grid = (unsigned)(want < cap ? (want ? want : 1) : cap);
    const bool f32 = query_fast32(v);
    switch (query_kind(v)) {
        case kQMono: k_query<kQMono, false><<<grid, 256, 0, stream>>>(v, keys, out, m); break;
        case kQDict:
            if (f32)
                k_query<kQDict, true><<<grid, 256, 0, stream>>>(v, keys, out, m);
            else
                k_query<kQDict, false><<<grid, 256, 0, stream>>>(v, keys, out, m);
            break;
        default:
            if (f32)
                k_query<kQInterleaved, true><<<grid, 256, 0, stream>>>(v, keys, out, m);
            else
                k_query<kQInterleaved, false><<<grid, 256, 0, stream>>>(v, keys, out, m);
            break;
    }
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace phobic
