// Device-side building blocks shared by the libphobic kernels.
//
// The hash functions restate this library's fixed spec for the quantities the
// paper leaves open: the master hash (Section 5 names xxHash; 64-bit keys use a
// bijective finaliser), the bucket hash, and the pilot hash h(x, s) of Section 4
// ("Hash Function").
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace phobic {

// spec constants
constexpr uint64_t kSeedMix = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kBucketMix = 0x5851F42D4C957F2Dull;
constexpr uint64_t kPilotMix = 0x2545F4914F6CDD1Dull;
constexpr int kTablePoints = 2048;   // Appendix C: gamma tabulated at 2048 points
constexpr uint32_t kMaxBucket = 1023; // larger buckets are rejected as unplaceable
constexpr uint32_t kMaxPartitionSize = 16384;

// status codes written by kernels into a device status word (priority order:
// a larger code wins when several partitions fail)
constexpr uint32_t kDevOk = 0;
constexpr uint32_t kDevTimeout = 1;
constexpr uint32_t kDevSearchLimit = 2;
constexpr uint32_t kDevDupHash = 3;

// SplitMix64 output function (Steele, Lea, Flood 2014), a 64-bit bijection.
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// floor(a * b / 2^64)
__device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b) { return __umul64hi(a, b); }

// floor(h * m / 2^64) for m < 2^32: fastrange onto [0, m).  With h = hi 2^32 +
// lo, h m / 2^32 = hi m + lo m / 2^32, and the fraction of lo m / 2^32 cannot
// carry into bit 32 of the integer part, so the result is bits 32..63 of
// hi m + floor(lo m / 2^32) (which stays below 2^64): one wide multiply-add and
// one high multiply, where a general 64 x 64 high product needs several.
__device__ __forceinline__ uint32_t fastrange32(uint64_t h, uint32_t m) {
    const uint64_t t = (uint64_t)(uint32_t)(h >> 32) * m + __umulhi((uint32_t)h, m);
    return (uint32_t)(t >> 32);
}

__host__ __device__ __forceinline__ uint64_t key_seed(uint64_t seed) { return mix64(seed ^ kSeedMix); }
__host__ __device__ __forceinline__ uint64_t key_hash(uint64_t key, uint64_t kseed) { return mix64(key ^ kseed); }
__device__ __forceinline__ uint64_t bucket_hash(uint64_t hk) { return mix64(hk ^ kBucketMix); }
__device__ __forceinline__ uint64_t pilot_seed(uint64_t s) { return mix64(s ^ kPilotMix); }
__device__ __forceinline__ uint32_t position_hash(uint64_t hk, uint64_t ps, uint32_t m) {
    return fastrange32(mix64(hk ^ ps), m);
}

// partition of a master hash, floor(hk N_P / 2^64)
__device__ __forceinline__ uint64_t partition_of(uint64_t hk, uint64_t np) { return mulhi64(hk, np); }

// Bits 32..95 of the 128-bit product j Q, mod 2^64: the offsets' expectation
// floor(j Q / 2^32) (Section 4 stores offsets as differences to it)
__device__ __forceinline__ uint64_t offset_expectation(uint64_t j, uint64_t Q) {
    return (__umul64hi(j, Q) << 32) | ((j * Q) >> 32);
}

// Section 3.1 / Appendix C: bucket of normalised hash x from the fixed-point
// table of gamma T_0..T_2048, by linear interpolation between T_k and T_{k+1}:
// v = T_k + ((T_{k+1} - T_k) f >> 32), bucket = min(B - 1, v B >> 32).
// The device holds the table packed, one word per interval (pack_bucket_table):
// low half min(T_k, 2^32 - 1), high half T_{k+1} - T_k (below 2^32), so that a
// lookup is one read.  The clamp changes no bucket: T_k = 2^32 gives v >= 2^32,
// hence B - 1, and the clamped v >= 2^32 - 1 gives B - 1 too.
__device__ __forceinline__ uint32_t bucket_of(uint64_t x, const uint64_t* __restrict__ qtable, uint32_t B) {
    const uint64_t e = __ldg(qtable + (x >> 53));
    const uint64_t v = (e & 0xFFFFFFFFull) + __umulhi((uint32_t)(e >> 32), (uint32_t)(x >> 21));
    if (v >> 32) return B - 1;
    const uint32_t b = __umulhi((uint32_t)v, B);
    return b > B - 1 ? B - 1 : b;
}

// T_0..T_2048 (kTablePoints + 1 words) -> the packed device form (kTablePoints words)
__host__ __forceinline__ void pack_bucket_table(const uint64_t* t, uint64_t* q) {
    for (int k = 0; k < kTablePoints; k++) {
        const uint64_t lo = t[k] < 0xFFFFFFFFull ? t[k] : 0xFFFFFFFFull;
        q[k] = lo | ((uint64_t)(uint32_t)(t[k + 1] - t[k]) << 32);
    }
}

// number of bits of v (0 for 0)
__host__ __device__ __forceinline__ uint32_t bitlen64(uint64_t v) {
#ifdef __CUDA_ARCH__
    return 64 - __clzll((long long)v);
#else
    return v ? 64 - __builtin_clzll(v) : 0;
#endif
}

// Read `w` (<= 64) bits at bit offset `o` of little-endian packed words.  The
// packed arrays carry one zero word of padding so that reading words o/64 and
// o/64+1 never leaves the buffer.
__device__ __forceinline__ uint64_t read_bits(const uint64_t* __restrict__ words, uint64_t o, uint32_t w) {
    if (w == 0) return 0;
    uint64_t i = o >> 6;
    uint32_t sh = (uint32_t)(o & 63);
    uint64_t lo = __ldg(words + i);
    uint64_t v = lo >> sh;
    if (sh + w > 64) v |= __ldg(words + i + 1) << (64 - sh);
    return w == 64 ? v : (v & ((1ull << w) - 1));
}

// Read w <= 32 bits at bit offset o (o < 2^32 bits into the array) through the
// 32-bit view of the little-endian packed words: one funnel shift of two
// adjacent 32-bit words (the padding word keeps the second read in bounds).
__device__ __forceinline__ uint32_t read_bits32(const uint64_t* __restrict__ words, uint32_t o, uint32_t w) {
    const uint32_t* w32 = reinterpret_cast<const uint32_t*>(words);
    const uint32_t i = o >> 5;
    const uint32_t x = __funnelshift_r(__ldg(w32 + i), __ldg(w32 + i + 1), o & 31);
    return w >= 32 ? x : (x & ((1u << w) - 1));
}

// words needed for `nbits` bits, including one padding word
__host__ __device__ __forceinline__ uint64_t packed_words(uint64_t nbits) { return (nbits + 63) / 64 + 1; }

// Per-structure view passed by value to the query kernel.
struct QueryView {
    uint64_t n, M, NP;
    uint32_t B;
    uint32_t encoder;    // 0 IC-C, 1 IC-D, 2 IC-R, 3 IC-EF, 4 IC-CR; 5..8 mono-C/D/R/EF (one column)
    uint32_t pilot_mode; // 0 additive, 1 xor
    uint32_t off_w;
    uint64_t kseed;      // mix64(seed ^ kSeedMix)
    uint64_t off_Q;
    int64_t off_dmin;
    const uint64_t* table;     // the packed bucket table (kTablePoints words, bucket_of)
    const uint64_t* off_words; // offsets, packed
    // IC-C: col_meta[b] = base | (width << 56); IC-D: col_meta[2b] = rank base | (rank width << 56),
    // col_meta[2b+1] = dict base | (dict width << 56)
    const uint64_t* col_meta;
    const uint64_t* pil_words;  // IC-C data, or IC-D ranks
    const uint64_t* dict_words; // IC-D dictionary
    // Elias-Fano remap of slots >= n
    uint64_t ef_N;
    uint32_t ef_l;
    const uint64_t* ef_low;
    const uint64_t* ef_high;
    const uint64_t* ef_samples;
    // IC-R: col_meta[2b] = low-part base | (Rice parameter << 56), col_meta[2b+1] =
    // unary base; pil_words = low parts; dict_words = the columns' select
    // samples (u32, rice_ns per column), followed by the unary bits at rice_high
    const uint64_t* rice_high;
    uint32_t rice_ns;
    uint32_t mix_c;       // IC-CR: columns below mix_c are Compact (sample column of b >= mix_c: b - mix_c)
    uint32_t small_bits;  // 1: every packed array has < 2^32 bits (32-bit offsets)
    uint32_t key_kind;    // 0: 64-bit keys, 1: byte strings (XXH64 with string_seed)
    uint64_t string_seed;
};


}  // namespace phobic
