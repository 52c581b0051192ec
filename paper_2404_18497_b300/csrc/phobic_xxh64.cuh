// XXH64 (Collet, "xxHash fast digest algorithm", XXH64), restated from its
// published specification: the 64-bit master hash of byte-string keys
// (Section 5 names xxHash).  Header-only so the hash and query kernels inline it.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace phobic {
namespace xxh {

constexpr uint64_t P1 = 0x9E3779B185EBCA87ull;
constexpr uint64_t P2 = 0xC2B2AE3D27D4EB4Full;
constexpr uint64_t P3 = 0x165667B19E3779F9ull;
constexpr uint64_t P4 = 0x85EBCA77C2B2AE63ull;
constexpr uint64_t P5 = 0x27D4EB2F165667C5ull;

__device__ __forceinline__ uint64_t rotl(uint64_t v, int r) { return (v << r) | (v >> (64 - r)); }

// Little-endian loads of 8 / 4 bytes at byte address p, where [base, end) is
// the readable buffer: two aligned 8-byte reads and a funnel shift when both
// aligned words lie inside the buffer, else byte by byte.
struct ByteSrc {
    const uint8_t* base;
    const uint8_t* end;
};
__device__ __forceinline__ uint64_t le64(const ByteSrc& b, const uint8_t* p) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    const uintptr_t a0 = a & ~uintptr_t(7);
    if (a0 >= reinterpret_cast<uintptr_t>(b.base) && a0 + 16 <= reinterpret_cast<uintptr_t>(b.end)) {
        const uint64_t* q = reinterpret_cast<const uint64_t*>(a0);
        const uint64_t lo = __ldg(q), hi = __ldg(q + 1);
        const uint32_t sh = (uint32_t)(a & 7) * 8;
        return sh ? (lo >> sh) | (hi << (64 - sh)) : lo;
    }
    uint64_t v = 0;
#pragma unroll
    for (int i = 7; i >= 0; i--) v = (v << 8) | __ldg(p + i);
    return v;
}

__device__ __forceinline__ uint64_t xround(uint64_t acc, uint64_t lane) { return rotl(acc + lane * P2, 31) * P1; }
__device__ __forceinline__ uint64_t xmerge(uint64_t acc, uint64_t v) { return (acc ^ xround(0, v)) * P1 + P4; }

__device__ __forceinline__ uint64_t xxh64(const ByteSrc& src, const uint8_t* p, uint64_t len, uint64_t seed) {
    uint64_t i = 0, acc;
    if (len >= 32) {
        uint64_t v1 = seed + P1 + P2, v2 = seed + P2, v3 = seed, v4 = seed - P1;
        for (; i + 32 <= len; i += 32) {
            v1 = xround(v1, le64(src, p + i));
            v2 = xround(v2, le64(src, p + i + 8));
            v3 = xround(v3, le64(src, p + i + 16));
            v4 = xround(v4, le64(src, p + i + 24));
        }
        acc = rotl(v1, 1) + rotl(v2, 7) + rotl(v3, 12) + rotl(v4, 18);
        acc = xmerge(acc, v1);
        acc = xmerge(acc, v2);
        acc = xmerge(acc, v3);
        acc = xmerge(acc, v4);
    } else {
        acc = seed + P5;
    }
    acc += len;
    for (; i + 8 <= len; i += 8) acc = rotl(acc ^ xround(0, le64(src, p + i)), 27) * P1 + P4;
    if (i + 4 <= len) {
        uint64_t v = 0;
#pragma unroll
        for (int t = 3; t >= 0; t--) v = (v << 8) | __ldg(p + i + t);
        acc = rotl(acc ^ (v * P1), 23) * P2 + P3;
        i += 4;
    }
    for (; i < len; i++) acc = rotl(acc ^ ((uint64_t)__ldg(p + i) * P5), 11) * P1;
    acc ^= acc >> 33;
    acc *= P2;
    acc ^= acc >> 29;
    acc *= P3;
    acc ^= acc >> 32;
    return acc;
}

}  // namespace xxh

// master hash of string i of (bytes, offsets); total = offsets[n] (readable bytes)
__device__ __forceinline__ uint64_t string_master_hash(const uint8_t* bytes, const uint64_t* offsets, uint64_t total,
                                                       uint64_t i, uint64_t seed) {
    const xxh::ByteSrc src{bytes, bytes + total};
    const uint64_t a = __ldg(offsets + i), b = __ldg(offsets + i + 1);
    return xxh::xxh64(src, bytes + a, b - a, seed);
}

}  // namespace phobic
