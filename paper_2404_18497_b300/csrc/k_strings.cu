// K1 for string keys: 64-bit master hashes of variable-length byte strings.
//
// Section 5: keys are first reduced to master hash codes with xxHash.  This is
// XXH64 restated from its published specification (Collet, "xxHash
// fast digest algorithm", XXH64), one thread per string.
#include "phobic_dev.cuh"
#include "phobic_kernels.cuh"

namespace phobic {

namespace {

constexpr uint64_t P1 = 0x9E3779B185EBCA87ull;
constexpr uint64_t P2 = 0xC2B2AE3D27D4EB4Full;
constexpr uint64_t P3 = 0x165667B19E3779F9ull;
constexpr uint64_t P4 = 0x85EBCA77C2B2AE63ull;
constexpr uint64_t P5 = 0x27D4EB2F165667C5ull;

__device__ __forceinline__ uint64_t rotl(uint64_t v, int r) { return (v << r) | (v >> (64 - r)); }

// little-endian loads from an arbitrary byte address
__device__ __forceinline__ uint64_t le64(const uint8_t* p) {
    uint64_t v = 0;
#pragma unroll
    for (int i = 7; i >= 0; i--) v = (v << 8) | __ldg(p + i);
    return v;
}
__device__ __forceinline__ uint64_t le32(const uint8_t* p) {
    uint64_t v = 0;
#pragma unroll
    for (int i = 3; i >= 0; i--) v = (v << 8) | __ldg(p + i);
    return v;
}

__device__ __forceinline__ uint64_t xround(uint64_t acc, uint64_t lane) { return rotl(acc + lane * P2, 31) * P1; }
__device__ __forceinline__ uint64_t xmerge(uint64_t acc, uint64_t v) { return (acc ^ xround(0, v)) * P1 + P4; }

__device__ uint64_t xxh64(const uint8_t* p, uint64_t len, uint64_t seed) {
    uint64_t i = 0, acc;
    if (len >= 32) {
        uint64_t v1 = seed + P1 + P2, v2 = seed + P2, v3 = seed, v4 = seed - P1;
        for (; i + 32 <= len; i += 32) {
            v1 = xround(v1, le64(p + i));
            v2 = xround(v2, le64(p + i + 8));
            v3 = xround(v3, le64(p + i + 16));
            v4 = xround(v4, le64(p + i + 24));
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
    for (; i + 8 <= len; i += 8) acc = rotl(acc ^ xround(0, le64(p + i)), 27) * P1 + P4;
    if (i + 4 <= len) {
        acc = rotl(acc ^ (le32(p + i) * P1), 23) * P2 + P3;
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

__global__ void k_hash_strings(const uint8_t* __restrict__ bytes, const uint64_t* __restrict__ offsets, uint64_t n,
                               uint64_t seed, uint64_t* __restrict__ out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t a = __ldg(offsets + i), b = __ldg(offsets + i + 1);
        out[i] = xxh64(bytes + a, b - a, seed);
    }
}

}  // namespace

cudaError_t launch_hash_strings(const uint8_t* bytes, const uint64_t* offsets, uint64_t n, uint64_t seed,
                                uint64_t* out, cudaStream_t stream) {
    if (n == 0) return cudaSuccess;
    uint64_t blocks = (n + 255) / 256;
    if (blocks > 16384) blocks = 16384;
    k_hash_strings<<<(unsigned)blocks, 256, 0, stream>>>(bytes, offsets, n, seed, out);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace phobic
