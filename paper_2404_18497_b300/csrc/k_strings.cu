// K1 for string keys: 64-bit master hashes (XXH64, phobic_xxh64.cuh) of
// variable-length byte strings, one thread per string.
#include "phobic_dev.cuh"
#include "phobic_kernels.cuh"
#include "phobic_xxh64.cuh"

namespace phobic {

namespace {

__global__ void k_hash_strings(const uint8_t* __restrict__ bytes, const uint64_t* __restrict__ offsets, uint64_t n,
                               uint64_t seed, uint64_t* __restrict__ out) {
    const uint64_t total = __ldg(offsets + n);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = string_master_hash(bytes, offsets, total, i, seed);
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
