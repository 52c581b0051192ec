// Exclusive scan of u32 counts into u64 offsets, three phases: per-tile
// sums, one block scanning the tile sums, then per-tile scans plus the tile's
// offset.  The grand total lands in tiles[ntiles] (see scan_total).
#include <mutex>
#include <set>

#include "phobic_dev.cuh"
#include "phobic_kernels.cuh"

namespace phobic {

cudaError_t allow_max_dynamic_smem(const void* kern) {
    static std::mutex mu;
    static std::set<std::pair<int, const void*>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({dev, kern})) return cudaSuccess;
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess) done.insert({dev, kern});
    return e;
}

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;
static_assert(kScanTile == (int)kScanTileItems, "scan tile");

__device__ __forceinline__ unsigned long long block_scan_excl(unsigned long long v, unsigned long long* total) {
    __shared__ unsigned long long ws[32];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= (uint32_t)o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned long long s = ws[lane], z = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, z, o);
            if (lane >= (uint32_t)o) z += y;
        }
        ws[lane] = z - s;
        if (lane == 31) *total = z;
    }
    __syncthreads();
    unsigned long long r = ws[warp] + x - v;
    __syncthreads();
    return r;
}

// phase 1: per-tile sums
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const uint32_t* __restrict__ in, uint64_t n,
                                                             unsigned long long* __restrict__ tile_sum) {
    __shared__ unsigned long long tot;
    uint64_t base = (uint64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    unsigned long long s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++)
        if (base + i < n) s += in[base + i];
    block_scan_excl(s, &tot);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

// phase 2: exclusive scan of the tile sums (one block); grand total at [ntiles]
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(unsigned long long* __restrict__ tile_sum, uint64_t ntiles) {
    __shared__ unsigned long long tot;
    unsigned long long carry = 0;
    for (uint64_t c = 0; c < ntiles; c += kScanThreads) {
        uint64_t i = c + threadIdx.x;
        unsigned long long v = i < ntiles ? tile_sum[i] : 0;
        unsigned long long e = block_scan_excl(v, &tot);
        if (i < ntiles) tile_sum[i] = carry + e;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) tile_sum[ntiles] = carry;
}

// phase 3: exclusive scan within tiles plus the tile offset
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const uint32_t* __restrict__ in, uint64_t n,
                                                             const unsigned long long* __restrict__ tile_sum,
                                                             unsigned long long* __restrict__ out) {
    __shared__ unsigned long long tot;
    uint64_t base = (uint64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    unsigned long long s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        v[i] = base + i < n ? in[base + i] : 0;
        s += v[i];
    }
    unsigned long long run = tile_sum[blockIdx.x] + block_scan_excl(s, &tot);
#pragma unroll
    for (int i = 0; i < kScanItems; i++)
        if (base + i < n) {
            out[base + i] = run;
            run += v[i];
        }
}

}  // namespace

uint64_t scan_num_tiles(uint64_t n) {
    uint64_t nt = (n + kScanTile - 1) / kScanTile;
    return nt ? nt : 1;
}

size_t scan_tiles_bytes(uint64_t n) { return (scan_num_tiles(n) + 2) * 8; }

const unsigned long long* scan_total(const unsigned long long* tiles, uint64_t n) { return tiles + scan_num_tiles(n); }

cudaError_t exclusive_scan_u32(const uint32_t* in, uint64_t n, unsigned long long* out, unsigned long long* tiles,
                               cudaStream_t st) {
    const uint64_t nt = scan_num_tiles(n);
    k_scan_tiles<<<(unsigned)nt, kScanThreads, 0, st>>>(in, n, tiles);
    note_launches(1);
    k_scan_sums<<<1, kScanThreads, 0, st>>>(tiles, nt);
    note_launches(1);
    k_scan_apply<<<(unsigned)nt, kScanThreads, 0, st>>>(in, n, tiles, out);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace phobic
