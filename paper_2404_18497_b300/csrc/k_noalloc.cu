// phobic_partition_sort_noalloc: the partition sort with its scratch memory in
// a fixed, file-scope device array instead of memory allocated per call.
//
// Who needs it: callers that may not allocate device memory while they run.
// Examples: a process whose memory budget is fully reserved up front, where
// an extra cudaMalloc can fail or evict something else; and host frameworks
// that own every device allocation and forbid libraries from calling the CUDA
// allocator behind their back.  Those callers still pass their own input and
// output buffers; only the sort's temporary space (ping-pong keys, digit
// histograms, look-back tile states, counters) comes from here.
//
// The paper has no counterpart; this is a deployment convenience.
#include <mutex>

#include "../../include/phobic.h"
#include "phobic_dev.cuh"
#include "phobic_kernels.cuh"

namespace {

constexpr size_t kErrorBytes = 256;
// the sort's scratch for PHOBIC_NOALLOC_MAX_KEYS keys at the widest digit
// (512 bins) and up to three passes (ping-pong keys, digit histograms,
// look-back tile states with two rows of padding and up to 256 bytes of
// alignment, tile counters), plus one error word; the same layout as
// sort_scratch_bytes, which each call checks against this size
constexpr size_t kMaxTiles = (PHOBIC_NOALLOC_MAX_KEYS + phobic::kSortTileKeys - 1) / phobic::kSortTileKeys;
constexpr size_t kSortBytes =
    (size_t)PHOBIC_NOALLOC_MAX_KEYS * 8 + 3 * 512 * 8 + 64 + 256 + (kMaxTiles + 2) * 512 * 8 + 64 + 256 + 64;
constexpr size_t kScratchBytes = (kSortBytes + 255) / 256 * 256 + kErrorBytes;

// Held by every GPU that loads this library, until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_addr[kMaxDevices] = {};

// Device address of the array on the current device (looked up once per
// device, with that device current).  Host code must not pass the symbol
// itself: on the host it is only a stand-in, not a device address.
cudaError_t scratch_address(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" phobic_status phobic_partition_sort_noalloc(const uint64_t* d_hk, uint64_t n, uint64_t num_partitions,
                                                       uint64_t* d_sorted, uint64_t* d_start,
                                                       phobic_stream_t stream) {
    if (n == 0 || num_partitions == 0 || !d_hk || !d_sorted || !d_start) return PHOBIC_ERR_INVALID_ARG;
    if (n > PHOBIC_NOALLOC_MAX_KEYS) return PHOBIC_ERR_INVALID_ARG;
    const size_t need = phobic::sort_scratch_bytes(n, num_partitions);
    if (need + kErrorBytes > kScratchBytes) return PHOBIC_ERR_INVALID_ARG;
    unsigned char* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return PHOBIC_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t* err = reinterpret_cast<uint32_t*>(base + kScratchBytes - kErrorBytes);
    // the array keeps the previous call's contents: the error word starts at
    // zero here, and the sort clears its own histograms, counters and tile states
    e = cudaMemsetAsync(err, 0, sizeof(uint32_t), st);
    if (e == cudaSuccess)
        e = phobic::launch_partition_sort(d_hk, 0, 0, n, num_partitions, d_sorted, d_start, base, err, st);
    uint32_t herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? PHOBIC_ERR_OOM : PHOBIC_ERR_CUDA;
    return herr ? PHOBIC_ERR_TIMEOUT : PHOBIC_OK;
}
