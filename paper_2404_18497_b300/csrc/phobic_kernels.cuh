// Launch wrappers of the libphobic kernels (internal; the public ABI is phobic.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "phobic_dev.cuh"

namespace phobic {

// process-wide count of kernel launches (diagnostic)
void note_launches(uint64_t k);

// ---- k_sort.cu: master hash + onesweep sort by partition id ----
constexpr uint32_t kSortTileKeys = 4096;  // keys per onesweep tile
void sort_plan(uint64_t np, uint32_t* passes, uint32_t* bits);
size_t sort_scratch_bytes(uint64_t n, uint64_t np);
cudaError_t launch_partition_sort(const uint64_t* in, int hash_input, uint64_t kseed, uint64_t n, uint64_t np,
                                  uint64_t* sorted, uint64_t* start, void* scratch, uint32_t* d_error,
                                  cudaStream_t stream);
cudaError_t launch_hash_u64(const uint64_t* keys, uint64_t n, uint64_t kseed, uint64_t* out, cudaStream_t stream);
cudaError_t launch_hash_strings(const uint8_t* bytes, const uint64_t* offsets, uint64_t n, uint64_t seed,
                                uint64_t* out, cudaStream_t stream);

// ---- k_scan.cu: exclusive scan of u32 counts into u64 offsets ----
constexpr uint32_t kScanTileItems = 4096;
uint64_t scan_num_tiles(uint64_t n);
size_t scan_tiles_bytes(uint64_t n);
const unsigned long long* scan_total(const unsigned long long* tiles, uint64_t n);
cudaError_t exclusive_scan_u32(const uint32_t* in, uint64_t n, unsigned long long* out, unsigned long long* tiles,
                               cudaStream_t st);

// ---- k_search.cu: partition sizes, table sizes, offsets T; bucketing + pilot search ----
// T[0..np] = exclusive scan of m_j with T[np] = M; stats[0] = M, stats[1] = max n_j, stats[2] = max m_j
size_t sizes_scratch_bytes(uint64_t np);
cudaError_t launch_sizes(const uint64_t* start, uint64_t np, double alpha, uint64_t* T, uint64_t* stats,
                         void* scratch, cudaStream_t stream);

struct SearchLaunch {
    const uint64_t* sorted;
    const uint64_t* start;
    const uint64_t* T;
    const uint64_t* table;
    uint64_t np;
    uint32_t B;
    uint32_t mode;
    uint32_t s_max;
    uint32_t cap_n; // largest n_j
    uint32_t cap_m; // largest m_j
    uint64_t* bkeys;       // [n] scratch for the bucket-sorted keys (used unless keys_in_smem)
    uint32_t keys_in_smem; // 1: keep each partition's keys in shared memory
    uint32_t window_bits;  // displacements per lane-window: 32 or 64 (speed only)
    uint32_t* pilots;      // [B x np], zero-filled by the caller
    uint32_t* taken_bits;  // global occupancy bitmap over [0, M) in u32 words, zero-filled; may be null
    uint32_t* status;      // device status word (kDev* codes, atomicMax)
    unsigned long long* work; // [2]: s tries, window steps (may be null)
};
size_t search_smem_bytes(uint32_t cap_n, uint32_t cap_m, uint32_t B, bool keys_in_smem);
size_t search_smem_limit();
cudaError_t launch_search(const SearchLaunch& a, cudaStream_t stream);

// ---- k_encode.cu ----
// offsets: D_j = T_j - floor(j Q / 2^32); mm[0] = min D (as int64 bits), mm[1] = max D
cudaError_t launch_offset_minmax(const uint64_t* T, uint64_t np, uint64_t Q, long long* mm, cudaStream_t stream);
cudaError_t launch_offset_pack(const uint64_t* T, uint64_t np, uint64_t Q, int64_t dmin, uint32_t w,
                               uint64_t* words, uint64_t nwords, cudaStream_t stream);
// per column max pilot: colmax[b]
cudaError_t launch_column_max(const uint32_t* pilots, uint64_t np, uint32_t B, uint32_t* colmax, cudaStream_t stream);
// IC-C: col_meta[b] = base | width << 56 (device copy made by the caller)
cudaError_t launch_compact_pack(const uint32_t* pilots, uint64_t np, uint32_t B, const uint64_t* col_meta,
                                const uint64_t* col_word_begin, uint64_t* words, uint64_t nwords,
                                cudaStream_t stream);
// IC-D, step 1: presence bitmaps of the pilot values of each column
cudaError_t launch_dict_mark(const uint32_t* pilots, uint64_t np, uint32_t B, const uint64_t* bm_base,
                             uint64_t* bitmaps, cudaStream_t stream);
// IC-D, step 2: per column, popcount prefix of its bitmap words -> rank base per word, and distinct count K_b
cudaError_t launch_dict_rank(const uint64_t* bm_base, uint32_t B, uint64_t* bitmaps_rank, const uint64_t* bitmaps,
                             uint64_t* K, cudaStream_t stream);
// IC-D, step 3: pack ranks and dictionaries
cudaError_t launch_dict_pack(const uint32_t* pilots, uint64_t np, uint32_t B, const uint64_t* bm_base,
                             const uint64_t* bitmaps, const uint64_t* bitmaps_rank, const uint64_t* col_meta,
                             const uint64_t* rank_word_begin, uint64_t* rank_words, uint64_t rank_nwords,
                             const uint64_t* dict_word_begin, uint64_t* dict_words, uint64_t dict_nwords,
                             cudaStream_t stream);

// ---- k_remap.cu: Elias-Fano remap of slots >= n (alpha < 1) ----
size_t remap_scratch_bytes(uint64_t n, uint64_t M);
cudaError_t launch_remap(const uint32_t* taken_bits, uint64_t n, uint64_t M, uint32_t l, uint64_t* fs,
                         uint64_t* ef_low, uint64_t low_nwords, uint64_t* ef_high, uint64_t high_nwords,
                         uint64_t* ef_samples, void* scratch, cudaStream_t stream);

// ---- k_query.cu ----
cudaError_t launch_query(const QueryView& v, const uint64_t* keys, uint64_t* out, uint64_t m, cudaStream_t stream);
cudaError_t launch_query_strings(const QueryView& v, const uint8_t* bytes, const uint64_t* offsets, uint64_t* out,
                                 uint64_t m, cudaStream_t stream);

}  // namespace phobic
