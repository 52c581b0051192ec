// Launch wrappers of the libphobic kernels (internal; the public ABI is phobic.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "phobic_dev.cuh"

namespace phobic {
// Lets `kern` launch with up to the device's opt-in maximum of dynamic shared
// memory.  Every caller sets the same value, so builds running in several host
// threads never lower the limit under one another's launch; the occupancy
// still follows each launch's own size.  Done once per kernel and device.
cudaError_t allow_max_dynamic_smem(const void* kern);


// process-wide count of kernel launches (diagnostic)
void note_launches(uint64_t k);

// ---- k_sort.cu: master hash + onesweep sort by partition id ----
constexpr uint32_t kSortTileKeys = 6144;  // keys per onesweep tile (384 threads x 16)
// one independent key set of a (batched) sort: keys [key_base, key_base + n)
// grouped by partition j = floor(hk np / 2^64) into [key_base, key_base + n);
// partition starts go to start[part_base + j]; tiles [first_tile, ...)
struct SortSeg {
    uint64_t key_base, n, np, part_base, first_tile;
};
// Self-test of the look-back wait: tile mute_tile never publishes its state,
// so the wait of its successor runs out after spin_limit polls.
struct SortWaitTest {
    uint64_t mute_tile;
    uint32_t spin_limit;
};
void sort_plan(uint64_t np, uint32_t* passes, uint32_t* bits);
uint64_t sort_tiles(uint64_t n);
size_t sort_seg_scratch_bytes(uint64_t n_total, uint64_t tiles, uint32_t nseg, uint64_t max_np);
size_t sort_scratch_bytes(uint64_t n, uint64_t np);
cudaError_t launch_partition_sort_segs(const uint64_t* in, int hash_input, uint64_t kseed, const SortSeg* d_segs,
                                       uint32_t nseg, uint64_t n_total, uint64_t tiles, uint64_t max_np,
                                       uint64_t total_parts, uint64_t* sorted, uint64_t* start, void* scratch,
                                       uint32_t* d_error, cudaStream_t stream,
                                       const SortWaitTest* wait_test = nullptr);
cudaError_t launch_partition_sort(const uint64_t* in, int hash_input, uint64_t kseed, uint64_t n, uint64_t np,
                                  uint64_t* sorted, uint64_t* start, void* scratch, uint32_t* d_error,
                                  cudaStream_t stream, const SortWaitTest* wait_test = nullptr);
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

// one key set of a search launch: its partitions are [part_base, part_base + np)
// in the global partition numbering; pilot of bucket b of local partition j at
// pilots[pilot_base + b * np + j]
struct SearchSet {
    uint64_t part_base, np, pilot_base;
    const uint64_t* table;  // packed bucket table of this set's (lambda, alpha, P) (bucket_of)
    uint32_t B, pad;
};

struct SearchLaunch {
    const uint64_t* sorted;  // master hashes grouped by global partition
    const uint64_t* start;   // [total_parts + 1]
    const uint64_t* T;       // [total_parts + 1] slot offsets (global over all sets)
    const SearchSet* sets;
    uint32_t nsets;
    uint64_t total_parts;
    uint32_t cap_B;        // largest B over the sets
    uint32_t mode;
    uint32_t s_max;        // requested seed limit (0xFFFFFFFF: none)
    uint32_t s_fast;       // min(s_max, floor((2^32 - 1) / cap_m)): no partition stops below it
    uint32_t cap_n; // largest n_j
    uint32_t cap_m; // largest m_j
    uint64_t* bkeys;       // [n] scratch for the bucket-sorted keys (used unless keys_in_smem)
    uint32_t keys_in_smem; // 1: keep each partition's keys in shared memory
    uint32_t window_bits;  // displacements per lane-window: 32 or 64 (speed only)
    uint32_t* pilots;      // zero-filled by the caller
    uint32_t* taken_bits;  // global occupancy bitmap over all slots in u32 words, zero-filled; may be null
    uint32_t* status;      // device status word (kDev* codes, atomicMax)
    unsigned long long* work;  // [2]: s tries, window steps (may be null)
    unsigned long long* queue; // work-queue counter (the launcher zeroes it)
    uint32_t use_queue;        // 1: persistent CTAs over a work queue; 0: one CTA per partition
    uint32_t warps;            // warps sharing one partition: 1, 2 or 4 (speed only)
};
// out[i] = src[idx[i]]
cudaError_t launch_gather_u64(const uint64_t* src, const uint64_t* idx, uint64_t* out, uint64_t count,
                              cudaStream_t stream);
size_t search_smem_bytes(uint32_t cap_n, uint32_t cap_m, uint32_t B, bool keys_in_smem, uint32_t warps);
size_t search_smem_limit();
cudaError_t launch_search(const SearchLaunch& a, cudaStream_t stream);

// ---- k_encode.cu: offsets and interleaved encoders, all key sets per launch ----
// offsets of one key set: its T values are T[part_base .. part_base + np]
struct OffDesc {
    uint64_t part_base, np, Q;  // Q = floor(M 2^32 / np)
    int64_t dmin;               // minimum stored difference (subtracted before packing)
    uint64_t dst_word;          // arena word where the set's packed offsets start
    uint32_t width, pad;
};
// one pilot column (bucket b of one key set)
struct ColDesc {
    uint64_t src;       // first pilot of the column in the pilot buffer
    uint64_t count;     // N_P of the set
    uint64_t dst_word;  // arena word where the set's packed pilots (IC-C) / ranks (IC-D) / low parts (IC-R) start
    uint64_t base;      // bit offset of this column inside that array
    uint32_t width;     // bits per value (IC-R: the Rice parameter)
    uint32_t dict_width;  // IC-D: bits per dictionary value
    uint64_t bm_base, bm_words;  // IC-D: the column's presence bitmap (words)
    uint64_t dict_dst_word, dict_base;  // IC-D: the set's dictionary array, this column's bit offset
    // IC-R: the set's select samples (u32) start at arena word samp_dst_word, this
    // column's at index samp_base; its unary bits at bit hi_base of the array at
    // arena word hi_dst_word
    uint64_t samp_dst_word, samp_base, hi_dst_word, hi_base;
    // a mono encoder's physical column b continues the set's single sequence:
    // idx0 = its first value's index b N_P, sum0 = the scanned quantity (Rice:
    // sum of pilot >> l; Elias-Fano: sum of pilots) of the columns before it.
    // Both 0 for an interleaved column.
    uint64_t idx0, sum0;
};
cudaError_t launch_offset_minmax(const uint64_t* T, const OffDesc* sets, uint32_t nsets, long long* mm,
                                 cudaStream_t stream);
cudaError_t launch_offset_pack(const uint64_t* T, const OffDesc* sets, uint32_t nsets, const uint64_t* word_begin,
                               uint64_t total_words, uint64_t* arena, cudaStream_t stream);
// colsum (may be null): sum of each column's pilots
cudaError_t launch_column_max(const uint32_t* pilots, const ColDesc* cols, uint32_t ncols, uint64_t max_count,
                              uint32_t* colmax, uint64_t* colsum, cudaStream_t stream);
// IC-R: hlen[c] = sum over the column of (pilot >> width), i.e. its unary bits minus N_P
cudaError_t launch_rice_unary_len(const uint32_t* pilots, const ColDesc* cols, uint32_t ncols, uint64_t* hlen,
                                  cudaStream_t stream);
// IC-R: unary bits and select samples of every column
cudaError_t launch_rice_unary(const uint32_t* pilots, const ColDesc* cols, uint32_t ncols, uint64_t* arena,
                              cudaStream_t stream);
// IC-EF: low bits, high bits and select samples of every column (prefix sums)
cudaError_t launch_ef_columns(const uint32_t* pilots, const ColDesc* cols, uint32_t ncols, uint64_t* arena,
                              cudaStream_t stream);
cudaError_t launch_pack_columns(const uint32_t* pilots, const ColDesc* cols, uint32_t ncols, const uint64_t* word_begin,
                                uint64_t total_words, bool ranks, const uint64_t* bitmaps,
                                const uint64_t* bitmaps_rank, uint64_t* arena, cudaStream_t stream);
cudaError_t launch_dict_mark(const uint32_t* pilots, const ColDesc* cols, uint32_t ncols, uint64_t* bitmaps,
                             cudaStream_t stream);
cudaError_t launch_dict_rank(const ColDesc* cols, uint32_t ncols, uint64_t* bitmaps_rank, const uint64_t* bitmaps,
                             uint64_t* K, cudaStream_t stream);
cudaError_t launch_dict_pack_values(const ColDesc* cols, uint32_t ncols, const uint64_t* bm_begin,
                                    uint64_t total_bm_words, const uint64_t* bitmaps, const uint64_t* bitmaps_rank,
                                    uint64_t* arena, cudaStream_t stream);

// ---- k_remap.cu: Elias-Fano remap of slots >= n (alpha < 1), all key sets per launch ----
struct RemapDesc {
    uint64_t g0, n, M;  // the set's slots are bits [g0, g0 + M) of the global occupancy bitmap
    uint64_t f_base;    // offset of the set's N = M - n entries in the F and fs buffers
    uint64_t low_dst, high_dst, samp_dst;  // arena words of the set's Elias-Fano arrays
    uint32_t l, pad;
};
size_t remap_scratch_bytes(uint64_t zwords, uint64_t twords, uint64_t ntotal);
cudaError_t launch_remap(const uint32_t* bm, const RemapDesc* d_sets, uint32_t nsets, const uint64_t* d_zbegin,
                         uint64_t zwords, const uint64_t* d_tbegin, uint64_t twords, const uint64_t* d_fbegin,
                         uint64_t ntotal, const uint64_t* d_lbegin, uint64_t lwords, uint64_t* arena, void* scratch,
                         cudaStream_t st);

// ---- k_query.cu ----
// one request of a coalesced query launch: keys[0 .. count) of one structure,
// at indexes [begin, begin + count) of the launch; the next request's begin
// (or the launch total) ends it
struct MultiQuery {
    QueryView v;
    const uint64_t* keys;
    uint64_t* out;
    uint64_t begin;
};
cudaError_t launch_query_multi(const MultiQuery* d_reqs, uint32_t nreq, uint64_t total, cudaStream_t stream);
// the query view of a handle (defined with the handle in phobic_api.cu)
}  // namespace phobic
struct phobic_handle;
namespace phobic {
const QueryView* handle_view(const phobic_handle* h);
// frees a handle that no in-flight work reads, without a device synchronisation
void handle_free_idle(phobic_handle* h, cudaStream_t st);
cudaError_t launch_query(const QueryView& v, const uint64_t* keys, uint64_t* out, uint64_t m, cudaStream_t stream);
cudaError_t launch_query_strings(const QueryView& v, const uint8_t* bytes, const uint64_t* offsets, uint64_t* out,
                                 uint64_t m, cudaStream_t stream);

// the calling thread's pinned read-back buffer, allocated ahead of its first build
cudaError_t warm_build_thread();

}  // namespace phobic
