/*
 * phobic.h -- C ABI of libphobic, a B300 (sm_103a) implementation of PHOBIC's
 * data-parallel hot path: partitioned pilot-search construction of a minimal
 * perfect hash function (MPHF) and its query.
 *
 * Paper: Hermann, Lehmann, Pibiri, Sanders, Walzer, "PHOBIC: Perfect Hashing
 * with Optimized Bucket Sizes and Interleaved Coding", arXiv 2404.18497.
 *
 * Problem (Section 1): n distinct keys are mapped one-to-one onto [0, n).
 * Output values are 0-based here; the paper writes [n] = {1..n}.
 *
 * Conventions for every entry point:
 *  - Pointers named d_* are CUDA device pointers on the current device; h_* are
 *    host pointers.  Sizes are element counts unless named *_bytes.
 *  - `stream` is a cudaStream_t (passed as phobic_stream_t so that this header
 *    needs no CUDA headers); NULL means the legacy default stream.
 *  - Entry points return a phobic_status.  No exception crosses the ABI and
 *    nothing is printed.  On error, *out handles are set to NULL and all
 *    temporaries are released.
 *  - The library allocates its own device memory (stream-ordered, from the
 *    device's default memory pool).  Inputs are borrowed, never freed.
 *  - Every step of construction and query runs in this library's CUDA kernels;
 *    there is no CPU fallback.
 */
#ifndef PHOBIC_H
#define PHOBIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* phobic_stream_t; /* same type as cudaStream_t */
typedef struct phobic_handle phobic_handle;   /* opaque: one built MPHF */

typedef enum {
    PHOBIC_OK = 0,
    PHOBIC_ERR_INVALID_ARG = 1,          /* bad size, pointer or parameter */
    PHOBIC_ERR_OOM = 2,                  /* device or host allocation failed */
    PHOBIC_ERR_DUP_HASH = 3,             /* two keys share a 64-bit master hash (duplicate keys) */
    PHOBIC_ERR_SEARCH_LIMIT = 4,         /* a bucket found no pilot below s_max, or holds > 1023 keys */
    PHOBIC_ERR_PARTITION_TOO_LARGE = 5,  /* a partition does not fit the search kernel's shared memory */
    PHOBIC_ERR_CUDA = 6,                 /* a CUDA runtime call failed */
    PHOBIC_ERR_TIMEOUT = 7,              /* a bounded device-side wait gave up */
    PHOBIC_ERR_FORMAT = 8                /* phobic_import: bytes are not a valid structure */
} phobic_status;

/* pilot encoders (Section 4.1, interleaved coding) */
typedef enum {
    PHOBIC_ENC_IC_C = 0, /* interleaved Compact: column width = bit length of its largest pilot */
    PHOBIC_ENC_IC_D = 1, /* interleaved Dictionary: sorted distinct pilots + compact ranks */
    PHOBIC_ENC_IC_R = 2, /* interleaved Golomb-Rice: per column, the low l bits packed at width l and the
                            rest in unary, l by Kiely's rule from the column mean; a select sample every
                            64 partitions.  Export layout: col_meta[2b] = low base | l << 56,
                            col_meta[2b+1] = unary base; the dictionary array holds the u32 select samples
                            (B x ceil(N_P/64), padded to whole words) followed by the unary bits */
    PHOBIC_ENC_IC_EF = 3, /* interleaved Elias-Fano: per column, the prefix sums E_j of its pilots with
                            l = floor(log2((E_last + 1) / N_P)) low bits packed, bit j + (E_j >> l) set in the
                            high part, a select sample every 64 partitions; the same export layout as IC-R */
    PHOBIC_ENC_IC_CR = 4, /* Section 4.1's mixture: the first c = min(compact_columns, B) columns (the largest
                             buckets) Compact, the others Golomb-Rice as IC-R.  The Compact values and Rice low
                             parts share the low array; col_meta[2b] = base | width << 56 for every column,
                             col_meta[2b+1] = unary base; select samples for columns b >= c only (sample
                             column b - c).  c is exported in bits 40..63 of the encoder header word */
    /* The "mono" encoders of the comparison in Section 5 (Figure 3b): ALL pilots in
     * one encoder, namely the column encoder above applied to a single column that
     * holds the B N_P pilots in column order (pilot of bucket b, partition j is value
     * b N_P + j).  One Compact width, one dictionary, one Rice parameter or one
     * Elias-Fano universe for the whole structure; the export layout is that of the
     * column encoder with one column (1 or 2 metadata words).  mono-R and mono-EF keep
     * 32-bit select samples, so their unary part must stay below 2^32 bits (about
     * 2 n / lambda bits): a larger build returns PHOBIC_ERR_INVALID_ARG. */
    PHOBIC_ENC_MONO_C = 5,
    PHOBIC_ENC_MONO_D = 6,
    PHOBIC_ENC_MONO_R = 7,
    PHOBIC_ENC_MONO_EF = 8
} phobic_encoder;

/* bucket assignment functions (Section 3, Figure 3a): the optimised beta_eps of
 * Theorem 2 (the default), and for ablations beta_* (eps = 0), PTHash's skewed
 * split (keys with normalised hash below 0.6 go to the first 30 % of the
 * buckets) and the uniform function of CHD.  For alpha < 1 each is rescaled as
 * gamma(alpha x) / gamma(alpha) (Appendix B). */
typedef enum {
    PHOBIC_BUCKET_OPTIMIZED = 0,
    PHOBIC_BUCKET_BETA_STAR = 1,
    PHOBIC_BUCKET_SKEWED = 2,
    PHOBIC_BUCKET_UNIFORM = 3
} phobic_bucket_function;

/* pilot hash (Section 4, "Hash Function") */
typedef enum {
    PHOBIC_PILOT_ADDITIVE = 0, /* p = s m + d; position (h(x, s) + d) mod m  (the paper's PHOBIC) */
    PHOBIC_PILOT_XOR = 1       /* PTHash: position h(x xor h(p)) reduced onto [0, m) */
} phobic_pilot_mode;

typedef struct {
    double lambda;                /* average bucket size, > 0 (Section 3) */
    double alpha;                 /* load factor in (0, 1]; < 1 builds on M = sum ceil(n_j/alpha) slots
                                     and remaps slots >= n with Elias-Fano (Section 5, Further Remarks) */
    uint32_t partition_size;      /* expected partition size P, 1..16384 (Section 4) */
    uint32_t encoder;             /* phobic_encoder */
    uint32_t pilot_mode;          /* phobic_pilot_mode */
    uint32_t s_max;               /* search limit: s < s_max (ADDITIVE), p < s_max*m (XOR); 0 = none beyond the
                                     32-bit pilot: in every partition s < floor((2^32-1)/m_j), which also
                                     caps any other value */
    uint64_t seed;                /* master-hash seed */
    uint32_t warps_per_partition; /* search tuning: warps sharing one partition, 1, 2, 4 or 8; 0 = chosen
                                     from the partition count and lambda (w = partitions / (32 x SMs);
                                     4 warps while w <= 0.15 e^(0.6 (lambda - 7)), 8 of them when also
                                     lambda >= 12 and w <= 1, else 1).  Several warps test consecutive
                                     candidate ranges of a bucket at once and the first success in
                                     enumeration order is kept, so results do not depend on it */
    uint32_t keep_pilots;         /* nonzero: keep the raw pilot matrix for phobic_copy_pilots */
    uint32_t record_timings;      /* nonzero: time the build phases with CUDA events on `stream` */
    uint32_t candidate_width;     /* search tuning: displacements per lane-window, 32 or 64 (0 = default 64);
                                     results do not depend on it */
    uint32_t search_schedule;     /* search tuning: 0 auto (one CTA per partition, the faster on this
                                     hardware for single builds and batches alike), 1 one CTA per
                                     partition, 2 persistent CTAs taking partitions from a device work
                                     queue; results do not depend on it */
    uint32_t bucket_function;     /* phobic_bucket_function: gamma of the bucket assignment (default 0) */
    uint32_t compact_columns;     /* PHOBIC_ENC_IC_CR: number of leading Compact columns (clamped to B) */
} phobic_params;

/* Device time of each build phase (CUDA events recorded on the build stream
 * around each phase's kernels; host gaps between phases are excluded). */
typedef struct {
    float sort_ms;     /* master hash + onesweep partition sort + partition starts */
    float sizes_ms;    /* table sizes m_j and offsets T */
    float search_ms;   /* bucketing + pilot search (one warp per partition) */
    float encode_ms;   /* offsets + interleaved pilot encoding */
    float remap_ms;    /* Elias-Fano remap of slots >= n (alpha < 1) */
    float total_ms;    /* first to last event, host synchronisations included */
    uint64_t search_s_tries; /* pilot-search work: (bucket, s) pairs tried */
    uint64_t search_steps;   /* pilot-search work: warp steps of the displacement scan */
} phobic_timings;

/* Structure sizes and space breakdown of a built MPHF. */
typedef struct {
    uint64_t n;             /* keys */
    uint64_t M;             /* slots = sum of table sizes m_j (M = n when alpha = 1) */
    uint64_t num_partitions;/* N_P = max(1, ceil(n / P)) */
    uint32_t num_buckets;   /* B = ceil(P / lambda) per partition */
    uint32_t partition_size;
    double lambda, alpha, epsilon;
    uint32_t encoder, pilot_mode;
    uint64_t seed;
    uint64_t max_partition; /* largest n_j */
    uint64_t bits_header, bits_offsets, bits_pilots, bits_remap, bits_total;
    uint64_t device_bytes;  /* device memory owned by the handle */
    uint32_t bucket_function;
    uint32_t compact_columns; /* PHOBIC_ENC_IC_CR: leading Compact columns (min(c, B)) */
} phobic_info;

/* Fills *p with the defaults: lambda 7, alpha 1, P 2500, IC-C, ADDITIVE,
 * s_max 0 (only the 32-bit pilot bound), seed 0. */
void phobic_params_init(phobic_params* p);

/*
 * Construction (Section 4 pipeline + Section 3 bucket function):
 *   hash keys -> radix-sort by partition -> per partition: bucket, order buckets by
 *   (size desc, expected size asc), pilot search -> offsets, interleaved encoding,
 *   Elias-Fano remap (alpha < 1).
 * d_keys: n distinct 64-bit keys (device), borrowed for the call.
 * The call returns after the device work finishes (the structure's sizes
 * depend on device results), so it synchronises `stream`.
 * Errors: INVALID_ARG for n = 0, NULL pointers, lambda <= 0, alpha outside (0,1],
 * P = 0, P > 16384 or P < lambda (a partition smaller than one average bucket);
 * DUP_HASH for duplicate keys; SEARCH_LIMIT; OOM; CUDA.
 * The environment variable PHOBIC_KEYS_IN_SMEM=1 makes the search keep each
 * partition's keys in shared memory instead of a bucket-sorted scratch array in
 * global memory (slower on this hardware; the results are the same).
 */
phobic_status phobic_build(const uint64_t* d_keys, uint64_t n, double lambda, double alpha,
                           uint32_t partition_size, uint64_t seed, phobic_stream_t stream,
                           phobic_handle** out);

/* Same, with every parameter of phobic_params. */
phobic_status phobic_build_ex(const uint64_t* d_keys, uint64_t n, const phobic_params* params,
                              phobic_stream_t stream, phobic_handle** out);

/*
 * Batched construction: n_sets independent key sets stored back to back in
 * d_keys, set s being d_keys[h_set_offsets[s] .. h_set_offsets[s+1]) (host array
 * of n_sets + 1 entries, strictly increasing: every set non-empty).  Each set
 * gets its own MPHF, exactly as phobic_build_ex would build it alone, with
 * partition size h_partition_sizes[s] (host array; NULL = params->partition_size
 * for all).  One segmented partition sort, one persistent search launch over the
 * partitions of all sets (device work queue) and one launch per encoding step
 * serve the whole batch.  out_handles[s] receives set s's handle; the handles
 * share one device allocation, released when the last of them is freed (each
 * must still be passed to phobic_free).  Errors as phobic_build_ex, for the
 * whole batch (no handle is returned on error).
 */
phobic_status phobic_build_batch(const uint64_t* d_keys, const uint64_t* h_set_offsets, uint32_t n_sets,
                                 const uint32_t* h_partition_sizes, const phobic_params* params,
                                 phobic_stream_t stream, phobic_handle** out_handles);

/*
 * Autotuner for phobic_build_batch (the paper has no counterpart).  From the
 * set sizes alone it picks, by timing trial batches of synthetic keys on the
 * current device (steady-state time per key: each trial and its first half are
 * built, and their difference is timed, so that a launch's fixed costs
 * cancel): the expected partition size of every set, one of 1024, 2500,
 * 4096, per decade size class (the fastest, or within 3% of it the one with the
 * fewest bits per key); and warps_per_partition (1, 2, 4) and candidate_width
 * (32, 64) for the launch, then with those the search schedule (one CTA per
 * partition, or persistent CTAs over the device work queue).  h_set_offsets as
 * for phobic_build_batch (only the sizes are read; no key is read).  Outputs:
 * h_partition_sizes_out[n_sets], *params_out = *params with the three search
 * knobs set;
 * *info (may be NULL) reports the measurements.  Decisions are cached for the
 * process per device and (lambda, alpha, encoder, pilot_mode, s_max): per size
 * class for P, per power of two of the partition count for the search knobs.
 * The trials allocate device memory (keys for up to about 2^27 + one set) and
 * synchronize `stream`.  Partition sizes below lambda are never tried (lambda
 * above 4096 leaves none: INVALID_ARG).  Errors: INVALID_ARG, OOM, CUDA, and any
 * build error of a trial.  Results of builds made with the outputs are exact
 * PHOBIC constructions with the chosen partition sizes.
 */
#define PHOBIC_TUNE_P_CHOICES 3
#define PHOBIC_TUNE_MAX_CLASSES 20
typedef struct {
    uint32_t sets;           /* sets of the batch in this class (0: none) */
    uint32_t partition_size; /* chosen expected partition size */
    float ns_per_key[PHOBIC_TUNE_P_CHOICES];   /* steady-state trial time per key for P = 1024, 2500, 4096 */
    float bits_per_key[PHOBIC_TUNE_P_CHOICES]; /* trial bits per key for the same */
} phobic_tune_class;
typedef struct {
    phobic_tune_class classes[PHOBIC_TUNE_MAX_CLASSES]; /* class c: sizes in [10^c, 10^(c+1)) */
    uint32_t warps_per_partition;
    uint32_t candidate_width;
    float launch_ns_per_key[6]; /* (warps, width) = (1,32) (1,64) (2,32) (2,64) (4,32) (4,64) */
    uint64_t total_partitions;  /* of the batch with the chosen sizes */
    uint32_t cached_classes;    /* classes answered from the cache */
    uint32_t cached_launch;     /* 1: search knobs answered from the cache */
    uint32_t search_schedule;   /* chosen: 1 one CTA per partition, 2 persistent CTAs over the work queue */
    float schedule_ns_per_key[2]; /* trial time per key of schedules 1 and 2 with the chosen warps and width */
} phobic_tune_info;
phobic_status phobic_tune_batch(const uint64_t* h_set_offsets, uint32_t n_sets, const phobic_params* params,
                                phobic_stream_t stream, uint32_t* h_partition_sizes_out,
                                phobic_params* params_out, phobic_tune_info* info);
/* Forget every tuning decision and free the trial keys. */
void phobic_tune_clear(void);

/* Same, from host memory: the keys are copied to a temporary device buffer on
 * `stream` (one copy; page-locked host memory gives the full link bandwidth),
 * then built as phobic_build_ex builds them. */
phobic_status phobic_build_host(const uint64_t* h_keys, uint64_t n, const phobic_params* params,
                                phobic_stream_t stream, phobic_handle** out);

/*
 * Query (Section 4 "Hash Function"): per key, partition j, offsets T_j, T_{j+1},
 * bucket b, decoded pilot p, local position (h(x, floor(p/m)) + p) mod m, global
 * position T_j + local, remapped through Elias-Fano when >= n.
 * d_keys [m] in, d_out [m] out (uint64, values in [0, n)).  Asynchronous and
 * stream-ordered: the caller keeps both buffers alive until `stream` is done.
 * A key outside the built set gets an unspecified value in [0, n).
 * m = 0 is a no-op.  Errors: INVALID_ARG (NULL handle/pointers), CUDA.
 */
phobic_status phobic_query(const phobic_handle* h, const uint64_t* d_keys, uint64_t* d_out, uint64_t m,
                           phobic_stream_t stream);

/*
 * Coalesced query (the paper has no counterpart; a serving convenience):
 * n_req batches against possibly different handles in one kernel launch.
 * Batch r: d_keys[r][0 .. counts[r]) against handles[r] into d_outs[r].  The
 * results equal those of n_req separate phobic_query calls.  The host arrays
 * are read before the call returns; the device buffers follow phobic_query's
 * rules.  Handles must be built from 64-bit keys.  Batches with counts[r] = 0
 * are skipped.  Errors: INVALID_ARG (NULL array, NULL or string handle, NULL
 * buffer of a non-empty batch), OOM, CUDA.
 */
phobic_status phobic_query_multi(const phobic_handle* const* handles, const uint64_t* const* d_keys,
                                 uint64_t* const* d_outs, const uint64_t* counts, uint32_t n_req,
                                 phobic_stream_t stream);

/* Query from host memory; returns after the results are in h_out.  Up to 2^22
 * keys go in one piece.  Larger batches are pipelined in chunks of 2^22 keys over
 * three device slots: chunk c+1 is copied in and chunk c queried on `stream`
 * while chunk c-1's results are copied out on a second stream of the calling
 * thread, so both copy directions overlap.  Page-locked host memory is needed
 * for the copies to overlap. */
phobic_status phobic_query_host(const phobic_handle* h, const uint64_t* h_keys, uint64_t* h_out,
                                uint64_t m, phobic_stream_t stream);

/*
 * String keys (Section 5: strings of 10-50 characters, reduced to 64-bit master
 * hash codes with xxHash).  String i is d_bytes[d_offsets[i] .. d_offsets[i+1]);
 * d_offsets has n+1 (m+1) entries and d_bytes must be readable for
 * d_offsets[n] bytes.  The master hash is XXH64 with params->seed.  Two
 * distinct strings with equal XXH64 give DUP_HASH (rebuild with another seed).
 * Query semantics and errors as for 64-bit keys; a handle built from strings
 * only answers phobic_query_strings, and a 64-bit handle only phobic_query.
 */
phobic_status phobic_build_strings(const uint8_t* d_bytes, const uint64_t* d_offsets, uint64_t n,
                                   const phobic_params* params, phobic_stream_t stream, phobic_handle** out);
phobic_status phobic_query_strings(const phobic_handle* h, const uint8_t* d_bytes, const uint64_t* d_offsets,
                                   uint64_t* d_out, uint64_t m, phobic_stream_t stream);

/* Space of the structure in bits per key (fixed accounting: header, offsets,
 * pilot encoders with their metadata, Elias-Fano remap).  NaN for NULL. */
double phobic_bits_per_key(const phobic_handle* h);

/* Structure sizes; INVALID_ARG for NULL. */
phobic_status phobic_get_info(const phobic_handle* h, phobic_info* info);

/*
 * Serialization (exact words).  With h_buf NULL, *len receives the byte size.
 * Otherwise *len is the buffer capacity on input and the bytes written on
 * output.  Synchronises the device.
 *
 * Format version 1, little-endian u64 words throughout.  A 28-word header:
 *   0 magic "PHOBIC01" (0x31304349424F4850)   1 version (1)
 *   2 n   3 M (table slots, >= n)   4 N_P (partitions)   5 B (buckets per partition)
 *   6 partition size P   7 lambda (IEEE double bits)   8 alpha (double bits)   9 seed
 *  10 encoder | bucket_function << 32 | compact_columns << 40
 *  11 pilot_mode | key_kind << 32 (0: u64 keys, 1: byte strings)
 *  12 offset width   13 offset slope Q   14 offset minimum (two's complement)
 *  15 Elias-Fano low bits of the remap
 *  16..22 word counts of the seven arrays below, in order
 *  23..27 space in bits: header, offsets, pilots, remap, total
 * followed by the seven arrays: packed offsets; column metadata (base | width
 * << 56, one or two words per column as the encoder's documentation above
 * says); packed values / ranks / low parts; dictionary, or u32 select samples
 * padded to whole words followed by unary bits; Elias-Fano remap low bits,
 * high bits and u64 select samples (empty when M = n).  Every packed array ends
 * with one padding word.  The bucket table is not stored: it follows from
 * lambda, alpha, P and the bucket function.
 */
phobic_status phobic_export(const phobic_handle* h, void* h_buf, size_t* len);

/* Rebuilds a handle from phobic_export bytes (FORMAT on malformed input, after
 * the checks of phobic_inspect). */
phobic_status phobic_import(const void* h_buf, size_t len, phobic_stream_t stream, phobic_handle** out);

/* Validates phobic_export bytes on the host, without a device, and fills info
 * as phobic_get_info would for the imported handle (device_bytes: what
 * phobic_import would allocate).  The checks are those phobic_import makes
 * before any copy:
 *   - magic and version;
 *   - parameters that phobic_build would accept, with N_P and B as they imply;
 *   - array sizes that add up to len;
 *   - every metadata entry inside its array;
 *   - for the unary encoders, each column's unary region holds exactly its
 *     number of ones, and every select sample is the position of its one.
 * Errors: FORMAT, INVALID_ARG (info NULL).  Safe on untrusted input: reads
 * stay within len, and the work is linear in len (checks whose loops the file
 * does not pay for in bits, such as zero-width offsets or ranks, are made in
 * closed form). */
phobic_status phobic_inspect(const void* h_buf, size_t len, phobic_info* info);

/* Copies the raw pilot matrix [B x N_P] (pilot of bucket b of partition j at
 * b * N_P + j) to d_out; needs params.keep_pilots at build time (else INVALID_ARG). */
phobic_status phobic_copy_pilots(const phobic_handle* h, uint32_t* d_out, phobic_stream_t stream);

/* Phase timings of the build that produced h (needs params.record_timings;
 * else INVALID_ARG). */
phobic_status phobic_get_timings(const phobic_handle* h, phobic_timings* t);

/* Number of CUDA kernels this library has launched in this process so far
 * (diagnostic; counts every launch of every entry point). */
uint64_t phobic_kernel_launches(void);

/* Device memory: builds take their buffers from the current device's default
 * stream-ordered pool, which keeps freed memory cached for the next build.
 * phobic_trim synchronizes the device and returns cached memory above
 * keep_bytes to the system; phobic_pool_bytes reports the pool's reserved and
 * in-use bytes (handles and running builds).  Errors: INVALID_ARG, CUDA. */
phobic_status phobic_trim(uint64_t keep_bytes);
phobic_status phobic_pool_bytes(uint64_t* reserved, uint64_t* used);

/* Releases every device buffer of h (synchronises the device).  NULL is a no-op. */
void phobic_free(phobic_handle* h);

/* Static string naming a status. */
const char* phobic_status_str(phobic_status s);

/* ---- stage entry points (each runs one kernel of the pipeline) ---- */

/* Master hash codes of 64-bit keys (Section 5: keys first become 64-bit hashes):
 * d_hk[i] = mix64(d_keys[i] xor mix64(seed xor C)); a bijection. */
phobic_status phobic_hash_u64(const uint64_t* d_keys, uint64_t n, uint64_t seed, uint64_t* d_hk,
                              phobic_stream_t stream);

/* Master hash codes of n byte strings: string i is d_bytes[d_offsets[i] ..
 * d_offsets[i+1]) (d_offsets has n+1 entries); 64-bit XXH64 with `seed`. */
phobic_status phobic_hash_strings(const uint8_t* d_bytes, const uint64_t* d_offsets, uint64_t n,
                                  uint64_t seed, uint64_t* d_hk, phobic_stream_t stream);

/* Radix sort (onesweep) of the master hashes d_hk[n] by partition id
 * j = floor(hk * num_partitions / 2^64) into d_sorted[n] (keys of partition j
 * contiguous, partitions ascending, order inside a partition unspecified), and
 * the partition starts d_start[num_partitions + 1].  Allocates its scratch. */
phobic_status phobic_partition_sort(const uint64_t* d_hk, uint64_t n, uint64_t num_partitions,
                                    uint64_t* d_sorted, uint64_t* d_start, phobic_stream_t stream);

/*
 * Self-test of failure detection in the partition sort (the paper has no
 * counterpart).  Every wait of the sort's decoupled look-back is bounded: after
 * a number of polls of a predecessor tile that has not published its state,
 * the kernel records a timeout in a device status word, stops waiting and
 * finishes; the call then returns PHOBIC_ERR_TIMEOUT and the context stays
 * usable.  This entry point runs phobic_partition_sort with tile mute_tile
 * (of 6144 keys each) withholding its state, so that the wait of the tile after
 * it runs out after spin_limit polls (a flag that nothing sets).  Nothing faults
 * or hangs.  Returns TIMEOUT when a wait ran out, OK when none did (mute_tile
 * past the last tile, or a single pass-free sort); d_sorted / d_start are then
 * unspecified.  Errors: INVALID_ARG (as phobic_partition_sort, or spin_limit 0),
 * OOM, CUDA.
 */
phobic_status phobic_selftest_sort_wait_timeout(const uint64_t* d_hk, uint64_t n, uint64_t num_partitions,
                                                uint64_t mute_tile, uint32_t spin_limit, uint64_t* d_sorted,
                                                uint64_t* d_start, phobic_stream_t stream);

/* Largest n accepted by phobic_partition_sort_noalloc. */
#define PHOBIC_NOALLOC_MAX_KEYS 1048576u

/*
 * phobic_partition_sort without any device allocation.  The paper has no
 * counterpart: this serves callers that may not allocate device memory while
 * they run, such as a process whose device budget is fully reserved up front
 * (an extra cudaMalloc could fail or push out other data) or a host framework
 * that owns every allocation and forbids libraries from calling the CUDA
 * allocator themselves.  The caller still owns d_hk, d_sorted and d_start;
 * the sort's temporary space comes from one fixed array of about 9.1 MiB inside
 * this library, which every GPU that loads the library holds until the
 * process exits.
 * Same inputs, outputs and results as phobic_partition_sort, for
 * n <= PHOBIC_NOALLOC_MAX_KEYS; a larger n (or a partition count whose digit
 * tables would not fit) returns PHOBIC_ERR_INVALID_ARG.
 * The first call on a device looks up the array's device address and keeps
 * it for the life of the process, so the library must not be used on a
 * device after cudaDeviceReset (the array's address may change).  Every call
 * synchronises `stream` and reads the sort's error word back to the host, so
 * it must not be called while `stream` (or the legacy default stream) is
 * being captured into a CUDA graph.  All calls share the one array, so calls
 * whose work overlaps on the GPU (on different streams or threads) race with
 * each other: the caller must serialise them.  Calls no cudaMalloc, cudaFree
 * or other allocating routine.
 */
phobic_status phobic_partition_sort_noalloc(const uint64_t* d_hk, uint64_t n, uint64_t num_partitions,
                                            uint64_t* d_sorted, uint64_t* d_start, phobic_stream_t stream);

/* ---- partition-sharded construction (Section 4: partitions are independent) ----
 *
 * One MPHF over n keys that are spread over several devices (one process per
 * device).  Partition j = floor(hk N_P / 2^64) belongs to shard
 * r = floor(j G / N_P) of G; a shard's partitions are the contiguous range
 * [ceil(r N_P / G), ceil((r + 1) N_P / G)).  Each process hashes its keys
 * (phobic_hash_u64) and groups them by partition (phobic_partition_sort with
 * the build's N_P), sends every shard the hashes of its partitions, and groups
 * what it receives again.  From the partition sizes of all shards it forms the
 * build's partition starts, and phobic_table_offsets turns them into the slot
 * offsets T.  phobic_search_partitions places the buckets of its own partitions
 * into a zero-filled pilot matrix and occupancy bitmap of the whole build;
 * summing those over the shards (their supports are disjoint, so the sum is the
 * union) gives every shard the whole build's pilots and occupancy, from which
 * phobic_assemble makes the same structure that phobic_build_ex makes from all
 * n keys on one device.  The exchanges are the caller's (the Python binding's
 * sharded_build does them with torch.distributed).
 */

/* Slot offsets from partition starts (Section 4: m_j = n_j for alpha = 1,
 * else max(n_j, ceil(n_j / alpha)) in IEEE double; T is the exclusive prefix
 * sum of m).  d_start: N_P + 1 partition starts (n_j = d_start[j+1] -
 * d_start[j]), device.  Writes d_T[N_P + 1] (device, T[N_P] = M) and, when
 * h_stats is not NULL, h_stats[0..2] = M, the largest n_j, the largest m_j.
 * Synchronises `stream`.  Errors: INVALID_ARG (NULL pointers, N_P = 0, alpha
 * outside (0, 1]), OOM, CUDA. */
phobic_status phobic_table_offsets(const uint64_t* d_start, uint64_t num_partitions, double alpha, uint64_t* d_T,
                                   uint64_t* h_stats, phobic_stream_t stream);

/* Bucketing and pilot search (Sections 3 and 4) of partitions [j0, j1) of an
 * n-key build with num_partitions = max(1, ceil(n / P)) partitions: one shard
 * of a partition-sharded build.
 *   d_sorted [n_local]: the master hashes of exactly those partitions, grouped
 *     by partition ascending (phobic_partition_sort with num_partitions leaves
 *     them so);
 *   d_start [num_partitions + 1]: starts into d_sorted; entries j0..j1 are read;
 *   d_T [num_partitions + 1]: the whole build's slot offsets
 *     (phobic_table_offsets of the whole build's partition starts).
 * Writes the pilot of bucket b of partition j, j0 <= j < j1, to
 * d_pilots[b * num_partitions + j] (the caller zero-fills d_pilots: empty
 * buckets are not written) and, when d_taken is not NULL, ORs the occupied
 * slots of those partitions into d_taken, the occupancy bitmap of the whole
 * build over its M slots (u32 words, bit g % 32 of word g / 32 = slot g,
 * zero-filled by the caller, (M + 31) / 32 + 1 words).  Pilots are those a
 * build of all n keys finds.  Synchronises `stream`.  Errors: INVALID_ARG (as
 * phobic_build_ex, a partition count other than max(1, ceil(n / P)), j0 > j1,
 * j1 > num_partitions, NULL pointers), PARTITION_TOO_LARGE, DUP_HASH,
 * SEARCH_LIMIT, OOM, CUDA; j0 = j1 does nothing. */
phobic_status phobic_search_partitions(const uint64_t* d_sorted, uint64_t n_local, const uint64_t* d_start,
                                       const uint64_t* d_T, uint64_t n, uint64_t num_partitions, uint64_t j0,
                                       uint64_t j1, const phobic_params* params, uint32_t* d_pilots, uint32_t* d_taken,
                                       phobic_stream_t stream);

/* The rest of a build from its partition starts and pilots: table sizes and
 * offsets, offsets as differences to their expectation (Section 4),
 * interleaved pilot encoding (Section 4.1) and, for alpha < 1, the Elias-Fano
 * remap of slots >= n.  d_start [N_P + 1] (device): the whole build's
 * partition starts, d_start[N_P] = n; d_pilots [B x N_P] (device): every
 * pilot; d_taken (device): the occupancy bitmap as phobic_search_partitions
 * leaves it summed over all shards (required when M > n, else may be NULL).
 * The handle equals the one phobic_build_ex makes from the same n 64-bit keys
 * with the same params (same export bytes, same answers); the inputs are
 * borrowed for the call.  Synchronises `stream`.  Errors: INVALID_ARG (as
 * phobic_build_ex, NULL pointers, starts that do not end at n, d_taken NULL
 * with M > n), OOM, CUDA. */
phobic_status phobic_assemble(const uint64_t* d_start, uint64_t n, const uint32_t* d_pilots, const uint32_t* d_taken,
                              const phobic_params* params, phobic_stream_t stream, phobic_handle** out);

/* Writes the 2049-entry fixed-point bucket table (Appendix C) to h_table. */
phobic_status phobic_bucket_table(double lambda, double alpha, uint32_t partition_size, uint64_t* h_table);
/* The same for any phobic_bucket_function. */
phobic_status phobic_bucket_table_ex(double lambda, double alpha, uint32_t partition_size, uint32_t bucket_function,
                                     uint64_t* h_table);

/*
 * Serving (the paper has no counterpart; a deployment layer that leaves the
 * construction and query arithmetic untouched).  A server keeps built MPHFs
 * resident on the current device and accepts requests from any host thread:
 *   build:   keys on the device -> a resident MPHF id (in the completion);
 *   query:   resident id, keys, output on the device -> positions in the output;
 *   release: resident id -> its memory returned.
 * Continuous mode (serial = 0): builds are admitted in arrival order while at
 * most build_slots run and the bytes of resident MPHFs plus the estimated
 * peak of admitted builds (32 B/key + 64 MiB) stay within hbm_budget_bytes
 * (0: no limit; a build larger than the budget runs alone); each build slot
 * has its own host thread and stream.  Pending queries against any resident
 * MPHFs are coalesced into one launch (at most max_batch_requests requests and
 * max_batch_keys keys) on a high-priority stream while builds run; up to
 * launch_slots coalesced launches are in flight.  A release completes once no
 * submitted query reads the MPHF.  Serial mode (serial = 1): one request at a
 * time in arrival order, each as its own launch sequence waited for to
 * completion; the budget is not applied.
 * Ownership: the caller keeps keys and outputs alive until the request's
 * completion is polled.  `ready` (may be NULL) is an event that the request's
 * input waits for; it must not be recorded again before that completion.
 * Results equal those of phobic_build_ex / phobic_query on the same inputs.
 * Errors at submission: INVALID_ARG (NULL arguments, unknown or releasing id,
 * an MPHF of string keys, a stopped server), OOM.  A request's own outcome is
 * the status of its completion.  phobic_server_destroy waits for every
 * submitted request, then frees every resident MPHF.
 */
typedef struct phobic_server phobic_server;
typedef struct CUevent_st* phobic_event_t; /* same type as cudaEvent_t */
enum { PHOBIC_REQ_BUILD = 0, PHOBIC_REQ_QUERY = 1, PHOBIC_REQ_RELEASE = 2 };
typedef struct {
    uint64_t hbm_budget_bytes;
    uint32_t build_slots;        /* 0: 2 */
    uint32_t max_batch_requests; /* 0: 1024 */
    uint64_t max_batch_keys;     /* 0: 2^24 */
    uint32_t launch_slots;       /* 0: 4 */
    uint32_t serial;
} phobic_server_config;
typedef struct {
    uint64_t request_id;
    uint32_t kind;             /* PHOBIC_REQ_* */
    int32_t status;            /* phobic_status of the request */
    uint64_t handle_id;        /* build: the new MPHF's id (0 on error); query, release: the target */
    uint64_t keys;             /* keys built or queried */
    int64_t t_submit_ns;       /* steady clock: submission, start on the device side, completion */
    int64_t t_start_ns;
    int64_t t_done_ns;
    uint32_t batch_requests;   /* query: requests in its launch */
    uint32_t pad;
    uint64_t batch_id;         /* query: its launch */
} phobic_completion;
typedef struct {
    uint64_t resident_bytes, reserved_bytes, peak_accounted_bytes, resident_handles;
    uint64_t builds_done, queries_done, releases_done;
    uint64_t query_launches, max_batch_requests_seen, builds_waited_for_memory;
    uint64_t pending;
} phobic_server_stats;
void phobic_server_config_init(phobic_server_config* c);
phobic_status phobic_server_create(const phobic_server_config* cfg, phobic_server** out);
phobic_status phobic_server_submit_build(phobic_server* s, const uint64_t* d_keys, uint64_t n,
                                         const phobic_params* params, phobic_event_t ready, uint64_t* request_id);
phobic_status phobic_server_submit_query(phobic_server* s, uint64_t handle_id, const uint64_t* d_keys,
                                         uint64_t* d_out, uint64_t m, phobic_event_t ready, uint64_t* request_id);
phobic_status phobic_server_submit_release(phobic_server* s, uint64_t handle_id, uint64_t* request_id);
/* Up to cap completions, oldest first; *count receives how many. */
phobic_status phobic_server_poll(phobic_server* s, phobic_completion* out, uint32_t cap, uint32_t* count);
/* Waits until every submitted request has completed; TIMEOUT after timeout_s seconds. */
phobic_status phobic_server_drain(phobic_server* s, double timeout_s);
/* The resident MPHF with this id (borrowed: valid until its release). */
phobic_status phobic_server_handle(phobic_server* s, uint64_t handle_id, const phobic_handle** out);
phobic_status phobic_server_get_stats(phobic_server* s, phobic_server_stats* out);
void phobic_server_destroy(phobic_server* s);

#ifdef __cplusplus
}
#endif
#endif /* PHOBIC_H */
