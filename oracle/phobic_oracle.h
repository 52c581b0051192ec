/*
 * PHOBIC CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, sequential C restatement of PHOBIC (Hermann, Lehmann, Pibiri,
 * Sanders, Walzer: "PHOBIC: Perfect Hashing with Optimized Bucket Sizes and
 * Interleaved Coding", arXiv 2404.18497).  It exists to check the CUDA library
 * and is only ever loaded by the tests, by the smoke check and by the
 * benchmark's CPU-baseline leg.  It shares no code with the CUDA path.
 *
 * Parity status per function is stated in phobic_oracle.c.  The three hash
 * constants are this implementation's own fixed spec and are "parity unpinned":
 * they are pinned only statistically (mix64, SplitMix64's output function, is
 * pinned to that generator's known outputs; XXH64 to published known answers).
 */
#ifndef PHOBIC_ORACLE_H
#define PHOBIC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes (same numbering as the library's, by spec) */
#define OR_OK 0
#define OR_ERR_INVALID_ARG 1
#define OR_ERR_OOM 2
#define OR_ERR_DUP_HASH 3
#define OR_ERR_SEARCH_LIMIT 4

#define OR_ENC_IC_C 0
#define OR_ENC_IC_D 1
#define OR_ENC_IC_R 2
#define OR_ENC_IC_EF 3
#define OR_ENC_IC_CR 4 /* mixture: the first compact_columns columns Compact, the rest Golomb-Rice */
/* mono-X: encoder X (C, D, R, EF) applied to ONE column holding all B N_P pilots
 * in column order (value i = b N_P + j); the comparison of Section 5, Figure 3b */
#define OR_ENC_MONO_C 5
#define OR_ENC_MONO_D 6
#define OR_ENC_MONO_R 7
#define OR_ENC_MONO_EF 8

/* bucket assignment functions (Figure 3a): the optimised beta_eps (Theorem 2),
 * beta_* (eps = 0), PTHash's skewed split (60 % of the keys into 30 % of the
 * buckets) and the uniform one (CHD) */
#define OR_BUCKET_OPTIMIZED 0
#define OR_BUCKET_BETA_STAR 1
#define OR_BUCKET_SKEWED 2
#define OR_BUCKET_UNIFORM 3

#define OR_PILOT_ADDITIVE 0
#define OR_PILOT_XOR 1

#define OR_TABLE_POINTS 2048      /* Appendix C: gamma tabulated at 2048 points */
#define OR_MAX_BUCKET 1023        /* buckets above this size are rejected as unplaceable */

typedef struct {
    double lambda;          /* average bucket size */
    double alpha;           /* load factor, (0, 1] */
    uint32_t partition_size;/* expected partition size P */
    uint32_t encoder;       /* OR_ENC_* */
    uint32_t pilot_mode;    /* OR_PILOT_* */
    uint32_t s_max;         /* search limit on s (ADDITIVE) or p/m (XOR); 0: only the 32-bit pilot bound,
                               s < floor((2^32 - 1) / m_j), which also caps any other value */
    uint64_t seed;
    uint32_t bucket_fn;     /* OR_BUCKET_*: the bucket assignment function gamma */
    uint32_t compact_columns; /* OR_ENC_IC_CR: columns 0 .. c-1 Compact, the rest Golomb-Rice */
} or_params;

typedef struct or_mphf or_mphf;

/* ---- primitives, exported so that the pin tests can call them ---- */
uint64_t or_mix64(uint64_t z);
uint64_t or_mulhi64(uint64_t a, uint64_t b);
uint32_t or_bitlen(uint64_t v);
/* Golomb-Rice parameter of a column with `count` values summing to `sum`
 * (Kiely's choice for a geometric source with the column's mean). */
uint32_t or_rice_param(uint64_t sum, uint64_t count);
double   or_beta_star(double x);
double   or_gamma(double x, double eps, double alpha);
double   or_epsilon(double lambda, uint32_t P);
void     or_bucket_table(double lambda, double alpha, uint32_t P, uint64_t* table /* 2049 */);
/* gamma of one of the OR_BUCKET_* functions, with the alpha rescaling, and its table */
double   or_gamma_fn(double x, double eps, double alpha, uint32_t fn);
void     or_bucket_table_fn(double lambda, double alpha, uint32_t P, uint32_t fn, uint64_t* table);
uint32_t or_num_buckets(double lambda, uint32_t P);
uint64_t or_num_partitions(uint64_t n, uint32_t P);
uint32_t or_bucket(uint64_t x, const uint64_t* table, uint32_t B);
uint64_t or_key_hash(uint64_t key, uint64_t seed);
void     or_key_hash_array(const uint64_t* keys, uint64_t n, uint64_t seed, uint64_t* out);
void     or_string_hash_array(const uint8_t* bytes, const uint64_t* offsets, uint64_t n, uint64_t seed, uint64_t* out);
uint64_t or_bucket_hash(uint64_t hk);
uint64_t or_position_hash(uint64_t hk, uint64_t s, uint64_t m);
uint64_t or_table_size(uint64_t n_j, double alpha);
uint64_t or_string_hash(const uint8_t* bytes, uint64_t len, uint64_t seed);

/* ---- whole build / query ---- */
int  or_build(const uint64_t* keys, uint64_t n, const or_params* prm, int threads, or_mphf** out);
int  or_build_hashed(const uint64_t* hk, uint64_t n, const or_params* prm, int threads, or_mphf** out);
void or_free(or_mphf* h);
void or_query(const or_mphf* h, const uint64_t* keys, uint64_t q, uint64_t* out);
void or_query_hashed(const or_mphf* h, const uint64_t* hk, uint64_t q, uint64_t* out);
double or_bits_per_key(const or_mphf* h);
uint64_t or_get_u64(const or_mphf* h, const char* name);
const void* or_get_array(const or_mphf* h, const char* name, uint64_t* count, uint32_t* elem_bytes);

/* ---- sampled mode for very large inputs ---- */
/* partition sizes n_j of all NP partitions (hashing only) */
int or_partition_sizes(const uint64_t* hk, uint64_t n, const or_params* prm, uint64_t* n_j /* NP */);
/* pilots of the listed partitions only; pilots_out is [nsel x B], row = selected partition */
int or_search_partitions(const uint64_t* hk, uint64_t n, const or_params* prm,
                         const uint64_t* sel, uint64_t nsel, int threads, uint32_t* pilots_out);

/* one partition's search from its own hashes: pilots_out[B], taken_out[m] */
int or_search_one_partition(const uint64_t* hk, uint64_t nj, const or_params* prm, uint32_t* pilots_out,
                            uint8_t* taken_out);

/* ---- tiny-n re-verification helper: returns 1 if every p' < pilot fails ---- */
int or_verify_first_valid(const or_mphf* h, const uint64_t* hk);

#ifdef __cplusplus
}
#endif
#endif
