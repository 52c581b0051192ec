/*
 * PHOBIC CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg load
 * this file's shared object.  The CUDA library never calls it, and the two share
 * no code: each restates the same written rules on its own.
 *
 * What it computes is PHOBIC (arXiv 2404.18497), step by step, sequentially,
 * with the simplest data structures:
 *   - Section 3 (Optimizing Bucket Sizes): the bucket assignment function.  It
 *     is beta_* with derivative -ln(1-x), perturbed by Theorem 2 to
 *     beta_eps = eps x + (1-eps) beta_*.  Appendix C sets eps = lambda/(5 sqrt P),
 *     tabulates gamma at 2048 points and interpolates linearly.  Appendix B maps
 *     alpha < 1 through gamma_alpha(x) = gamma(alpha x)/gamma(alpha).
 *   - Section 4 (Fine-Grained Partitioning): partitions of expected size P.
 *     Offsets are stored as differences to their expectation.  The additive
 *     displacement pilot is p = s m + d, with position (h(x, s) + d) mod m.
 *   - Section 1 / Section 3: buckets are placed in non-increasing size.
 *     Section 5 ("Further Remarks") adds a secondary order: increasing expected
 *     size.
 *   - Section 4.1 (Interleaved Coding): encoder i holds the pilot of bucket i of
 *     every partition (Compact; Dictionary as named in Figure 3b; Golomb-Rice
 *     with Kiely's parameter and a select sample every 64 values; Elias-Fano
 *     over the column's prefix sums, named in Figure 3b as IC-EF; and the
 *     mixture of Section 4.1 with Compact for the first columns, the large
 *     buckets, and Golomb-Rice for the rest).
 *   - Section 5 ("Further Remarks"): the PTHash non-minimal trick of building on
 *     M > n slots and remapping slots >= n onto free slots < n, with Elias-Fano.
 *
 * Readings where the paper is silent (hash functions, rounding of B and m_j,
 * bit layouts, bits/key accounting) follow one fixed written spec.  The CUDA
 * library implements the same spec independently.  The three hash constants
 * below are "parity unpinned": nothing in the paper fixes them, so they are
 * pinned only by their statistical effect.  The mixer around them is
 * SplitMix64's output function, pinned to that generator's known outputs, and
 * the string hash is XXH64, pinned to published known answers for every input
 * path (tails, lanes, stripes, seeds).  The bits/key accounting is pinned by a
 * term-by-term recount from independently derived sizes.
 *
 * Floating point appears only in building the bucket table and in
 * ceil(n_j / alpha).  Compile with -ffp-contract=off so that no fused
 * multiply-add changes a rounding.
 */
#include "phobic_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* fixed spec constants (this implementation's own choice)                   */
/* ------------------------------------------------------------------------- */
#define C_SEED 0x9E3779B97F4A7C15ULL /* mixes the user seed */
#define C_BUCKET 0x5851F42D4C957F2DULL /* separates the bucket hash from hk */
#define C_PILOT 0x2545F4914F6CDD1DULL  /* separates the pilot hash */

/* SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014, "Fast splittable
 * pseudorandom number generators"; the "mix64" variant with shifts 30/27/31).
 * A bijection on 64-bit words. */
uint64_t or_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* floor(a * b / 2^64): "fastrange" reduction of a 64-bit hash onto [0, b) */
uint64_t or_mulhi64(uint64_t a, uint64_t b) {
    return (uint64_t)(((unsigned __int128)a * (unsigned __int128)b) >> 64);
}

/* number of bits needed to write v in binary; 0 for v = 0 */
uint32_t or_bitlen(uint64_t v) {
    uint32_t b = 0;
    while (v) {
        b++;
        v >>= 1;
    }
    return b;
}

/* ------------------------------------------------------------------------- */
/* Section 3: bucket assignment function                                      */
/* ------------------------------------------------------------------------- */

/* beta_*(x) = x + (1 - x) ln(1 - x)   (Section 3.2), with beta_*(1) = 1 */
double or_beta_star(double x) {
    if (x >= 1.0) return 1.0;
    return x + (1.0 - x) * log1p(-x);
}

/* Appendix C: eps = lambda / (5 sqrt(P)); clamped to 1 so that beta_eps stays
 * a bucket assignment function (reading: the paper never has eps > 1). */
double or_epsilon(double lambda, uint32_t P) {
    double eps = lambda / (5.0 * sqrt((double)P));
    if (eps > 1.0) eps = 1.0;
    return eps;
}

/* gamma(x) = beta_eps(x) = eps x + (1 - eps) beta_*(x)   (Theorem 2), and for
 * alpha < 1 the non-minimal variant gamma_alpha(x) = gamma(alpha x)/gamma(alpha)
 * (Appendix B). */
double or_gamma(double x, double eps, double alpha) {
    if (alpha == 1.0) {
        if (x >= 1.0) return 1.0;
        return eps * x + (1.0 - eps) * or_beta_star(x);
    }
    double ax = alpha * x;
    double num = eps * ax + (1.0 - eps) * or_beta_star(ax);
    double den = eps * alpha + (1.0 - eps) * or_beta_star(alpha);
    return num / den;
}

/* The other bucket assignment functions of Figure 3a, for the ablations:
 * beta_* itself (eps = 0); PTHash's skewed split, which sends the keys with
 * normalised hash below 0.6 (60 %) to the first 30 % of the buckets and the
 * rest to the other 70 %; and the uniform gamma(x) = x of CHD.  For alpha < 1
 * every one is rescaled as gamma(alpha x) / gamma(alpha) (Appendix B). */
static double gamma_base(double x, double eps, uint32_t fn) {
    if (x >= 1.0) return 1.0;
    switch (fn) {
        case OR_BUCKET_BETA_STAR: return or_beta_star(x);
        case OR_BUCKET_SKEWED: return x < 0.6 ? 0.5 * x : 0.3 + 1.75 * (x - 0.6);
        case OR_BUCKET_UNIFORM: return x;
        default: return eps * x + (1.0 - eps) * or_beta_star(x);
    }
}

double or_gamma_fn(double x, double eps, double alpha, uint32_t fn) {
    if (fn == OR_BUCKET_OPTIMIZED) return or_gamma(x, eps, alpha);
    if (alpha == 1.0) return gamma_base(x, eps, fn);
    return gamma_base(alpha * x, eps, fn) / gamma_base(alpha, eps, fn);
}

/* Appendix C: gamma tabulated at 2048 points, here as 32-bit fixed point:
 * table[k] = round(gamma(k / 2048) * 2^32), k = 0..2048. */
void or_bucket_table_fn(double lambda, double alpha, uint32_t P, uint32_t fn, uint64_t* table) {
    double eps = or_epsilon(lambda, P);
    for (int k = 0; k <= OR_TABLE_POINTS; k++) {
        double x = (double)k / (double)OR_TABLE_POINTS;
        double g = or_gamma_fn(x, eps, alpha, fn);
        double v = g * 4294967296.0;
        long long r = llround(v);
        if (r < 0) r = 0;
        if (r > 4294967296LL) r = 4294967296LL;
        table[k] = (uint64_t)r;
    }
}

void or_bucket_table(double lambda, double alpha, uint32_t P, uint64_t* table) {
    or_bucket_table_fn(lambda, alpha, P, OR_BUCKET_OPTIMIZED, table);
}

/* Section 4.1: B = P / lambda buckets per partition (rounded up, at least 1) */
uint32_t or_num_buckets(double lambda, uint32_t P) {
    double b = ceil((double)P / lambda);
    if (b < 1.0) b = 1.0;
    return (uint32_t)b;
}

/* Section 4: number of partitions for expected partition size P */
uint64_t or_num_partitions(uint64_t n, uint32_t P) {
    uint64_t np = (n + P - 1) / P;
    return np ? np : 1;
}

/* Section 3.1: the key with normalised hash x goes to bucket ceil(gamma(x) B)
 * (1-based).  Here 0-based, floor(gamma(x) B), with gamma read from the table by
 * linear interpolation in integer arithmetic: the top 11 bits of x select the
 * interval and the next 32 bits are the fraction inside it. */
uint32_t or_bucket(uint64_t x, const uint64_t* table, uint32_t B) {
    uint64_t k = x >> 53;
    uint64_t f = (x >> 21) & 0xFFFFFFFFULL;
    uint64_t lo = table[k], hi = table[k + 1];
    uint64_t v = lo + (((hi - lo) * f) >> 32);
    uint64_t b = (v * (uint64_t)B) >> 32;
    if (b > B - 1) b = B - 1;
    return (uint32_t)b;
}

/* Section 5: keys are first reduced to 64-bit master hash codes.  For 64-bit
 * keys: hk = mix64(key xor mix64(seed xor C_SEED)); a bijection, so distinct keys
 * never share hk. */
uint64_t or_key_hash(uint64_t key, uint64_t seed) {
    return or_mix64(key ^ or_mix64(seed ^ C_SEED));
}

void or_key_hash_array(const uint64_t* keys, uint64_t n, uint64_t seed, uint64_t* out) {
    for (uint64_t i = 0; i < n; i++) out[i] = or_key_hash(keys[i], seed);
}

uint64_t or_bucket_hash(uint64_t hk) { return or_mix64(hk ^ C_BUCKET); }

/* Section 4 ("Hash Function"): h(x, s) in [0, m) */
uint64_t or_position_hash(uint64_t hk, uint64_t s, uint64_t m) {
    return or_mulhi64(or_mix64(hk ^ or_mix64(s ^ C_PILOT)), m);
}

/* table size of a partition: m_j = n_j for alpha = 1, else ceil(n_j / alpha) */
uint64_t or_table_size(uint64_t n_j, double alpha) {
    if (alpha == 1.0) return n_j;
    uint64_t m = (uint64_t)ceil((double)n_j / alpha);
    return m < n_j ? n_j : m;
}

/* 64-bit string hash: XXH64 (Collet, xxHash specification, XXH64 algorithm),
 * the initial hash the paper names in Section 5. */
#define XP1 0x9E3779B185EBCA87ULL
#define XP2 0xC2B2AE3D27D4EB4FULL
#define XP3 0x165667B19E3779F9ULL
#define XP4 0x85EBCA77C2B2AE63ULL
#define XP5 0x27D4EB2F165667C5ULL
static uint64_t rotl64(uint64_t v, int r) { return (v << r) | (v >> (64 - r)); }
static uint64_t rd64(const uint8_t* p) {
    uint64_t v = 0;
    for (int i = 7; i >= 0; i--) v = (v << 8) | p[i];
    return v;
}
static uint64_t rd32(const uint8_t* p) {
    uint64_t v = 0;
    for (int i = 3; i >= 0; i--) v = (v << 8) | p[i];
    return v;
}
static uint64_t xround(uint64_t acc, uint64_t lane) {
    acc += lane * XP2;
    acc = rotl64(acc, 31);
    return acc * XP1;
}
static uint64_t xmerge(uint64_t acc, uint64_t v) {
    acc ^= xround(0, v);
    return acc * XP1 + XP4;
}
uint64_t or_string_hash(const uint8_t* p, uint64_t len, uint64_t seed) {
    uint64_t i = 0, acc;
    if (len >= 32) {
        uint64_t v1 = seed + XP1 + XP2, v2 = seed + XP2, v3 = seed, v4 = seed - XP1;
        for (; i + 32 <= len; i += 32) {
            v1 = xround(v1, rd64(p + i));
            v2 = xround(v2, rd64(p + i + 8));
            v3 = xround(v3, rd64(p + i + 16));
            v4 = xround(v4, rd64(p + i + 24));
        }
        acc = rotl64(v1, 1) + rotl64(v2, 7) + rotl64(v3, 12) + rotl64(v4, 18);
        acc = xmerge(acc, v1);
        acc = xmerge(acc, v2);
        acc = xmerge(acc, v3);
        acc = xmerge(acc, v4);
    } else {
        acc = seed + XP5;
    }
    acc += len;
    for (; i + 8 <= len; i += 8) {
        acc ^= xround(0, rd64(p + i));
        acc = rotl64(acc, 27) * XP1 + XP4;
    }
    if (i + 4 <= len) {
        acc ^= rd32(p + i) * XP1;
        acc = rotl64(acc, 23) * XP2 + XP3;
        i += 4;
    }
    for (; i < len; i++) {
        acc ^= (uint64_t)p[i] * XP5;
        acc = rotl64(acc, 11) * XP1;
    }
    acc ^= acc >> 33;
    acc *= XP2;
    acc ^= acc >> 29;
    acc *= XP3;
    acc ^= acc >> 32;
    return acc;
}

/* strings i = 0..n-1 occupy bytes[offsets[i] .. offsets[i+1]) */
void or_string_hash_array(const uint8_t* bytes, const uint64_t* offsets, uint64_t n, uint64_t seed,
                          uint64_t* out) {
    for (uint64_t i = 0; i < n; i++)
        out[i] = or_string_hash(bytes + offsets[i], offsets[i + 1] - offsets[i], seed);
}

/* ------------------------------------------------------------------------- */
/* plain bit packing: value v of width w at bit offset o, little-endian words */
/* ------------------------------------------------------------------------- */
static uint64_t packed_words(uint64_t nbits) { return (nbits + 63) / 64 + 1; }

static void put_bits(uint64_t* words, uint64_t o, uint64_t v, uint32_t w) {
    for (uint32_t t = 0; t < w; t++)
        if ((v >> t) & 1ULL) words[(o + t) >> 6] |= 1ULL << ((o + t) & 63);
}

static uint64_t get_bits(const uint64_t* words, uint64_t o, uint32_t w) {
    uint64_t v = 0;
    for (uint32_t t = 0; t < w; t++)
        if ((words[(o + t) >> 6] >> ((o + t) & 63)) & 1ULL) v |= 1ULL << t;
    return v;
}

/* ------------------------------------------------------------------------- */
/* the structure                                                               */
/* ------------------------------------------------------------------------- */
struct or_mphf {
    or_params prm;
    uint64_t n, M, NP;
    uint32_t B;
    double eps;
    uint64_t table[OR_TABLE_POINTS + 1];
    uint64_t* part_size;  /* n_j  [NP] */
    uint64_t* table_size; /* m_j  [NP] */
    uint64_t* T;          /* [NP + 1] */
    uint32_t* pilots;     /* [B * NP], pilots[b * NP + j] (interleaved order) */
    /* partition offsets, Section 4 */
    uint64_t off_Q;
    int64_t off_dmin;
    uint32_t off_w;
    uint64_t off_nbits;
    uint64_t* off_words;
    /* IC-C */
    uint32_t* col_w;
    uint64_t* col_base;
    uint64_t pil_nbits;
    uint64_t* pil_words;
    /* IC-D */
    uint32_t* col_rw;
    uint64_t* col_rbase;
    uint32_t* col_dw;
    uint64_t* col_dbase;
    uint64_t* col_K;
    uint64_t rank_nbits, dict_nbits;
    uint64_t* rank_words;
    uint64_t* dict_words;
    /* IC-R */
    uint32_t* col_l;      /* Rice parameter: low bits per value */
    uint64_t* col_lbase;  /* bit offset of the column's low parts */
    uint64_t* col_hbase;  /* bit offset of the column's unary parts */
    uint64_t* col_H;      /* bits of the column's unary parts */
    uint64_t rlow_nbits, rhigh_nbits, rsamp_count;
    uint64_t* rice_low;
    uint64_t* rice_high;
    uint32_t* rice_samples;
    /* remap of slots >= n (alpha < 1) */
    uint64_t ef_N, ef_U;
    uint32_t ef_l;
    uint64_t* fs;       /* raw remap targets [ef_N] */
    uint64_t ef_low_nbits, ef_high_nbits, ef_nsamples;
    uint64_t* ef_low;
    uint64_t* ef_high;
    uint64_t* ef_samples;
    /* space */
    uint64_t bits_header, bits_offsets, bits_pilots, bits_remap, bits_total;
    /* work statistics */
    uint64_t stat_candidates, stat_key_tests, stat_s_tries;
};

static int check_params(uint64_t n, const or_params* p) {
    if (!p || n == 0) return OR_ERR_INVALID_ARG;
    if (!(p->lambda > 0.0) || !isfinite(p->lambda)) return OR_ERR_INVALID_ARG;
    if (!(p->alpha > 0.0) || p->alpha > 1.0) return OR_ERR_INVALID_ARG;
    if (p->partition_size == 0) return OR_ERR_INVALID_ARG;
    if ((double)p->partition_size < p->lambda) return OR_ERR_INVALID_ARG; /* P below one average bucket */
    if (p->encoder > OR_ENC_MONO_EF || p->pilot_mode > OR_PILOT_XOR) return OR_ERR_INVALID_ARG;
    if (p->bucket_fn > OR_BUCKET_UNIFORM) return OR_ERR_INVALID_ARG;
    return OR_OK;
}

/* --- Section 3 / Section 4: search of one partition ----------------------- */

typedef struct {
    uint32_t b;
    uint32_t size;
} bucket_ref;

/* Section 1 and Proposition (largest-to-smallest): non-increasing size; Section 5
 * ("Further Remarks"): ties by increasing expected size.  Expected size
 * decreases in the bucket index (Intuition 1 (iii)), so ties go by index
 * descending. */
static int bucket_order_cmp(const void* a, const void* b) {
    const bucket_ref* x = (const bucket_ref*)a;
    const bucket_ref* y = (const bucket_ref*)b;
    if (x->size != y->size) return x->size > y->size ? -1 : 1;
    if (x->b != y->b) return x->b > y->b ? -1 : 1;
    return 0;
}

typedef struct {
    uint64_t candidates, key_tests, s_tries;
} search_stats;

/* Searches one partition: hk[0..nj) are its keys, m its table size.  Writes
 * pilot[b] for every bucket b (0 for empty buckets) and the final table
 * occupancy to taken[0..m).  Returns an OR_* status. */
static int search_partition(const uint64_t* hk, uint64_t nj, uint64_t m, const uint64_t* table,
                            uint32_t B, const or_params* prm, uint32_t* pilot, uint8_t* taken,
                            search_stats* st) {
    for (uint32_t b = 0; b < B; b++) pilot[b] = 0;
    for (uint64_t t = 0; t < m; t++) taken[t] = 0;
    if (nj == 0) return OR_OK;
    /* seeds s < s_lim: the requested limit (0: none), and never past the
     * largest s whose pilots s m + d all fit 32 bits in this partition */
    const uint64_t s_cap = 0xFFFFFFFFULL / m;
    const uint64_t s_lim = (prm->s_max && prm->s_max < s_cap) ? prm->s_max : s_cap;

    /* Section 3.1: bucket of every key */
    uint32_t* bk = (uint32_t*)malloc(nj * sizeof(uint32_t));
    uint32_t* cnt = (uint32_t*)calloc(B + 1, sizeof(uint32_t));
    uint64_t* sorted = (uint64_t*)malloc(nj * sizeof(uint64_t));
    bucket_ref* order = (bucket_ref*)malloc(B * sizeof(bucket_ref));
    uint64_t* hpos = (uint64_t*)malloc(nj * sizeof(uint64_t));
    uint32_t* mark = (uint32_t*)calloc(m, sizeof(uint32_t));
    if (!bk || !cnt || !sorted || !order || !hpos || !mark) {
        free(bk); free(cnt); free(sorted); free(order); free(hpos); free(mark);
        return OR_ERR_OOM;
    }
    int status = OR_OK;
    for (uint64_t i = 0; i < nj; i++) {
        bk[i] = or_bucket(or_bucket_hash(hk[i]), table, B);
        cnt[bk[i] + 1]++;
    }
    /* group keys by bucket (start offsets in cnt) */
    for (uint32_t b = 0; b < B; b++) cnt[b + 1] += cnt[b];
    {
        uint32_t* fill = (uint32_t*)malloc(B * sizeof(uint32_t));
        memcpy(fill, cnt, B * sizeof(uint32_t));
        for (uint64_t i = 0; i < nj; i++) sorted[fill[bk[i]]++] = hk[i];
        free(fill);
    }
    uint32_t nb = 0;
    for (uint32_t b = 0; b < B; b++) {
        uint32_t sz = cnt[b + 1] - cnt[b];
        if (sz == 0) continue; /* empty bucket: pilot 0, never searched */
        if (sz > OR_MAX_BUCKET) status = OR_ERR_SEARCH_LIMIT;
        order[nb].b = b;
        order[nb].size = sz;
        nb++;
    }
    if (status != OR_OK) goto done;
    qsort(order, nb, sizeof(bucket_ref), bucket_order_cmp);

    uint32_t stamp = 0;
    for (uint32_t r = 0; r < nb && status == OR_OK; r++) {
        const uint64_t* keys = sorted + cnt[order[r].b];
        uint32_t k = order[r].size;
        int found = 0;
        uint64_t p = 0;
        if (prm->pilot_mode == OR_PILOT_ADDITIVE) {
            /* Section 4 "Hash Function": p = s m + d, d in [0, m); for each s
             * compute h(x, s) for all keys of the bucket, then try d = 0, 1, ...
             * until all (h + d) mod m are free; if none, increment s. */
            for (uint64_t s = 0; s < s_lim && !found; s++) {
                st->s_tries++;
                for (uint32_t i = 0; i < k; i++) hpos[i] = or_position_hash(keys[i], s, m);
                /* If two keys share h(x, s), every displacement d moves them
                 * together, so no d in [0, m) can work for this s.  Skipping it
                 * gives the same pilot as trying each d. */
                int self = 0;
                for (uint32_t i = 0; i < k && !self; i++)
                    for (uint32_t i2 = i + 1; i2 < k; i2++)
                        if (hpos[i] == hpos[i2]) {
                            self = 1;
                            break;
                        }
                if (self) continue;
                for (uint64_t d = 0; d < m; d++) {
                    int ok = 1;
                    stamp++;
                    st->candidates++;
                    for (uint32_t i = 0; i < k; i++) {
                        uint64_t pos = (hpos[i] + d) % m;
                        st->key_tests++;
                        if (taken[pos] || mark[pos] == stamp) {
                            ok = 0;
                            break;
                        }
                        mark[pos] = stamp;
                    }
                    if (ok) {
                        p = s * m + d;
                        found = 1;
                        break;
                    }
                }
            }
        } else {
            /* PTHash's XOR form (Section 4 "Hash Function"): position
             * h(x xor h(p)) reduced onto [0, m), pilots p = 0, 1, 2, ... */
            uint64_t limit = s_lim * m;
            for (uint64_t q = 0; q < limit; q++) {
                int ok = 1;
                stamp++;
                st->candidates++;
                for (uint32_t i = 0; i < k; i++) {
                    uint64_t pos = or_position_hash(keys[i], q, m);
                    st->key_tests++;
                    if (taken[pos] || mark[pos] == stamp) {
                        ok = 0;
                        break;
                    }
                    mark[pos] = stamp;
                }
                if (ok) {
                    p = q;
                    found = 1;
                    break;
                }
            }
        }
        if (!found) {
            status = OR_ERR_SEARCH_LIMIT;
            break;
        }
        /* place the bucket */
        for (uint32_t i = 0; i < k; i++) {
            uint64_t pos;
            if (prm->pilot_mode == OR_PILOT_ADDITIVE)
                pos = (or_position_hash(keys[i], p / m, m) + p) % m;
            else
                pos = or_position_hash(keys[i], p, m);
            taken[pos] = 1;
        }
        pilot[order[r].b] = (uint32_t)p;
    }
done:
    free(bk); free(cnt); free(sorted); free(order); free(hpos); free(mark);
    return status;
}

/* keys of every partition, grouped (counting sort by partition id) */
static int group_by_partition(const uint64_t* hk, uint64_t n, uint64_t NP, uint64_t** start_out,
                              uint64_t** grouped_out) {
    uint64_t* start = (uint64_t*)calloc(NP + 1, sizeof(uint64_t));
    uint64_t* grouped = (uint64_t*)malloc(n * sizeof(uint64_t));
    if (!start || !grouped) {
        free(start); free(grouped);
        return OR_ERR_OOM;
    }
    for (uint64_t i = 0; i < n; i++) start[or_mulhi64(hk[i], NP) + 1]++;
    for (uint64_t j = 0; j < NP; j++) start[j + 1] += start[j];
    uint64_t* fill = (uint64_t*)malloc(NP * sizeof(uint64_t));
    if (!fill) {
        free(start); free(grouped);
        return OR_ERR_OOM;
    }
    memcpy(fill, start, NP * sizeof(uint64_t));
    for (uint64_t i = 0; i < n; i++) grouped[fill[or_mulhi64(hk[i], NP)]++] = hk[i];
    free(fill);
    *start_out = start;
    *grouped_out = grouped;
    return OR_OK;
}

static int cmp_u64(const void* a, const void* b) {
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}
static int cmp_u32(const void* a, const void* b) {
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* any two equal master hashes make the search impossible */
static int has_duplicates(const uint64_t* hk, uint64_t n) {
    uint64_t* c = (uint64_t*)malloc(n * sizeof(uint64_t));
    if (!c) return -1;
    memcpy(c, hk, n * sizeof(uint64_t));
    qsort(c, n, sizeof(uint64_t), cmp_u64);
    int dup = 0;
    for (uint64_t i = 1; i < n; i++)
        if (c[i] == c[i - 1]) {
            dup = 1;
            break;
        }
    free(c);
    return dup;
}

/* ---- Section 4: offsets stored as difference to their expectation ---- */
static void encode_offsets(or_mphf* h) {
    uint64_t NP = h->NP;
    /* expectation E_j = floor(j * Q / 2^32), Q = floor(M 2^32 / NP) */
    h->off_Q = (uint64_t)((((unsigned __int128)h->M) << 32) / NP);
    int64_t* D = (int64_t*)malloc((NP + 1) * sizeof(int64_t));
    int64_t dmin = 0, dmax = 0;
    for (uint64_t j = 0; j <= NP; j++) {
        uint64_t E = (uint64_t)(((unsigned __int128)j * h->off_Q) >> 32);
        D[j] = (int64_t)(h->T[j] - E);
        if (j == 0 || D[j] < dmin) dmin = D[j];
        if (j == 0 || D[j] > dmax) dmax = D[j];
    }
    h->off_dmin = dmin;
    h->off_w = or_bitlen((uint64_t)(dmax - dmin));
    h->off_nbits = (NP + 1) * (uint64_t)h->off_w;
    h->off_words = (uint64_t*)calloc(packed_words(h->off_nbits), sizeof(uint64_t));
    for (uint64_t j = 0; j <= NP; j++)
        put_bits(h->off_words, j * h->off_w, (uint64_t)(D[j] - dmin), h->off_w);
    free(D);
}

static uint64_t decode_offset(const or_mphf* h, uint64_t j) {
    uint64_t E = (uint64_t)(((unsigned __int128)j * h->off_Q) >> 32);
    uint64_t v = get_bits(h->off_words, j * h->off_w, h->off_w);
    return E + (uint64_t)h->off_dmin + v;
}

/* ---- Section 4.1: interleaved coding, encoder b = bucket b of all partitions ---- */
static void encode_compact(or_mphf* h) {
    uint32_t B = h->B;
    uint64_t NP = h->NP;
    h->col_w = (uint32_t*)calloc(B, sizeof(uint32_t));
    h->col_base = (uint64_t*)calloc(B, sizeof(uint64_t));
    uint64_t base = 0;
    for (uint32_t b = 0; b < B; b++) {
        uint32_t mx = 0;
        for (uint64_t j = 0; j < NP; j++)
            if (h->pilots[(uint64_t)b * NP + j] > mx) mx = h->pilots[(uint64_t)b * NP + j];
        h->col_w[b] = or_bitlen(mx); /* Compact: width of the largest value */
        h->col_base[b] = base;
        base += NP * (uint64_t)h->col_w[b];
    }
    h->pil_nbits = base;
    h->pil_words = (uint64_t*)calloc(packed_words(base), sizeof(uint64_t));
    for (uint32_t b = 0; b < B; b++)
        for (uint64_t j = 0; j < NP; j++)
            put_bits(h->pil_words, h->col_base[b] + j * h->col_w[b], h->pilots[(uint64_t)b * NP + j],
                     h->col_w[b]);
}

static void encode_dictionary(or_mphf* h) {
    uint32_t B = h->B;
    uint64_t NP = h->NP;
    h->col_rw = (uint32_t*)calloc(B, sizeof(uint32_t));
    h->col_dw = (uint32_t*)calloc(B, sizeof(uint32_t));
    h->col_rbase = (uint64_t*)calloc(B, sizeof(uint64_t));
    h->col_dbase = (uint64_t*)calloc(B, sizeof(uint64_t));
    h->col_K = (uint64_t*)calloc(B, sizeof(uint64_t));
    uint32_t** dicts = (uint32_t**)calloc(B, sizeof(uint32_t*));
    uint32_t* tmp = (uint32_t*)malloc(NP * sizeof(uint32_t));
    uint64_t rbase = 0, dbase = 0;
    for (uint32_t b = 0; b < B; b++) {
        memcpy(tmp, h->pilots + (uint64_t)b * NP, NP * sizeof(uint32_t));
        qsort(tmp, NP, sizeof(uint32_t), cmp_u32);
        uint64_t K = 0;
        for (uint64_t j = 0; j < NP; j++)
            if (j == 0 || tmp[j] != tmp[j - 1]) tmp[K++] = tmp[j];
        dicts[b] = (uint32_t*)malloc(K * sizeof(uint32_t));
        memcpy(dicts[b], tmp, K * sizeof(uint32_t));
        h->col_K[b] = K;
        h->col_rw[b] = or_bitlen(K - 1);
        h->col_dw[b] = or_bitlen(dicts[b][K - 1]);
        h->col_rbase[b] = rbase;
        h->col_dbase[b] = dbase;
        rbase += NP * (uint64_t)h->col_rw[b];
        dbase += K * (uint64_t)h->col_dw[b];
    }
    h->rank_nbits = rbase;
    h->dict_nbits = dbase;
    h->rank_words = (uint64_t*)calloc(packed_words(rbase), sizeof(uint64_t));
    h->dict_words = (uint64_t*)calloc(packed_words(dbase), sizeof(uint64_t));
    for (uint32_t b = 0; b < B; b++) {
        for (uint64_t r = 0; r < h->col_K[b]; r++)
            put_bits(h->dict_words, h->col_dbase[b] + r * h->col_dw[b], dicts[b][r], h->col_dw[b]);
        for (uint64_t j = 0; j < NP; j++) {
            uint32_t v = h->pilots[(uint64_t)b * NP + j];
            /* rank of v in the sorted dictionary (binary search) */
            uint64_t lo = 0, hi = h->col_K[b];
            while (hi - lo > 1) {
                uint64_t mid = (lo + hi) / 2;
                if (dicts[b][mid] <= v) lo = mid; else hi = mid;
            }
            put_bits(h->rank_words, h->col_rbase[b] + j * h->col_rw[b], lo, h->col_rw[b]);
        }
        free(dicts[b]);
    }
    free(dicts);
    free(tmp);
}

/* Golomb-Rice (Section 4.1 names it with Kiely's parameter choice).  For a
 * geometric source with parameter theta, the Rice parameter with the smallest
 * expected code length is max(0, 1 + floor(log2(log(phi - 1) / log(theta)))),
 * phi the golden ratio (Kiely 2004).  The column's values are modelled as
 * geometric with the column's mean mu: theta = mu / (mu + 1). */
uint32_t or_rice_param(uint64_t sum, uint64_t count) {
    if (sum == 0 || count == 0) return 0;
    double mu = (double)sum / (double)count;
    double theta = mu / (mu + 1.0);
    double ratio = log((sqrt(5.0) - 1.0) / 2.0) / log(theta);
    double k = 1.0 + floor(log2(ratio));
    if (!(k > 0.0)) return 0;
    if (k > 31.0) return 31;
    return (uint32_t)k;
}

/* Column b: the low l bits of each value packed at width l; the rest in unary,
 * value j setting bit j + sum_{i <= j} (v_i >> l) of the column's unary bits;
 * the position of that bit for every 64th value kept as a select sample. */
static void encode_rice(or_mphf* h) {
    uint32_t B = h->B;
    uint64_t NP = h->NP, ns = (NP + 63) / 64;
    h->col_l = (uint32_t*)calloc(B, sizeof(uint32_t));
    h->col_lbase = (uint64_t*)calloc(B, sizeof(uint64_t));
    h->col_hbase = (uint64_t*)calloc(B, sizeof(uint64_t));
    h->col_H = (uint64_t*)calloc(B, sizeof(uint64_t));
    uint64_t lbase = 0, hbase = 0;
    for (uint32_t b = 0; b < B; b++) {
        uint64_t sum = 0;
        for (uint64_t j = 0; j < NP; j++) sum += h->pilots[(uint64_t)b * NP + j];
        uint32_t l = or_rice_param(sum, NP);
        uint64_t H = NP;
        for (uint64_t j = 0; j < NP; j++) H += h->pilots[(uint64_t)b * NP + j] >> l;
        h->col_l[b] = l;
        h->col_lbase[b] = lbase;
        h->col_hbase[b] = hbase;
        h->col_H[b] = H;
        lbase += NP * (uint64_t)l;
        hbase += H;
    }
    h->rlow_nbits = lbase;
    h->rhigh_nbits = hbase;
    h->rsamp_count = (uint64_t)B * ns;
    h->rice_low = (uint64_t*)calloc(packed_words(lbase), sizeof(uint64_t));
    h->rice_high = (uint64_t*)calloc(packed_words(hbase), sizeof(uint64_t));
    h->rice_samples = (uint32_t*)calloc(h->rsamp_count ? h->rsamp_count : 1, sizeof(uint32_t));
    for (uint32_t b = 0; b < B; b++) {
        uint32_t l = h->col_l[b];
        uint64_t acc = 0;
        for (uint64_t j = 0; j < NP; j++) {
            uint32_t v = h->pilots[(uint64_t)b * NP + j];
            put_bits(h->rice_low, h->col_lbase[b] + j * l, l ? (v & ((1ULL << l) - 1)) : 0, l);
            acc += v >> l;
            uint64_t pos = j + acc; /* the j-th one of the column */
            put_bits(h->rice_high, h->col_hbase[b] + pos, 1, 1);
            if (j % 64 == 0) h->rice_samples[(uint64_t)b * ns + j / 64] = (uint32_t)pos;
        }
    }
}

/* IC-EF: column b stores the inclusive prefix sums E_j = v_0 + ... + v_j of its
 * values with Elias-Fano over the universe [0, E_last]: with N = N_P values and
 * U = E_last + 1, l = floor(log2(U / N)) (0 when U < N) low bits of E_j packed
 * at width l, and in the high part bit j + (E_j >> l) set (N + (E_last >> l) + 1
 * bits); the position of every 64th one is a select sample.  A value is
 * E_j - E_{j-1}.  The arrays and samples reuse the IC-R slots. */
static uint32_t ef_low_bits(uint64_t last, uint64_t count) {
    uint64_t U = last + 1;
    if (U < count || count == 0) return 0;
    return or_bitlen(U / count) - 1;
}

static void encode_ef_columns(or_mphf* h) {
    uint32_t B = h->B;
    uint64_t NP = h->NP, ns = (NP + 63) / 64;
    h->col_l = (uint32_t*)calloc(B, sizeof(uint32_t));
    h->col_lbase = (uint64_t*)calloc(B, sizeof(uint64_t));
    h->col_hbase = (uint64_t*)calloc(B, sizeof(uint64_t));
    h->col_H = (uint64_t*)calloc(B, sizeof(uint64_t));
    uint64_t lbase = 0, hbase = 0;
    for (uint32_t b = 0; b < B; b++) {
        uint64_t last = 0;
        for (uint64_t j = 0; j < NP; j++) last += h->pilots[(uint64_t)b * NP + j];
        uint32_t l = ef_low_bits(last, NP);
        h->col_l[b] = l;
        h->col_lbase[b] = lbase;
        h->col_hbase[b] = hbase;
        h->col_H[b] = NP + (last >> l) + 1;
        lbase += NP * (uint64_t)l;
        hbase += h->col_H[b];
    }
    h->rlow_nbits = lbase;
    h->rhigh_nbits = hbase;
    h->rsamp_count = (uint64_t)B * ns;
    h->rice_low = (uint64_t*)calloc(packed_words(lbase), sizeof(uint64_t));
    h->rice_high = (uint64_t*)calloc(packed_words(hbase), sizeof(uint64_t));
    h->rice_samples = (uint32_t*)calloc(h->rsamp_count ? h->rsamp_count : 1, sizeof(uint32_t));
    for (uint32_t b = 0; b < B; b++) {
        uint32_t l = h->col_l[b];
        uint64_t E = 0;
        for (uint64_t j = 0; j < NP; j++) {
            E += h->pilots[(uint64_t)b * NP + j];
            put_bits(h->rice_low, h->col_lbase[b] + j * l, l ? (E & ((1ULL << l) - 1)) : 0, l);
            uint64_t pos = j + (E >> l);
            put_bits(h->rice_high, h->col_hbase[b] + pos, 1, 1);
            if (j % 64 == 0) h->rice_samples[(uint64_t)b * ns + j / 64] = (uint32_t)pos;
        }
    }
}

/* Section 4.1: interleaving lets each column use its own encoder.  IC-CR puts
 * the first c = min(compact_columns, B) columns (the largest buckets, read most
 * often) in Compact form, width = bit length of the column's largest pilot, and
 * the others in Golomb-Rice form as IC-R.  The Compact values and the Rice low
 * parts share one array in column order; unary bits and select samples exist
 * for the Rice columns only (column b >= c has sample column b - c). */
static void encode_mixture(or_mphf* h) {
    uint32_t B = h->B;
    uint64_t NP = h->NP, ns = (NP + 63) / 64;
    uint32_t c = h->prm.compact_columns < B ? h->prm.compact_columns : B;
    h->col_l = (uint32_t*)calloc(B, sizeof(uint32_t));
    h->col_lbase = (uint64_t*)calloc(B, sizeof(uint64_t));
    h->col_hbase = (uint64_t*)calloc(B, sizeof(uint64_t));
    h->col_H = (uint64_t*)calloc(B, sizeof(uint64_t));
    uint64_t lbase = 0, hbase = 0;
    for (uint32_t b = 0; b < B; b++) {
        const uint32_t* col = h->pilots + (uint64_t)b * NP;
        uint32_t l;
        uint64_t H = 0;
        if (b < c) {
            uint32_t mx = 0;
            for (uint64_t j = 0; j < NP; j++)
                if (col[j] > mx) mx = col[j];
            l = or_bitlen(mx);
        } else {
            uint64_t sum = 0;
            for (uint64_t j = 0; j < NP; j++) sum += col[j];
            l = or_rice_param(sum, NP);
            H = NP;
            for (uint64_t j = 0; j < NP; j++) H += col[j] >> l;
        }
        h->col_l[b] = l;
        h->col_lbase[b] = lbase;
        h->col_hbase[b] = hbase;
        h->col_H[b] = H;
        lbase += NP * (uint64_t)l;
        hbase += H;
    }
    h->rlow_nbits = lbase;
    h->rhigh_nbits = hbase;
    h->rsamp_count = (uint64_t)(B - c) * ns;
    h->rice_low = (uint64_t*)calloc(packed_words(lbase), sizeof(uint64_t));
    h->rice_high = (uint64_t*)calloc(packed_words(hbase), sizeof(uint64_t));
    h->rice_samples = (uint32_t*)calloc(h->rsamp_count ? h->rsamp_count : 1, sizeof(uint32_t));
    for (uint32_t b = 0; b < B; b++) {
        const uint32_t* col = h->pilots + (uint64_t)b * NP;
        uint32_t l = h->col_l[b];
        uint64_t acc = 0;
        for (uint64_t j = 0; j < NP; j++) {
            uint32_t v = col[j];
            put_bits(h->rice_low, h->col_lbase[b] + j * l, l ? (v & ((1ULL << l) - 1)) : 0, l);
            if (b < c) continue;
            acc += v >> l;
            uint64_t pos = j + acc;
            put_bits(h->rice_high, h->col_hbase[b] + pos, 1, 1);
            if (j % 64 == 0) h->rice_samples[(uint64_t)(b - c) * ns + j / 64] = (uint32_t)pos;
        }
    }
}

/* the select-sample column of column b (IC-CR: Rice columns only) */
static uint64_t sample_column(const or_mphf* h, uint32_t b) {
    if (h->prm.encoder != OR_ENC_IC_CR) return b;
    uint32_t c = h->prm.compact_columns < h->B ? h->prm.compact_columns : h->B;
    return b - c;
}

/* position (relative to the column) of the t-th one of column b's unary bits */
static uint64_t rice_select(const or_mphf* h, uint32_t b, uint64_t t) {
    uint64_t ns = (h->NP + 63) / 64;
    uint64_t pos = h->rice_samples[sample_column(h, b) * ns + t / 64];
    uint64_t left = t % 64; /* ones still to pass */
    while (left) {
        pos++;
        if (get_bits(h->rice_high, h->col_hbase[b] + pos, 1)) left--;
    }
    return pos;
}

static uint32_t decode_rice(const or_mphf* h, uint32_t b, uint64_t j) {
    uint64_t c = rice_select(h, b, j);
    uint64_t q = (j == 0) ? c : c - rice_select(h, b, j - 1) - 1;
    uint32_t l = h->col_l[b];
    return (uint32_t)((q << l) | get_bits(h->rice_low, h->col_lbase[b] + j * l, l));
}

/* IC-EF: E_j from its high part (select) and its low bits */
static uint64_t ef_prefix(const or_mphf* h, uint32_t b, uint64_t j) {
    uint32_t l = h->col_l[b];
    uint64_t pos = rice_select(h, b, j);
    return ((pos - j) << l) | get_bits(h->rice_low, h->col_lbase[b] + j * l, l);
}

static uint32_t decode_ef_column(const or_mphf* h, uint32_t b, uint64_t j) {
    uint64_t e = ef_prefix(h, b, j);
    return (uint32_t)(j == 0 ? e : e - ef_prefix(h, b, j - 1));
}

static uint32_t decode_column(const or_mphf* h, uint32_t enc, uint32_t b, uint64_t j) {
    if (enc == OR_ENC_IC_C)
        return (uint32_t)get_bits(h->pil_words, h->col_base[b] + j * h->col_w[b], h->col_w[b]);
    if (enc == OR_ENC_IC_R) return decode_rice(h, b, j);
    if (enc == OR_ENC_IC_EF) return decode_ef_column(h, b, j);
    if (enc == OR_ENC_IC_CR) {
        uint32_t c = h->prm.compact_columns < h->B ? h->prm.compact_columns : h->B;
        if (b < c) return (uint32_t)get_bits(h->rice_low, h->col_lbase[b] + j * h->col_l[b], h->col_l[b]);
        return decode_rice(h, b, j);
    }
    uint64_t r = get_bits(h->rank_words, h->col_rbase[b] + j * h->col_rw[b], h->col_rw[b]);
    return (uint32_t)get_bits(h->dict_words, h->col_dbase[b] + r * h->col_dw[b], h->col_dw[b]);
}

/* a mono encoder is its column encoder over the single column of all pilots:
 * pilot (b, j) is value b N_P + j of column 0 (column 0 decodes the same whatever
 * N_P is, as only the column index scales by it) */
static uint32_t decode_pilot(const or_mphf* h, uint32_t b, uint64_t j) {
    if (h->prm.encoder >= OR_ENC_MONO_C)
        return decode_column(h, h->prm.encoder - OR_ENC_MONO_C, 0, (uint64_t)b * h->NP + j);
    return decode_column(h, h->prm.encoder, b, j);
}

/* ---- Section 5 (PTHash non-minimal trick): slots q in [n, M) are remapped
 * onto the free slots below n.  F = free slots < n in increasing order,
 * rank(q) = number of occupied slots in [n, q); fs[q - n] = F[min(rank, |F|-1)].
 * A slot q >= n that no key occupies repeats the value of the next occupied
 * slot, so fs is non-decreasing and Elias-Fano applies. ---- */
static void build_remap(or_mphf* h, const uint8_t* taken_global) {
    uint64_t n = h->n, M = h->M;
    h->ef_N = M - n;
    h->ef_U = n;
    if (h->ef_N == 0) return;
    uint64_t nF = 0;
    for (uint64_t q = 0; q < n; q++)
        if (!taken_global[q]) nF++;
    uint64_t* F = (uint64_t*)malloc((nF ? nF : 1) * sizeof(uint64_t));
    nF = 0;
    for (uint64_t q = 0; q < n; q++)
        if (!taken_global[q]) F[nF++] = q;
    h->fs = (uint64_t*)malloc(h->ef_N * sizeof(uint64_t));
    uint64_t rank = 0;
    for (uint64_t q = n; q < M; q++) {
        uint64_t r = rank < nF ? rank : (nF ? nF - 1 : 0);
        h->fs[q - n] = nF ? F[r] : 0;
        if (taken_global[q]) rank++;
    }
    free(F);

    /* Elias-Fano: l = floor(log2(U / N)) low bits per value; high part in unary,
     * bit (v_i >> l) + i set; a select sample at every 64th one. */
    uint64_t N = h->ef_N, U = h->ef_U;
    h->ef_l = (U / N >= 1) ? or_bitlen(U / N) - 1 : 0;
    h->ef_low_nbits = N * (uint64_t)h->ef_l;
    h->ef_high_nbits = N + (U >> h->ef_l) + 1;
    h->ef_nsamples = (N + 63) / 64;
    h->ef_low = (uint64_t*)calloc(packed_words(h->ef_low_nbits), sizeof(uint64_t));
    h->ef_high = (uint64_t*)calloc(packed_words(h->ef_high_nbits), sizeof(uint64_t));
    h->ef_samples = (uint64_t*)calloc(h->ef_nsamples, sizeof(uint64_t));
    uint64_t lmask = h->ef_l ? ((1ULL << h->ef_l) - 1) : 0;
    for (uint64_t i = 0; i < N; i++) {
        put_bits(h->ef_low, i * h->ef_l, h->fs[i] & lmask, h->ef_l);
        uint64_t pos = (h->fs[i] >> h->ef_l) + i;
        h->ef_high[pos >> 6] |= 1ULL << (pos & 63);
        if (i % 64 == 0) h->ef_samples[i / 64] = pos;
    }
}

/* Elias-Fano access: the i-th value */
static uint64_t ef_access(const or_mphf* h, uint64_t i) {
    uint64_t pos = h->ef_samples[i / 64];
    uint64_t need = i % 64; /* ones to skip after the sampled one */
    while (need) {
        pos++;
        if ((h->ef_high[pos >> 6] >> (pos & 63)) & 1ULL) need--;
    }
    uint64_t high = pos - i;
    uint64_t low = get_bits(h->ef_low, i * h->ef_l, h->ef_l);
    return (high << h->ef_l) | low;
}

/* ---- space accounting (fixed spec) ---- */
static void account_bits(or_mphf* h) {
    uint64_t NP = h->NP;
    h->bits_header = 9 * 64;
    h->bits_offsets = (NP + 1) * (uint64_t)h->off_w + 64 + 64 + 8;
    /* a mono encoder: one column of B N_P values */
    int mono = h->prm.encoder >= OR_ENC_MONO_C;
    uint32_t enc = mono ? h->prm.encoder - OR_ENC_MONO_C : h->prm.encoder;
    uint32_t ncol = mono ? 1 : h->B;
    uint64_t nv = mono ? (uint64_t)h->B * NP : NP;
    uint64_t bp = 0;
    for (uint32_t b = 0; b < ncol; b++) {
        if (enc == OR_ENC_IC_C)
            bp += nv * (uint64_t)h->col_w[b] + 64 + 8;
        else if (enc == OR_ENC_IC_R || enc == OR_ENC_IC_EF ||
                 (enc == OR_ENC_IC_CR && b >= h->prm.compact_columns))
            bp += nv * (uint64_t)h->col_l[b] + h->col_H[b] + 32 * ((nv + 63) / 64) + 64 + 64 + 8;
        else if (enc == OR_ENC_IC_CR)
            bp += nv * (uint64_t)h->col_l[b] + 64 + 8; /* a Compact column of the mixture */
        else
            bp += nv * (uint64_t)h->col_rw[b] + h->col_K[b] * (uint64_t)h->col_dw[b] + 64 + 64 + 8 + 8;
    }
    if (enc == OR_ENC_IC_CR) bp += 32; /* the number of Compact columns */
    h->bits_pilots = bp;
    h->bits_remap = 0;
    if (h->ef_N)
        h->bits_remap = h->ef_low_nbits + h->ef_high_nbits + 64 * h->ef_nsamples + 3 * 64;
    h->bits_total = h->bits_header + h->bits_offsets + h->bits_pilots + h->bits_remap;
}

void or_free(or_mphf* h) {
    if (!h) return;
    free(h->part_size); free(h->table_size); free(h->T); free(h->pilots);
    free(h->off_words);
    free(h->col_w); free(h->col_base); free(h->pil_words);
    free(h->col_rw); free(h->col_rbase); free(h->col_dw); free(h->col_dbase); free(h->col_K);
    free(h->rank_words); free(h->dict_words);
    free(h->col_l); free(h->col_lbase); free(h->col_hbase); free(h->col_H);
    free(h->rice_low); free(h->rice_high); free(h->rice_samples);
    free(h->fs); free(h->ef_low); free(h->ef_high); free(h->ef_samples);
    free(h);
}

int or_build_hashed(const uint64_t* hk, uint64_t n, const or_params* prm, int threads, or_mphf** out) {
    *out = NULL;
    int st = check_params(n, prm);
    if (st != OR_OK) return st;
    int dup = has_duplicates(hk, n);
    if (dup < 0) return OR_ERR_OOM;
    if (dup) return OR_ERR_DUP_HASH;

    or_mphf* h = (or_mphf*)calloc(1, sizeof(or_mphf));
    if (!h) return OR_ERR_OOM;
    h->prm = *prm;
    h->n = n;
    h->NP = or_num_partitions(n, prm->partition_size);
    h->B = or_num_buckets(prm->lambda, prm->partition_size);
    h->eps = or_epsilon(prm->lambda, prm->partition_size);
    or_bucket_table_fn(prm->lambda, prm->alpha, prm->partition_size, prm->bucket_fn, h->table);
    uint64_t NP = h->NP;
    uint32_t B = h->B;

    uint64_t *start = NULL, *grouped = NULL;
    st = group_by_partition(hk, n, NP, &start, &grouped);
    if (st != OR_OK) {
        or_free(h);
        return st;
    }
    h->part_size = (uint64_t*)malloc(NP * sizeof(uint64_t));
    h->table_size = (uint64_t*)malloc(NP * sizeof(uint64_t));
    h->T = (uint64_t*)malloc((NP + 1) * sizeof(uint64_t));
    h->pilots = (uint32_t*)calloc((uint64_t)B * NP, sizeof(uint32_t));
    /* Section 4: concatenate the partitions by the prefix sum of their sizes */
    h->T[0] = 0;
    for (uint64_t j = 0; j < NP; j++) {
        h->part_size[j] = start[j + 1] - start[j];
        h->table_size[j] = or_table_size(h->part_size[j], prm->alpha);
        h->T[j + 1] = h->T[j] + h->table_size[j];
    }
    h->M = h->T[NP];
    uint8_t* taken_global = (uint8_t*)calloc(h->M, 1);

    /* partitions are independent; the loop order does not change any result */
    int status = OR_OK;
    uint64_t cand = 0, ktests = 0, stries = 0;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel
#endif
    {
        uint32_t* pil = (uint32_t*)malloc(B * sizeof(uint32_t));
        uint8_t* taken = NULL;
        uint64_t cap = 0;
        search_stats loc = {0, 0, 0};
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4)
#endif
        for (int64_t jj = 0; jj < (int64_t)NP; jj++) {
            uint64_t j = (uint64_t)jj;
            uint64_t m = h->table_size[j];
            if (m + 1 > cap) {
                free(taken);
                cap = m + 1;
                taken = (uint8_t*)malloc(cap);
            }
            int s = search_partition(grouped + start[j], h->part_size[j], m, h->table, B, prm, pil, taken,
                                     &loc);
            if (s != OR_OK) {
#ifdef _OPENMP
#pragma omp critical
#endif
                { if (status == OR_OK) status = s; }
                continue;
            }
            for (uint32_t b = 0; b < B; b++) h->pilots[(uint64_t)b * NP + j] = pil[b];
            for (uint64_t t = 0; t < m; t++)
                if (taken[t]) taken_global[h->T[j] + t] = 1;
        }
#ifdef _OPENMP
#pragma omp critical
#endif
        {
            cand += loc.candidates;
            ktests += loc.key_tests;
            stries += loc.s_tries;
        }
        free(pil);
        free(taken);
    }
    free(start);
    free(grouped);
    h->stat_candidates = cand;
    h->stat_key_tests = ktests;
    h->stat_s_tries = stries;
    if (status != OR_OK) {
        free(taken_global);
        or_free(h);
        return status;
    }
    encode_offsets(h);
    /* a mono encoder runs its column encoder over one column of B N_P values: the
     * column-major pilot array is that column, so B and N_P are swapped meanwhile */
    int mono = prm->encoder >= OR_ENC_MONO_C;
    uint32_t enc = mono ? prm->encoder - OR_ENC_MONO_C : prm->encoder;
    uint32_t B_saved = h->B;
    uint64_t NP_saved = h->NP;
    if (mono) {
        h->NP = (uint64_t)h->B * h->NP;
        h->B = 1;
    }
    if (enc == OR_ENC_IC_C)
        encode_compact(h);
    else if (enc == OR_ENC_IC_R)
        encode_rice(h);
    else if (enc == OR_ENC_IC_EF)
        encode_ef_columns(h);
    else if (enc == OR_ENC_IC_CR)
        encode_mixture(h);
    else
        encode_dictionary(h);
    h->B = B_saved;
    h->NP = NP_saved;
    build_remap(h, taken_global);
    free(taken_global);
    account_bits(h);
    *out = h;
    return OR_OK;
}

int or_build(const uint64_t* keys, uint64_t n, const or_params* prm, int threads, or_mphf** out) {
    *out = NULL;
    if (!keys || n == 0 || !prm) return OR_ERR_INVALID_ARG;
    uint64_t* hk = (uint64_t*)malloc(n * sizeof(uint64_t));
    if (!hk) return OR_ERR_OOM;
    for (uint64_t i = 0; i < n; i++) hk[i] = or_key_hash(keys[i], prm->seed);
    int st = or_build_hashed(hk, n, prm, threads, out);
    free(hk);
    return st;
}

/* Section 4: query = partition, offsets, bucket, decoded pilot, position */
void or_query_hashed(const or_mphf* h, const uint64_t* hkv, uint64_t q, uint64_t* out) {
    for (uint64_t i = 0; i < q; i++) {
        uint64_t hk = hkv[i];
        uint64_t j = or_mulhi64(hk, h->NP);
        uint64_t Tj = decode_offset(h, j);
        uint64_t m = decode_offset(h, j + 1) - Tj;
        if (m == 0) { /* only reachable by a key outside the set */
            out[i] = 0;
            continue;
        }
        uint32_t b = or_bucket(or_bucket_hash(hk), h->table, h->B);
        uint64_t p = decode_pilot(h, b, j);
        uint64_t local;
        if (h->prm.pilot_mode == OR_PILOT_ADDITIVE)
            local = (or_position_hash(hk, p / m, m) + p) % m; /* (h(x, floor(p/m)) + p) mod m */
        else
            local = or_position_hash(hk, p, m);
        uint64_t g = Tj + local;
        if (g >= h->n) g = ef_access(h, g - h->n);
        out[i] = g;
    }
}

void or_query(const or_mphf* h, const uint64_t* keys, uint64_t q, uint64_t* out) {
    for (uint64_t i = 0; i < q; i++) {
        uint64_t hk = or_key_hash(keys[i], h->prm.seed);
        or_query_hashed(h, &hk, 1, out + i);
    }
}

double or_bits_per_key(const or_mphf* h) { return (double)h->bits_total / (double)h->n; }

uint64_t or_get_u64(const or_mphf* h, const char* name) {
#define G(x) if (!strcmp(name, #x)) return (uint64_t)h->x
    G(n); G(M); G(NP); G(B); G(off_Q); G(off_w); G(off_nbits); G(pil_nbits); G(rank_nbits);
    G(dict_nbits); G(rlow_nbits); G(rhigh_nbits); G(rsamp_count); G(ef_N); G(ef_U); G(ef_l); G(ef_low_nbits); G(ef_high_nbits); G(ef_nsamples);
    G(bits_header); G(bits_offsets); G(bits_pilots); G(bits_remap); G(bits_total);
    G(stat_candidates); G(stat_key_tests); G(stat_s_tries);
#undef G
    if (!strcmp(name, "off_dmin")) return (uint64_t)h->off_dmin;
    return ~0ULL;
}

const void* or_get_array(const or_mphf* h, const char* name, uint64_t* count, uint32_t* eb) {
#define A(x, cnt, sz) if (!strcmp(name, #x)) { *count = (cnt); *eb = (sz); return h->x; }
    A(table, OR_TABLE_POINTS + 1, 8);
    A(part_size, h->NP, 8);
    A(table_size, h->NP, 8);
    A(T, h->NP + 1, 8);
    A(pilots, (uint64_t)h->B * h->NP, 4);
    A(off_words, packed_words(h->off_nbits), 8);
    uint32_t enc = h->prm.encoder >= OR_ENC_MONO_C ? h->prm.encoder - OR_ENC_MONO_C : h->prm.encoder;
    uint64_t nc = h->prm.encoder >= OR_ENC_MONO_C ? 1 : h->B; /* a mono encoder has one column */
    if (enc == OR_ENC_IC_C) {
        A(col_w, nc, 4);
        A(col_base, nc, 8);
        A(pil_words, packed_words(h->pil_nbits), 8);
    } else if (enc >= OR_ENC_IC_R) {
        A(col_l, nc, 4);
        A(col_lbase, nc, 8);
        A(col_hbase, nc, 8);
        A(col_H, nc, 8);
        A(rice_low, packed_words(h->rlow_nbits), 8);
        A(rice_high, packed_words(h->rhigh_nbits), 8);
        A(rice_samples, h->rsamp_count, 4);
    } else {
        A(col_rw, nc, 4);
        A(col_rbase, nc, 8);
        A(col_dw, nc, 4);
        A(col_dbase, nc, 8);
        A(col_K, nc, 8);
        A(rank_words, packed_words(h->rank_nbits), 8);
        A(dict_words, packed_words(h->dict_nbits), 8);
    }
    if (h->ef_N) {
        A(fs, h->ef_N, 8);
        A(ef_low, packed_words(h->ef_low_nbits), 8);
        A(ef_high, packed_words(h->ef_high_nbits), 8);
        A(ef_samples, h->ef_nsamples, 8);
    }
#undef A
    *count = 0;
    *eb = 0;
    return NULL;
}

/* ---- sampled mode ---- */
int or_partition_sizes(const uint64_t* hk, uint64_t n, const or_params* prm, uint64_t* n_j) {
    int st = check_params(n, prm);
    if (st != OR_OK) return st;
    uint64_t NP = or_num_partitions(n, prm->partition_size);
    memset(n_j, 0, NP * sizeof(uint64_t));
    for (uint64_t i = 0; i < n; i++) n_j[or_mulhi64(hk[i], NP)]++;
    return OR_OK;
}

int or_search_partitions(const uint64_t* hk, uint64_t n, const or_params* prm, const uint64_t* sel,
                         uint64_t nsel, int threads, uint32_t* pilots_out) {
    int st = check_params(n, prm);
    if (st != OR_OK) return st;
    uint64_t NP = or_num_partitions(n, prm->partition_size);
    uint32_t B = or_num_buckets(prm->lambda, prm->partition_size);
    uint64_t table[OR_TABLE_POINTS + 1];
    or_bucket_table_fn(prm->lambda, prm->alpha, prm->partition_size, prm->bucket_fn, table);
    int status = OR_OK;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t t = 0; t < (int64_t)nsel; t++) {
        uint64_t j = sel[t];
        if (j >= NP) {
#ifdef _OPENMP
#pragma omp critical
#endif
            { status = OR_ERR_INVALID_ARG; }
            continue;
        }
        uint64_t cnt = 0;
        for (uint64_t i = 0; i < n; i++)
            if (or_mulhi64(hk[i], NP) == j) cnt++;
        uint64_t* keys = (uint64_t*)malloc((cnt ? cnt : 1) * sizeof(uint64_t));
        cnt = 0;
        for (uint64_t i = 0; i < n; i++)
            if (or_mulhi64(hk[i], NP) == j) keys[cnt++] = hk[i];
        uint64_t m = or_table_size(cnt, prm->alpha);
        uint8_t* taken = (uint8_t*)malloc(m + 1);
        search_stats loc = {0, 0, 0};
        int s = search_partition(keys, cnt, m, table, B, prm, pilots_out + (uint64_t)t * B, taken, &loc);
        if (s != OR_OK) {
#ifdef _OPENMP
#pragma omp critical
#endif
            { if (status == OR_OK) status = s; }
        }
        free(keys);
        free(taken);
    }
    return status;
}

/* One partition alone (Section 4: partitions are searched independently):
 * its nj master hashes, table size m = or_table_size(nj, alpha); pilots_out[B]
 * and the final occupancy taken_out[m] (one byte per slot). */
int or_search_one_partition(const uint64_t* hk, uint64_t nj, const or_params* prm, uint32_t* pilots_out,
                            uint8_t* taken_out) {
    int st = check_params(nj ? nj : 1, prm);
    if (st != OR_OK) return st;
    uint32_t B = or_num_buckets(prm->lambda, prm->partition_size);
    uint64_t table[OR_TABLE_POINTS + 1];
    or_bucket_table_fn(prm->lambda, prm->alpha, prm->partition_size, prm->bucket_fn, table);
    uint64_t m = or_table_size(nj, prm->alpha);
    search_stats loc = {0, 0, 0};
    return search_partition(hk, nj, m, table, B, prm, pilots_out, taken_out, &loc);
}

/* ---- re-verification: replay every partition's buckets in order and check
 * that every pilot p' < p fails on the table state at that moment (Section 4.2:
 * the search returns the smallest working pilot). ---- */
int or_verify_first_valid(const or_mphf* h, const uint64_t* hk) {
    uint64_t NP = h->NP;
    uint64_t *start = NULL, *grouped = NULL;
    if (group_by_partition(hk, h->n, NP, &start, &grouped) != OR_OK) return 0;
    int ok_all = 1;
    for (uint64_t j = 0; j < NP && ok_all; j++) {
        uint64_t nj = start[j + 1] - start[j], m = h->table_size[j];
        const uint64_t* keys = grouped + start[j];
        uint8_t* taken = (uint8_t*)calloc(m + 1, 1);
        uint8_t* used = (uint8_t*)calloc(nj + 1, 1);
        /* buckets in placement order: recompute sizes */
        uint32_t* sz = (uint32_t*)calloc(h->B, sizeof(uint32_t));
        uint32_t* bk = (uint32_t*)malloc((nj + 1) * sizeof(uint32_t));
        for (uint64_t i = 0; i < nj; i++) {
            bk[i] = or_bucket(or_bucket_hash(keys[i]), h->table, h->B);
            sz[bk[i]]++;
        }
        bucket_ref* order = (bucket_ref*)malloc(h->B * sizeof(bucket_ref));
        uint32_t nb = 0;
        for (uint32_t b = 0; b < h->B; b++)
            if (sz[b]) {
                order[nb].b = b;
                order[nb].size = sz[b];
                nb++;
            }
        qsort(order, nb, sizeof(bucket_ref), bucket_order_cmp);
        uint64_t* pos = (uint64_t*)malloc((nj + 1) * sizeof(uint64_t));
        for (uint32_t r = 0; r < nb && ok_all; r++) {
            uint32_t b = order[r].b;
            uint64_t p = h->pilots[(uint64_t)b * NP + j];
            for (uint64_t q = 0; q <= p; q++) {
                uint32_t c = 0;
                int valid = 1;
                for (uint64_t i = 0; i < nj; i++) {
                    if (bk[i] != b) continue;
                    uint64_t x;
                    if (h->prm.pilot_mode == OR_PILOT_ADDITIVE)
                        x = (or_position_hash(keys[i], q / m, m) + q) % m;
                    else
                        x = or_position_hash(keys[i], q, m);
                    if (taken[x]) valid = 0;
                    for (uint32_t c2 = 0; c2 < c; c2++)
                        if (pos[c2] == x) valid = 0;
                    pos[c++] = x;
                }
                if (q < p && valid) ok_all = 0;   /* an earlier pilot would have worked */
                if (q == p && !valid) ok_all = 0; /* the stored pilot does not work */
                if (q == p)
                    for (uint32_t c2 = 0; c2 < c; c2++) taken[pos[c2]] = 1;
            }
        }
        free(pos); free(order); free(bk); free(sz); free(used); free(taken);
    }
    free(start);
    free(grouped);
    return ok_all;
}
