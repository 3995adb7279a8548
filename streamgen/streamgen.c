/*
 * streamgen.c -- seeded synthetic stream generator.
 *
 * This file produces the input tuples (group id, int32 value) that both the
 * CPU oracle and the CUDA path consume.  It contains no aggregation or window
 * arithmetic of any kind: it only turns (seed, stream index) into numbers.
 *
 * Stream shape (Section 5.1 of the paper): tuples (id, attr) where id is a
 * group identifier and attr an integer.  The paper's three datasets are a
 * round-robin assignment of tuples to groups (DS1), a Zipf distribution whose
 * most frequent groups have the smallest ids (DS2) and a randomly permuted
 * DS2 (DS3).  The distributions below reproduce those shapes:
 *   key_dist 0  uniform over [0, G)
 *   key_dist 1  Zipf(s) over ranks 1..G, rank r mapped to key perm[r-1]
 *               (identity perm = DS2 shape, random perm = DS3 shape), the
 *               permutation optionally re-drawn every `repermute_every`
 *               tuples so that the heavy hitters move
 *   key_dist 2  round robin, key = t mod G (DS1 shape)
 *   val_dist 0  uniform integer in [lo, hi)
 *   val_dist 1  normal(mean, sd) floored and clipped to [lo, hi]
 *   val_dist 2  lo + (t mod (hi - lo))           (closed-form test streams)
 *
 * Randomness: SplitMix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), written from its published
 * definition.  The generator is counter based: output i of a stream seeded
 * with x is the SplitMix64 finaliser applied to x + (i + 1) * gamma, so any
 * tuple range [t0, t0 + n) can be produced independently of the others.
 *
 * Zipf sampling: inverse CDF over a cumulative double table, i.e. the rank is
 * the first r with cdf[r] > u for u = (x >> 11) * 2^-53.  A guide table (the
 * "indexed search" of Chen and Asau, 1974) only accelerates that search; the
 * sampled rank is identical to a binary upper_bound on the table.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SG_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t sg_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Output number i (0-based) of the SplitMix64 generator seeded with `seed`. */
uint64_t sg_splitmix64_at(uint64_t seed, uint64_t i) {
    return sg_mix(seed + (i + 1) * SG_GAMMA);
}

/* Uniform double in [0, 1) with 53 random bits. */
double sg_unit_double(uint64_t seed, uint64_t i) {
    return (double)(sg_splitmix64_at(seed, i) >> 11) * 0x1.0p-53;
}

/* Uniform integer in [0, n) by the multiply-high map of a 64-bit draw. */
static inline uint64_t sg_below(uint64_t x, uint64_t n) {
    return (uint64_t)(((unsigned __int128)x * n) >> 64);
}

/* round(exp(U(ln lo, ln hi))) : log-uniform integer in [lo, hi]. */
int64_t sg_log_uniform_int(uint64_t seed, uint64_t i, int64_t lo, int64_t hi) {
    double u = sg_unit_double(seed, i);
    double x = exp(log((double)lo) + u * (log((double)hi) - log((double)lo)));
    int64_t r = (int64_t)llround(x);
    if (r < lo) r = lo;
    if (r > hi) r = hi;
    return r;
}

typedef struct sg_stream {
    int64_t G;
    int key_dist;
    double s;
    int permute;
    int64_t repermute_every;
    int val_dist;
    double mean, sd;
    int64_t lo, hi;
    uint64_t seed_keys, seed_vals, seed_perm;
    double *cdf;       /* cdf[r] = P(rank <= r + 1) */
    int32_t *guide;    /* guide[j] = first r with cdf[r] > j / G */
    int32_t *perm;     /* rank - 1 -> key for the cached epoch */
    int64_t perm_epoch;
} sg_stream;

static void sg_draw_perm(sg_stream *st, int64_t epoch) {
    int64_t G = st->G;
    for (int64_t i = 0; i < G; i++) st->perm[i] = (int32_t)i;
    if (st->permute) {
        /* Fisher-Yates with its own counter stream per epoch. */
        uint64_t ps = sg_splitmix64_at(st->seed_perm, (uint64_t)epoch);
        uint64_t c = 0;
        for (int64_t i = G - 1; i > 0; i--) {
            int64_t j = (int64_t)sg_below(sg_splitmix64_at(ps, c++), (uint64_t)(i + 1));
            int32_t t = st->perm[i];
            st->perm[i] = st->perm[j];
            st->perm[j] = t;
        }
    }
    st->perm_epoch = epoch;
}

sg_stream *sg_create(int64_t G, int key_dist, double s, int permute, int64_t repermute_every,
                     int val_dist, double mean, double sd, int64_t lo, int64_t hi, uint64_t seed) {
    if (G < 1 || G > 2147483647LL) return NULL;
    if (val_dist == 0 && hi <= lo) return NULL;
    if (val_dist == 2 && hi <= lo) return NULL;
    sg_stream *st = (sg_stream *)calloc(1, sizeof(sg_stream));
    if (!st) return NULL;
    st->G = G;
    st->key_dist = key_dist;
    st->s = s;
    st->permute = permute;
    st->repermute_every = repermute_every;
    st->val_dist = val_dist;
    st->mean = mean;
    st->sd = sd;
    st->lo = lo;
    st->hi = hi;
    st->seed_keys = sg_splitmix64_at(seed, 0);
    st->seed_vals = sg_splitmix64_at(seed, 1);
    st->seed_perm = sg_splitmix64_at(seed, 2);
    st->perm_epoch = -1;
    if (key_dist == 1) {
        st->cdf = (double *)malloc(sizeof(double) * (size_t)G);
        st->guide = (int32_t *)malloc(sizeof(int32_t) * (size_t)G);
        st->perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)G);
        if (!st->cdf || !st->guide || !st->perm) {
            free(st->cdf); free(st->guide); free(st->perm); free(st);
            return NULL;
        }
        double total = 0.0;
        for (int64_t r = 0; r < G; r++) total += pow((double)(r + 1), -s);
        double acc = 0.0;
        for (int64_t r = 0; r < G; r++) {
            acc += pow((double)(r + 1), -s);
            st->cdf[r] = acc / total;
        }
        st->cdf[G - 1] = 1.0;
        int64_t r = 0;
        for (int64_t j = 0; j < G; j++) {
            double thr = (double)j / (double)G;
            while (st->cdf[r] <= thr) r++;
            st->guide[j] = (int32_t)r;
        }
        sg_draw_perm(st, 0);
    }
    return st;
}

void sg_destroy(sg_stream *st) {
    if (!st) return;
    free(st->cdf);
    free(st->guide);
    free(st->perm);
    free(st);
}

/* Zipf rank (0-based) of draw x: first r with cdf[r] > u. */
static inline int64_t sg_zipf_rank(const sg_stream *st, uint64_t x) {
    double u = (double)(x >> 11) * 0x1.0p-53;
    int64_t j = (int64_t)(u * (double)st->G);
    if (j >= st->G) j = st->G - 1;
    int64_t r = st->guide[j];
    while (st->cdf[r] <= u) r++;
    return r;
}

/* One tuple: key and value of stream index t (perm already drawn for t). */
static inline void sg_one(const sg_stream *st, uint64_t t, int32_t *kp, int32_t *vp) {
    int32_t k;
    if (st->key_dist == 0) {
        k = (int32_t)sg_below(sg_splitmix64_at(st->seed_keys, t), (uint64_t)st->G);
    } else if (st->key_dist == 1) {
        k = st->perm[sg_zipf_rank(st, sg_splitmix64_at(st->seed_keys, t))];
    } else {
        k = (int32_t)(t % (uint64_t)st->G);
    }
    int32_t v;
    if (st->val_dist == 0) {
        v = (int32_t)(st->lo + (int64_t)sg_below(sg_splitmix64_at(st->seed_vals, t),
                                                 (uint64_t)(st->hi - st->lo)));
    } else if (st->val_dist == 1) {
        /* Box-Muller with u1 in (0, 1] and u2 in [0, 1). */
        double u1 = ((double)(sg_splitmix64_at(st->seed_vals, 2 * t) >> 11) + 1.0) * 0x1.0p-53;
        double u2 = (double)(sg_splitmix64_at(st->seed_vals, 2 * t + 1) >> 11) * 0x1.0p-53;
        double z = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
        double x = floor(st->mean + st->sd * z);
        if (x < (double)st->lo) x = (double)st->lo;
        if (x > (double)st->hi) x = (double)st->hi;
        v = (int32_t)x;
    } else {
        v = (int32_t)(st->lo + (int64_t)(t % (uint64_t)(st->hi - st->lo)));
    }
    if (kp) *kp = k;
    if (vp) *vp = v;
}

/* Fill tuples t0 .. t0 + n - 1 of the stream.  The range is cut at
 * permutation epochs; each piece is filled by all host threads. */
void sg_fill(sg_stream *st, int64_t t0, int64_t n, int32_t *keys, int32_t *vals) {
    int64_t i = 0;
    while (i < n) {
        int64_t t = t0 + i;
        int64_t end = n;
        if (st->key_dist == 1) {
            int64_t epoch = st->repermute_every > 0 ? t / st->repermute_every : 0;
            if (epoch != st->perm_epoch) sg_draw_perm(st, epoch);
            if (st->repermute_every > 0) {
                int64_t next = (epoch + 1) * st->repermute_every - t0;
                if (next < end) end = next;
            }
        }
        const sg_stream *cst = st;
        #pragma omp parallel for schedule(static) if (end - i > 65536)
        for (int64_t j = i; j < end; j++)
            sg_one(cst, (uint64_t)(t0 + j), keys ? keys + j : NULL, vals ? vals + j : NULL);
        i = end;
    }
}

/* Probability of rank r (0-based) under the stream's Zipf table. */
double sg_zipf_pmf(const sg_stream *st, int64_t r) {
    if (!st || st->key_dist != 1 || r < 0 || r >= st->G) return 0.0;
    return r == 0 ? st->cdf[0] : st->cdf[r] - st->cdf[r - 1];
}

/* Key of rank r (0-based) for the permutation of tuple index t. */
int32_t sg_key_of_rank(sg_stream *st, int64_t t, int64_t r) {
    if (!st || st->key_dist != 1 || r < 0 || r >= st->G) return -1;
    int64_t epoch = st->repermute_every > 0 ? t / st->repermute_every : 0;
    if (epoch != st->perm_epoch) sg_draw_perm(st, epoch);
    return st->perm[r];
}
