/*
 * oracle.c -- plain CPU oracle for the continuous windowed group-by
 * aggregate.  TEST INFRASTRUCTURE: only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code,
 * header or constant table with the CUDA path.
 *
 * What it computes (Section 3 of the paper: a group-by over tuples
 * (id, attr), each group aggregating the attribute values of a fixed-size
 * sliding window; iterations of fixed-size batches, Section 3.1):
 *
 *   After pushes totalling N tuples t = 0 .. N-1, with a global count-based
 *   window of W tuples, the window is the stream indices
 *   [max(0, N - W), N).  For every group g in [0, G):
 *     COUNT_g = #{ t in window : key_t = g }
 *     SUM_g   = sum of val_t over those t        (exact, int64)
 *     MIN_g   = min of val_t over those t        (INT32_MAX if COUNT_g = 0)
 *     MAX_g   = max of val_t over those t        (INT32_MIN if COUNT_g = 0)
 *     AVG_g   = (double)SUM_g / (double)COUNT_g  (IEEE binary64, round to
 *               nearest even; the quiet NaN 0x7FF8000000000000 if empty)
 *
 * The window is global (the last W tuples of the stream, whatever their
 * group) and the aggregates are emitted once per pushed batch; the paper
 * keeps one window per group and recomputes a SUM after every tuple.  Both
 * are readings recorded with the build's design notes.
 *
 * The implementation is the definition written out: the last W tuples are
 * kept in an array indexed by (stream index mod W), and the results are
 * recomputed from scratch over the window every time they are requested.
 * Nothing is incremental, nothing is retracted.
 *
 * Status codes: 0 ok, 1 invalid argument, 2 out of memory, 3 key outside
 * [0, G) (the push is rejected and the query is poisoned), 7 query poisoned.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OQ_OK = 0, OQ_EINVAL = 1, OQ_ENOMEM = 2, OQ_EKEY = 3, OQ_EPOISONED = 7 };

typedef struct oq_query {
    int64_t G;        /* number of groups, keys in [0, G) */
    int64_t W;        /* window length in tuples */
    int64_t N;        /* tuples pushed so far */
    int32_t *key;     /* key[t mod W] = key of stream tuple t, t in window */
    int32_t *val;     /* val[t mod W] = value of stream tuple t */
    int poisoned;
} oq_query;

int oq_create(int64_t groups, int64_t window, oq_query **out) {
    if (!out) return OQ_EINVAL;
    *out = NULL;
    if (groups < 1 || groups > 2147483647LL || window < 1 || window > 2147483647LL) return OQ_EINVAL;
    oq_query *q = (oq_query *)calloc(1, sizeof(oq_query));
    if (!q) return OQ_ENOMEM;
    q->G = groups;
    q->W = window;
    q->key = (int32_t *)malloc(sizeof(int32_t) * (size_t)window);
    q->val = (int32_t *)malloc(sizeof(int32_t) * (size_t)window);
    if (!q->key || !q->val) {
        free(q->key);
        free(q->val);
        free(q);
        return OQ_ENOMEM;
    }
    *out = q;
    return OQ_OK;
}

void oq_destroy(oq_query *q) {
    if (!q) return;
    free(q->key);
    free(q->val);
    free(q);
}

int64_t oq_seen(const oq_query *q) { return q ? q->N : -1; }

/* Append a batch of n tuples to the stream (Section 3.1: one iteration).
 * Every tuple is written in stream order, so a batch longer than the window
 * simply overwrites its own earlier tuples. */
int oq_push(oq_query *q, const int32_t *keys, const int32_t *vals, int64_t n) {
    if (!q) return OQ_EINVAL;
    if (q->poisoned) return OQ_EPOISONED;
    if (n < 0) return OQ_EINVAL;
    if (n == 0) return OQ_OK;
    if (!keys || !vals) return OQ_EINVAL;
    for (int64_t i = 0; i < n; i++) {
        if (keys[i] < 0 || (int64_t)keys[i] >= q->G) {
            q->poisoned = 1;
            return OQ_EKEY;
        }
    }
    for (int64_t i = 0; i < n; i++) {
        int64_t t = q->N + i;
        q->key[t % q->W] = keys[i];
        q->val[t % q->W] = vals[i];
    }
    q->N += n;
    return OQ_OK;
}

static void oq_finish_avg(int64_t sum, int64_t cnt, double *avg) {
    if (cnt == 0) {
        uint64_t nan_bits = 0x7FF8000000000000ULL;
        memcpy(avg, &nan_bits, sizeof(double));
    } else {
        *avg = (double)sum / (double)cnt;
    }
}

/* Aggregates of every group over the current window, from scratch.
 * Any output pointer may be NULL. */
int oq_results(const oq_query *q, int64_t *sum, int32_t *cnt, int32_t *mn, int32_t *mx, double *avg) {
    if (!q) return OQ_EINVAL;
    if (q->poisoned) return OQ_EPOISONED;
    int64_t G = q->G;
    int64_t *s = (int64_t *)calloc((size_t)G, sizeof(int64_t));
    int64_t *c = (int64_t *)calloc((size_t)G, sizeof(int64_t));
    int32_t *lo = (int32_t *)malloc(sizeof(int32_t) * (size_t)G);
    int32_t *hi = (int32_t *)malloc(sizeof(int32_t) * (size_t)G);
    if (!s || !c || !lo || !hi) {
        free(s); free(c); free(lo); free(hi);
        return OQ_ENOMEM;
    }
    for (int64_t g = 0; g < G; g++) {
        lo[g] = INT32_MAX;
        hi[g] = INT32_MIN;
    }
    int64_t first = q->N > q->W ? q->N - q->W : 0;
    for (int64_t t = first; t < q->N; t++) {
        int32_t g = q->key[t % q->W];
        int32_t v = q->val[t % q->W];
        c[g] += 1;
        s[g] += v;
        if (v < lo[g]) lo[g] = v;
        if (v > hi[g]) hi[g] = v;
    }
    for (int64_t g = 0; g < G; g++) {
        if (sum) sum[g] = s[g];
        if (cnt) cnt[g] = (int32_t)c[g];
        if (mn) mn[g] = lo[g];
        if (mx) mx[g] = hi[g];
        if (avg) oq_finish_avg(s[g], c[g], &avg[g]);
    }
    free(s); free(c); free(lo); free(hi);
    return OQ_OK;
}

/* Aggregates of one group over the current window, from scratch. */
int oq_group(const oq_query *q, int64_t g, int64_t *sum, int32_t *cnt, int32_t *mn, int32_t *mx, double *avg) {
    if (!q || g < 0 || g >= q->G) return OQ_EINVAL;
    if (q->poisoned) return OQ_EPOISONED;
    int64_t s = 0, c = 0;
    int32_t lo = INT32_MAX, hi = INT32_MIN;
    int64_t first = q->N > q->W ? q->N - q->W : 0;
    for (int64_t t = first; t < q->N; t++) {
        if (q->key[t % q->W] != g) continue;
        int32_t v = q->val[t % q->W];
        c += 1;
        s += v;
        if (v < lo) lo = v;
        if (v > hi) hi = v;
    }
    if (sum) *sum = s;
    if (cnt) *cnt = (int32_t)c;
    if (mn) *mn = lo;
    if (mx) *mx = hi;
    if (avg) oq_finish_avg(s, c, avg);
    return OQ_OK;
}
