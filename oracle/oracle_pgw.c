/*
 * oracle_pgw.c -- plain CPU oracle for the paper's own aggregate: one
 * count-based window per group.  TEST INFRASTRUCTURE: only the tests, the
 * smoke check and the benchmark's CPU-baseline leg load this library.  It
 * shares no code, header or constant table with the CUDA path.
 *
 * What it computes, step by step as Sections 3.2 and 5.1 of the paper
 * describe the GPU kernel's work:
 *
 *   Every group g in [0, G) owns a window of the last w values of its
 *   tuples, kept in a ring of w cells with a pointer to the oldest cell
 *   (nextPos).  Tuples are taken in stream order.  For a tuple (k, v):
 *     1. v is written at nextPos of group k's ring (overwriting the oldest
 *        value once the window is full) and nextPos moves to the next cell;
 *     2. the complete window of group k is scanned and its SUM computed
 *        from scratch (int64); the scan is repeated `passes` times (the
 *        paper's heavier variant checks the window elements ten times per
 *        update), each pass giving the same sum;
 *     3. that sum is the tuple's output.
 *
 * Status codes: 0 ok, 1 invalid argument, 2 out of memory, 3 key outside
 * [0, G) (the whole push is rejected and the query is poisoned), 7 query
 * poisoned.
 */
#include <stdint.h>
#include <stdlib.h>

enum { OW_OK = 0, OW_EINVAL = 1, OW_ENOMEM = 2, OW_EKEY = 3, OW_EPOISONED = 7 };

typedef struct ow_query {
    int64_t G;        /* groups */
    int32_t w;        /* window length per group */
    int32_t passes;   /* scans of the window per update */
    int32_t *cell;    /* G x w ring cells */
    int32_t *next;    /* per group: index of the oldest cell (nextPos) */
    int32_t *fill;    /* per group: values in the window (<= w) */
    int64_t seen;     /* tuples pushed */
    int poisoned;
} ow_query;

int ow_create(int64_t groups, int32_t window, int32_t passes, ow_query **out) {
    if (!out) return OW_EINVAL;
    *out = NULL;
    if (groups < 1 || groups > 2147483647LL || window < 1 || passes < 1) return OW_EINVAL;
    ow_query *q = (ow_query *)calloc(1, sizeof(ow_query));
    if (!q) return OW_ENOMEM;
    q->G = groups;
    q->w = window;
    q->passes = passes;
    q->cell = (int32_t *)calloc((size_t)groups * (size_t)window, sizeof(int32_t));
    q->next = (int32_t *)calloc((size_t)groups, sizeof(int32_t));
    q->fill = (int32_t *)calloc((size_t)groups, sizeof(int32_t));
    if (!q->cell || !q->next || !q->fill) {
        free(q->cell);
        free(q->next);
        free(q->fill);
        free(q);
        return OW_ENOMEM;
    }
    *out = q;
    return OW_OK;
}

void ow_destroy(ow_query *q) {
    if (!q) return;
    free(q->cell);
    free(q->next);
    free(q->fill);
    free(q);
}

int64_t ow_seen(const ow_query *q) { return q ? q->seen : -1; }

/* Push n tuples in stream order; out[i] receives the window sum of tuple i's
 * group right after tuple i is inserted (out may be NULL). */
int ow_push(ow_query *q, const int32_t *keys, const int32_t *vals, int64_t n, int64_t *out) {
    if (!q || n < 0 || (n > 0 && (!keys || !vals))) return OW_EINVAL;
    if (q->poisoned) return OW_EPOISONED;
    for (int64_t i = 0; i < n; i++)
        if (keys[i] < 0 || (int64_t)keys[i] >= q->G) {
            q->poisoned = 1;
            return OW_EKEY;
        }
    const int32_t w = q->w;
    for (int64_t i = 0; i < n; i++) {
        const int64_t g = keys[i];
        int32_t *win = q->cell + g * (int64_t)w;
        win[q->next[g]] = vals[i];
        q->next[g] = q->next[g] + 1 == w ? 0 : q->next[g] + 1;
        if (q->fill[g] < w) q->fill[g]++;
        /* the cells holding values are 0 .. fill-1 until the ring wraps, then all w */
        int64_t sum = 0;
        for (int32_t p = 0; p < q->passes; p++) {
            sum = 0;
            for (int32_t c = 0; c < q->fill[g]; c++) sum += win[c];
        }
        if (out) out[i] = sum;
    }
    q->seen += n;
    return OW_OK;
}

/* The current window sum of group g (0 for an empty group). */
int ow_group_sum(const ow_query *q, int64_t g, int64_t *sum, int32_t *count) {
    if (!q || g < 0 || g >= q->G || !sum || !count) return OW_EINVAL;
    if (q->poisoned) return OW_EPOISONED;
    const int32_t *win = q->cell + g * (int64_t)q->w;
    int64_t s = 0;
    for (int32_t c = 0; c < q->fill[g]; c++) s += win[c];
    *sum = s;
    *count = q->fill[g];
    return OW_OK;
}
