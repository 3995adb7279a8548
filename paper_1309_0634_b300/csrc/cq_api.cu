/*
 * cq_api.cu -- the C ABI of include/cq.h: host-side window bookkeeping and
 * kernel launches for one continuous query.
 *
 * Window bookkeeping of a push of n tuples (Section 3.1: one iteration):
 *   N        tuples seen before the push; the old window is [H, N) with
 *            H = max(0, N - W)
 *   n_eff    min(n, W): only the last n_eff tuples of the batch can be in
 *            the new window [H', N + n), H' = max(0, N + n - W); the first
 *            n - n_eff enter and leave within the push and are never read
 *   slots    the effective tuple with stream index t goes to slot t mod W
 *            and evicts the slot's occupant if the ring held one
 *   expiry   the evicted tuples are exactly the old tuples in [H, H')
 *   flips    MIN/MAX keep a front [H, F) and a back [F, N):
 *              H' <= F       the departing tuples are all in the front
 *              H' >= N       every old tuple departs (n >= W): the epoch
 *                            advances, both segments restart empty
 *              F < H' < N    the front is used up: the old back [F, N)
 *                            becomes the new front (flip), then the
 *                            departing tuples [F, H') leave it
 */
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "cq_group.cuh"
#include "cq_heavy.cuh"
#include "cq_host.h"
#include "cq_internal.h"
#include "cq_push.cuh"
#include "cq_stream.cuh"

using namespace cq;

struct cq_query {
    DeviceState d;
    Options opt;
    int64_t G = 0, W = 0;
    uint32_t aggs = 0;
    int minmax = 0, avg = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0, num_sms = 148;
    int64_t N = 0, F = 0;
    uint32_t epoch = 1;
    int *h_err = nullptr;
    int poison = 0;            /* 0 ok, else CQ_EKEY observed */
    bool poison_reported = false;
    /* cq_push_host: two device slots for the copied batches, filled on a
       copy stream so that the next batch goes up while this one is pushed */
    int32_t *stage_k[2] = {nullptr, nullptr}, *stage_v[2] = {nullptr, nullptr};
    int64_t stage_cap = 0;
    int stage_slot = 0;
    cudaStream_t h2d = nullptr;
    cudaEvent_t ev_staged[2] = {nullptr, nullptr}, ev_consumed[2] = {nullptr, nullptr};
    int64_t pushes = 0, flips = 0, resets = 0, launches = 0;
    int64_t device_bytes = 0;
    unsigned long long bar_base = 0;   /* grid-barrier arrivals so far */
    unsigned long long draw_base = 0;  /* register-staged kernel's range draws so far (bar[1]) */
    int hot_parity = 0;                /* which half of hotlist is current */
    int last_path = 0;
    unsigned long long *trace = nullptr;   /* caller-owned phase-stamp buffer */
    int64_t trace_slots = 0;
    int *bad = nullptr;                    /* device: bad keys seen by the running push */
    cudaEvent_t ev = nullptr;              /* orders the query's stream with group launches */
    /* launch plans already computed, keyed by (n_eff, front, options) */
    struct PlanKey {
        int64_t n;
        int front, cps, rbits, tma;
    } plan_key[8];
    PushPlan plan_val[8];
    int plan_ok[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int plan_used = 0;
    /* cq_push_many: scratch of the persistent launch (grown on demand),
       two pinned descriptor slots (each reused once its copy is done) */
    struct Stream {
        void *stage = nullptr;
        int64_t stage_bytes = 0;
        void *pairs = nullptr;
        int64_t pairs_bytes = 0;
        HotAcc *hotpart = nullptr;
        int32_t *lists = nullptr;            /* keys, then counts: 2 x [kSListSlots][2][kMaxHot] */
        unsigned long long *ctl = nullptr;   /* SCtl words, then list_n ints */
        SBatch *d_desc = nullptr;
        SBatch *h_desc[2] = {nullptr, nullptr};
        cudaEvent_t ev_desc[2] = {nullptr, nullptr};
        int desc_slot = 0;
        int64_t wait_us = 2000000;
        int stall_batch = -1;
        int pp_opt = -1;                     /* CQ_OPT_STREAM_PRODUCERS (-1: automatic) */
    } sm;
};

namespace {

const int64_t kMaxSize = 2147483647LL;
const int64_t kMaxGroups = (1LL << 30) - 2;   /* a delta's key word keeps two flag bits */

int64_t pad16(int64_t x) { return (x + 15) / 16 * 16; }

/* Inserts in a push of n_eff tuples that make a heavy hitter sure of a list
 * slot: more than n_eff / cap.  Fewer than cap keys can have that many (their
 * inserts would add up to more than n_eff), so they always fit; the keys
 * above the detection threshold but below this one take the slots left. */
uint32_t hot_guarantee(int64_t n_eff, int cap) {
    if (cap <= 0) return 0xFFFFFFFFu;
    const int64_t g = n_eff / cap + 1;
    return g > 0xFFFFFFFFLL ? 0xFFFFFFFFu : (uint32_t)g;
}

cq_status cuda_status(cudaError_t e) {
    return e == cudaSuccess ? CQ_OK : (e == cudaErrorMemoryAllocation ? CQ_ENOMEM : CQ_ECUDA);
}

void set_device(const cq_query *q) {
    int cur = -1;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != q->device) cudaSetDevice(q->device);
}

/* Report a bad key once as CQ_EKEY, then CQ_EPOISONED. */
cq_status poison_status(cq_query *q) {
    if (!q->poison && q->h_err) {
        int f = *(volatile int *)q->h_err;
        if (f) q->poison = (f & 2) ? CQ_ETIMEOUT : CQ_EKEY;
    }
    if (!q->poison) return CQ_OK;
    if (!q->poison_reported) {
        q->poison_reported = true;
        return (cq_status)q->poison;
    }
    return CQ_EPOISONED;
}

/* A push that failed after its bookkeeping began (prepare_push may already
 * have advanced the epoch, moved the front or queued a flip) leaves the query
 * inconsistent: it is poisoned.  This call reports the failure; every later
 * call except cq_destroy returns CQ_EPOISONED. */
cq_status fail_prepared(cq_query *q, cudaError_t e) {
    const cq_status st = e == cudaSuccess ? CQ_ECUDA : cuda_status(e);
    if (!q->poison) {
        q->poison = st;
        q->poison_reported = true;
    }
    return st;
}

template <typename T>
cudaError_t dmalloc(cq_query *q, T **p, int64_t n) {
    size_t bytes = sizeof(T) * (size_t)(n > 0 ? n : 1);
    cudaError_t e = cudaMalloc((void **)p, bytes);
    if (e == cudaSuccess) q->device_bytes += (int64_t)bytes;
    return e;
}

void free_all(cq_query *q) {
    DeviceState &d = q->d;
    cudaFree(d.ring_k);
    cudaFree(d.ring_v);
    cudaFree(d.sum);
    cudaFree(d.cnt);
    cudaFree(d.rmin);
    cudaFree(d.rmax);
    cudaFree(d.ravg);
    cudaFree(d.bmin);
    cudaFree(d.bmax);
    cudaFree(d.fmin);
    cudaFree(d.fmax);
    cudaFree(d.sufs);
    cudaFree(d.fptr);
    cudaFree(d.fdep);
    cudaFree(d.touched);
    cudaFree(d.err);
    cudaFree(d.stage);
    cudaFree(d.off);
    cudaFree(d.hotpart);
    cudaFree(d.hotacc);
    cudaFree(d.emkey);
    cudaFree(d.emacc);
    cudaFree(d.emfolds);
    cudaFree(d.hotlist);
    cudaFree(d.hotlist_n);
    cudaFree(d.hotlist_cnt);
    cudaFree(d.bar);
    cudaFree(q->bad);
    if (q->ev) cudaEventDestroy(q->ev);
    flip_free(d);
    if (q->h2d) cudaStreamSynchronize(q->h2d);
    for (int b = 0; b < 2; b++) {
        cudaFree(q->stage_k[b]);
        cudaFree(q->stage_v[b]);
        if (q->ev_staged[b]) cudaEventDestroy(q->ev_staged[b]);
        if (q->ev_consumed[b]) cudaEventDestroy(q->ev_consumed[b]);
    }
    if (q->h2d) cudaStreamDestroy(q->h2d);
    cudaFree(q->sm.stage);
    cudaFree(q->sm.pairs);
    cudaFree(q->sm.hotpart);
    cudaFree(q->sm.lists);
    cudaFree(q->sm.ctl);
    cudaFree(q->sm.d_desc);
    for (int b = 0; b < 2; b++) {
        if (q->sm.ev_desc[b]) cudaEventSynchronize(q->sm.ev_desc[b]);
        if (q->sm.h_desc[b]) cudaFreeHost(q->sm.h_desc[b]);
        if (q->sm.ev_desc[b]) cudaEventDestroy(q->sm.ev_desc[b]);
    }
    if (q->h_err) cudaFreeHost(q->h_err);
    if (q->own_stream && q->stream) cudaStreamDestroy(q->stream);
}

void bump_epoch(cq_query *q) {
    if (q->epoch >= 0xFFFFFFFEu) {
        /* every tag is about to be rewritten or dropped: start over at 1 */
        launch_reset_tags(q->d, q->stream);
        q->launches += 1;
        q->epoch = 1;
    } else {
        q->epoch++;
    }
}

/* Device buffer of at least `bytes`, grown on demand (waits for the stream
 * before freeing the old one). */
/* kMaxHot heavy-hitter accumulators at their identity (host copy). */
const HotAcc *hot_acc_identity() {
    static HotAcc id[kMaxHot];
    static bool ready = false;
    if (!ready) {
        for (int h = 0; h < kMaxHot; h++) {
            id[h].sum = 0;
            id[h].ins = id[h].ret = 0;
            id[h].imin = INT32_MAX;
            id[h].imax = INT32_MIN;
            id[h].fdep = 0;
            id[h].pad_ = 0;
        }
        ready = true;
    }
    return id;
}

cudaError_t ensure_buffer(cq_query *q, void **p, int64_t *have, int64_t bytes) {
    if (*have >= bytes) return cudaSuccess;
    cudaError_t e = cudaStreamSynchronize(q->stream);
    if (e != cudaSuccess) return e;
    if (*p) {
        cudaFree(*p);
        q->device_bytes -= *have;
    }
    *p = nullptr;
    *have = 0;
    e = cudaMalloc(p, (size_t)bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return e;
    }
    *have = bytes;
    q->device_bytes += bytes;
    return cudaSuccess;
}

bool make_plan_uncached(cq_query *q, int64_t n_eff, bool front, bool tma, int rbits, PushPlan *out);

const int kMaxDevices = 64;

/* The dynamic shared-memory limit of the register-staged kernel variant the
 * push uses (raised, never lowered, per device: raise_dyn_smem). */
cudaError_t raise_smem_attr(bool minmax, bool front, int64_t bytes) {
    return raise_dyn_smem(push_kernel_ptr(minmax, front), (int)bytes);
}

/* Shape of the partitioned push for n_eff tuples (false if the key space is
 * too large for key-range partitions that fit shared memory).  `wide` asks
 * for the widest key ranges (kMaxRBits) when no partition width is set.
 * Plans are cached: the occupancy query and the shared-memory attribute are
 * host driver calls that would otherwise cost every push. */
bool make_plan(cq_query *q, int64_t n_eff, bool front, bool tma, PushPlan *out, bool wide = false) {
    const int rbits = q->opt.partition_bits > 0 ? (int)q->opt.partition_bits : (wide ? kMaxRBits : 0);
    for (int i = 0; i < q->plan_used; i++) {
        const cq_query::PlanKey &k = q->plan_key[i];
        if (k.n == n_eff && k.front == (int)front && k.cps == q->opt.ctas_per_sm && k.rbits == rbits &&
            k.tma == (int)tma) {
            *out = q->plan_val[i];
            return q->plan_ok[i] != 0;
        }
    }
    PushPlan pl;
    const bool ok = make_plan_uncached(q, n_eff, front, tma, rbits, &pl);
    int slot = q->plan_used < 8 ? q->plan_used++ : (int)(n_eff & 7);
    q->plan_key[slot] = cq_query::PlanKey{n_eff, (int)front, q->opt.ctas_per_sm, rbits, (int)tma};
    q->plan_val[slot] = pl;
    q->plan_ok[slot] = ok;
    *out = pl;
    return ok;
}

bool make_plan_uncached(cq_query *q, int64_t n_eff, bool front, bool tma, int rbits, PushPlan *out) {
    const void *fn = push_kernel_ptr(q->minmax != 0, front);
    const int threads = kPushThreads;
    const int chunk_cap = kChunkCap;
    const int max_cps = q->opt.ctas_per_sm;
    for (int cps = max_cps; cps >= 1; cps--) {
        PushPlan pl;
        pl.tma = tma;
        int64_t grid = (int64_t)q->num_sms * cps;
        const int64_t want = (n_eff + 511) / 512;
        if (grid > want) grid = want;
        if (grid < 1) grid = 1;
        pl.grid = (int)grid;
        pl.rounds = (int)((n_eff + grid * chunk_cap - 1) / (grid * chunk_cap));
        pl.C = pl.grid * pl.rounds;
        pl.S = (n_eff + pl.C - 1) / pl.C;
        if (tma) pl.S = (pl.S + 3) / 4 * 4;   /* chunk starts 16-byte aligned */
        if (pl.S > chunk_cap) return false;
        if (rbits > 0) {
            pl.rbits = rbits;
        } else {
            /* small partitions (about 8 per CTA) balance phase B */
            int64_t max_p = 8 * (int64_t)pl.grid;
            if (max_p > kMaxParts) max_p = kMaxParts;
            pl.rbits = 0;
            while (pl.rbits < kMaxRBits && ((q->G + ((int64_t)1 << pl.rbits) - 1) >> pl.rbits) > max_p) pl.rbits++;
        }
        if (tma && pl.rbits < 2) pl.rbits = 2;   /* key ranges start 16-byte aligned */
        pl.P = (int)((q->G + ((int64_t)1 << pl.rbits) - 1) >> pl.rbits);
        if (pl.P > kMaxParts) return false;
        const int R = 1 << pl.rbits;
        const int64_t per_cta = (pl.P + (int64_t)pl.grid - 1) / pl.grid;
        const int table_max = tma ? kMaxTable / 2 : kMaxTable;
        int64_t ppp = table_max / R;
        if (ppp > per_cta) ppp = per_cta;
        if (ppp < 1) ppp = 1;
        pl.ppp = (int)ppp;
        pl.tcap = (int)((ppp * R + 3) / 4 * 4);
        pl.dcap = push_delta_cap(front);
        pl.stride = (2 * pl.S + pl.P + 2 + 1) & ~1LL;   /* runs padded to even lengths */
        pl.smem = push_smem_bytes(pl, front);
        if (pl.smem > 227 * 1024) continue;
        if (raise_smem_attr(q->minmax != 0, front, pl.smem) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, (size_t)pl.smem) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        if ((int64_t)occ * q->num_sms >= pl.grid) {
            *out = pl;
            return true;
        }
    }
    return false;
}

cudaError_t launch_partitioned(cq_query *q, const IngestArgs &a, const PushPlan &pl, bool front) {
    DeviceState &d = q->d;
    const int64_t dsize = 8;   /* every delta is 8 bytes */
    cudaError_t e = ensure_buffer(q, &d.stage, &d.stage_bytes, (int64_t)pl.C * pl.stride * dsize);
    if (e == cudaSuccess)
        e = ensure_buffer(q, (void **)&d.off, &d.off_bytes, (int64_t)pl.C * (pl.P + 1) * 4);
    if (e == cudaSuccess)
        e = ensure_buffer(q, &d.hotpart, &d.hotpart_bytes, (int64_t)kMaxHot * pl.grid * hot_rec_bytes());
    if (e != cudaSuccess) return e;
    PushArgs p;
    memset(&p, 0, sizeof(p));
    p.keys = a.keys;
    p.vals = a.vals;
    p.n = a.n;
    p.slot0 = a.slot0;
    p.hmod = a.hmod;
    p.old_len = a.old_len;
    p.fa = a.fa;
    p.fb = a.fb;
    p.G = q->G;
    p.W = q->W;
    p.epoch = a.epoch;
    p.avg = q->avg;
    p.grid = pl.grid;
    p.rounds = pl.rounds;
    p.C = pl.C;
    p.S = pl.S;
    p.rbits = pl.rbits;
    p.P = pl.P;
    p.tcap = pl.tcap;
    p.ppp = pl.ppp;
    p.dcap = pl.dcap;
    p.stride = pl.stride;
    p.ring_k = d.ring_k;
    p.ring_v = d.ring_v;
    p.sufs = d.sufs;
    p.fptr = d.fptr;
    p.sum = d.sum;
    p.cnt = d.cnt;
    p.bmin = d.bmin;
    p.bmax = d.bmax;
    p.fmin = d.fmin;
    p.fmax = d.fmax;
    p.rmin = d.rmin;
    p.rmax = d.rmax;
    p.ravg = d.ravg;
    p.stage = d.stage;
    p.off = d.off;
    p.hotpart = d.hotpart;
    p.emkey = d.emkey;
    p.emacc = d.emacc;
    p.emfolds = d.emfolds;
    const int cur = q->hot_parity, nxt = cur ^ 1;
    p.hot_cur = d.hotlist + cur * 2 * kMaxHot;
    p.hot_cur_n = d.hotlist_n + 2 * cur;
    p.hot_next = d.hotlist + nxt * 2 * kMaxHot;
    p.hot_next_n = d.hotlist_n + 2 * nxt;
    p.hot_cur_cnt = d.hotlist_cnt + cur * 2 * kMaxHot;
    p.hot_next_cnt = d.hotlist_cnt + nxt * 2 * kMaxHot;
    p.hot_cap = q->opt.hot_keys;
    p.hot_gthr = hot_guarantee(a.n, q->opt.hot_keys);
    int64_t thr = q->opt.hot_threshold;
    if (thr <= 0) {
        thr = a.n / pl.P;
        if (thr < 64) thr = 64;
    }
    p.hot_threshold = (uint32_t)(thr > 0x7FFFFFFF ? 0x7FFFFFFF : thr);
    p.heavy_min = heavy_key_min(pl.S, a.n, p.hot_threshold);
    p.heavy_bound = heavy_bound(pl.S * (a.old_len > 0 ? 2 : 1), pl.P, p.heavy_min);
    p.bar = d.bar;
    p.bar_target = q->bar_base + (unsigned long long)pl.grid;
    p.draw_base = q->draw_base;
    p.err = d.err;
    p.err_host = d.err_host;
    p.trace = (q->trace && q->trace_slots >= (int64_t)pl.grid * 8) ? q->trace : nullptr;
    void *args[] = {&p};
    const void *fn = push_kernel_ptr(q->minmax != 0, front);
    e = cudaLaunchCooperativeKernel(fn, dim3(pl.grid), dim3(kPushThreads), args,
                                    (size_t)pl.smem, q->stream);
    if (e != cudaSuccess) return e;
    q->bar_base += (unsigned long long)pl.grid;
    /* every CTA draws until a draw lands past the last range */
    q->draw_base += (unsigned long long)((pl.P + pl.ppp - 1) / pl.ppp + pl.grid);
    return cudaSuccess;
}

/* ---- the group kernel: one cooperative launch for one or many queries ---- */


struct GPlan {
    int rbits = 0, P = 0, C = 0, ppp = 0, R = 0;
    int64_t S = 0, stride = 0;
    int aligned = 0;
};

int group_grid(int device, int num_sms) { (void)device; return 2 * num_sms; }

/* CTAs of a group launch on this part (2 per SM x 148 SMs), for the share
 * of a push one CTA's key ranges should carry. */
constexpr int64_t kGridShare = 296;

/* Chunks and key ranges of one query's push of n tuples; false when the key
 * space needs more partitions than the group kernel supports. */
bool group_plan(const cq_query *q, int64_t n, const int32_t *k, const int32_t *v, int64_t slot0, int grid, bool single,
                GPlan *pl, bool replace = false) {
    /* a window-replacing single-query launch stages one delta per tuple and
       no ring slots, so its chunks may be twice as long */
    const int64_t cap = single && replace ? kGChunkReplace : kGChunk;
    int r = 2;
    if (q->opt.partition_bits > 0) r = q->opt.partition_bits < 2 ? 2 : q->opt.partition_bits;
    else
        while (r <= 10 && ((q->G + ((int64_t)1 << r) - 1) >> r) > kGMaxParts) r++;
    if (r > 10) return false;
    const int64_t P = (q->G + ((int64_t)1 << r) - 1) >> r;
    if (P > kGMaxParts) return false;
    pl->rbits = r;
    pl->P = (int)P;
    int64_t c = (n + cap - 1) / cap;
    if (single) {
        if (n >= (int64_t)grid * 1024) {
            c = (c + grid - 1) / grid * grid;   /* whole rounds over the CTAs */
        } else {
            int64_t want = (n + 255) / 256;     /* small batch: spread it */
            if (want > grid) want = grid;
            if (c < want) c = want;
        }
    }
    if (c < 1) c = 1;
    int64_t S = (n + c - 1) / c;
    S = (S + 3) / 4 * 4;
    if (S > cap) S = cap;
    pl->S = S;
    pl->C = (int)((n + S - 1) / S);
    if (pl->C < 1) pl->C = 1;
    int64_t ppp = (P + grid - 1) / grid;
    const int64_t lo = (256 >> r) > 1 ? (256 >> r) : 1, hi = (kGTable >> r) > 1 ? (kGTable >> r) : 1;
    if (ppp < lo) ppp = lo;
    if (ppp > hi) ppp = hi;
    if (ppp > P) ppp = P;
    pl->ppp = (int)ppp;
    pl->R = (int)((P + ppp - 1) / ppp);
    pl->stride = ((single && replace ? 1 : 2) * S + P + 2 + 1) / 2 * 2;
    pl->aligned = ((uintptr_t)k % 16 == 0) && ((uintptr_t)v % 16 == 0) && (slot0 % 4 == 0) && (q->W % 4 == 0);
    return true;
}

/* The group kernel's key ranges hold at most kGTable groups, so a key space
 * of more than 2^19 groups is cut into hundreds of ranges, and every chunk's
 * run for every range is a separate copy in phase B.  When those runs would
 * average under 8 deltas, the register-staged kernel with its widest ranges
 * (2^kMaxRBits groups) moves the same deltas in fewer, cheaper runs.  Only
 * the automatic path choice of a single-query push follows this: a group
 * launch keeps every member it can take, since pushing a member on its own
 * costs a launch of its own. */
bool prefer_wide_ranges(const cq_query *q, const GPlan &gp, int64_t n) {
    return q->opt.path == 0 && q->opt.partition_bits == 0 && q->G > ((int64_t)1 << 19) &&
           2 * n < 8 * (int64_t)gp.R * gp.C;
}

/* Bytes of a group launch's run table: per key range, a (begin, length) pair
 * for each chunk, rows padded to an even chunk count (16-byte rows). */
int64_t group_pair_bytes(const GPlan &pl) { return (int64_t)pl.R * ((pl.C + 1) & ~1) * 8; }

/* Fill a query's descriptor; the scratch pointers (stage, off, hotpart) are
 * the query's own buffers, as they stand. */
void group_desc_fill(const cq_query *q, const IngestArgs &a, const GPlan &pl, bool front, QDesc *d) {
    const DeviceState &st = q->d;
    memset(d, 0, sizeof(*d));
    d->keys = a.keys;
    d->vals = a.vals;
    d->n = a.n;
    d->slot0 = a.slot0;
    d->hmod = a.hmod;
    const bool replace = a.n == q->W && a.old_len > 0;   /* the whole window leaves */
    d->old_len = replace ? 0 : a.old_len;
    d->fa = a.fa;
    d->fb = a.fb;
    d->G = q->G;
    d->W = q->W;
    d->S = pl.S;
    d->stride = pl.stride;
    d->epoch = a.epoch;
    d->flags = (q->minmax ? QF_MINMAX : 0) | (front ? QF_FRONT : 0) | (q->avg ? QF_AVG : 0) |
               (pl.aligned ? QF_ALIGNED : 0) | (replace ? QF_REPLACE : 0);
    d->rbits = pl.rbits;
    d->P = pl.P;
    d->C = pl.C;
    d->ppp = pl.ppp;
    d->R = pl.R;
    d->hot_cap = q->opt.hot_keys;
    d->hot_gthr = hot_guarantee(a.n, q->opt.hot_keys);
    int64_t thr = q->opt.hot_threshold;
    if (thr <= 0) {
        /* more inserts than an average partition's, or than a CTA's share of
           the push when the key space has fewer partitions than the grid has
           CTAs: a few-group query's keys would otherwise make its one or two
           key ranges the launch's longest work */
        const int64_t parts = pl.P > kGridShare ? pl.P : kGridShare;
        thr = a.n / parts;
        if (thr < 64) thr = 64;
    }
    d->hot_threshold = (uint32_t)(thr > 0x7FFFFFFF ? 0x7FFFFFFF : thr);
    d->heavy_min = heavy_key_min(pl.S, a.n, d->hot_threshold);
    d->heavy_bound = heavy_bound(pl.S * (d->old_len > 0 ? 2 : 1), pl.P, d->heavy_min);
    d->ring_k = st.ring_k;
    d->ring_v = st.ring_v;
    d->sufs = st.sufs;
    d->fptr = st.fptr;
    d->sum = st.sum;
    d->cnt = st.cnt;
    d->bmin = st.bmin;
    d->bmax = st.bmax;
    d->fmin = st.fmin;
    d->fmax = st.fmax;
    d->rmin = st.rmin;
    d->rmax = st.rmax;
    d->ravg = st.ravg;
    d->stage = st.stage;
    d->off = st.off;
    d->hotacc = (HotAcc *)st.hotacc;
    d->emkey = st.emkey;
    d->emacc = (HotAcc *)st.emacc;
    d->emfolds = st.emfolds;
    const int cur = q->hot_parity, nxt = cur ^ 1;
    d->hot_cur = st.hotlist + cur * 2 * kMaxHot;
    d->hot_cur_n = st.hotlist_n + 2 * cur;
    d->hot_cur_cnt = st.hotlist_cnt + cur * 2 * kMaxHot;
    d->hot_next = st.hotlist + nxt * 2 * kMaxHot;
    d->hot_next_n = st.hotlist_n + 2 * nxt;
    d->hot_next_cnt = st.hotlist_cnt + nxt * 2 * kMaxHot;
    d->err = st.err;
    d->err_host = st.err_host;
    d->bad = q->bad;
}

/* Fill a query's descriptor for a launch whose deltas are `ds` bytes, growing
 * the query's scratch buffers first. */
cudaError_t group_desc(cq_query *q, const IngestArgs &a, const GPlan &pl, bool front, int ds, QDesc *d) {
    DeviceState &st = q->d;
    cudaError_t e = ensure_buffer(q, &st.stage, &st.stage_bytes, (int64_t)pl.C * pl.stride * ds);
    if (e == cudaSuccess) e = ensure_buffer(q, (void **)&st.off, &st.off_bytes, group_pair_bytes(pl));
    if (e != cudaSuccess) return e;
    group_desc_fill(q, a, pl, front, d);
    return cudaSuccess;
}

/* Launch the group kernel over nq descriptors (chunk/range bases filled in
 * here).  For nq > 1 the descriptors and bases are copied from the pinned
 * host arrays to the device arrays first, on the same stream. */
/* A group launch replayed from a CUDA graph while its shape is unchanged: the
 * graph resets the barrier counter, copies the descriptors from the pinned
 * host array (rewritten every round) and runs the kernel.  A shape is
 * captured when it comes twice in a row, so launches whose shape keeps
 * changing (a serving loop) pay no capture. */
struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    int shape[10] = {0};     /* shape of `exec` */
    int last[10] = {0};      /* shape of the latest launch */
    bool unsupported = false;
};

cudaError_t launch_group(cudaStream_t stream, int device, int num_sms, QDesc *hd, int nq, QDesc *dd, int *hbase,
                         int *dbase, unsigned long long *bar, unsigned long long *bar_base, unsigned long long *trace,
                         int64_t trace_slots, bool front_any, GraphCache *gc = nullptr) {
    GroupArgs ga;
    memset(&ga, 0, sizeof(ga));
    int C_tot = 0, R_tot = 0, maxP = 1, maxC = 1, tcap = 4, maxS = 4;
    bool replace_all = true;
    for (int i = 0; i < nq; i++) {
        QDesc &d = hd[i];
        d.chunk_base = C_tot;
        d.range_base = R_tot;
        if (hbase) {
            hbase[i] = C_tot;
            hbase[nq + 1 + i] = R_tot;
        }
        C_tot += d.C;
        R_tot += d.R;
        if (d.P > maxP) maxP = d.P;
        if (d.C > maxC) maxC = d.C;
        if (d.S > maxS) maxS = (int)d.S;
        if (!(d.flags & QF_REPLACE)) replace_all = false;
        const int t = (d.ppp << d.rbits);
        if (t > tcap) tcap = t;
    }
    if (hbase) {
        hbase[nq] = C_tot;
        hbase[2 * nq + 1] = R_tot;
    }
    tcap = (tcap + 3) / 4 * 4;
    const int dcap = 8192;
    /* a single query streams its chunks through two input sets when that
       keeps two CTAs on every SM */
    const void *fn = group_kernel_ptr(front_any);
    cudaError_t e = cudaSuccess;
    bool dbuf = false;
    int64_t smem = group_smem_bytes(maxP, maxC, maxS, tcap, dcap, front_any, nq, false, replace_all);
    int occ = 0;
    if (nq == 1) {
        const int64_t smem2 = group_smem_bytes(maxP, maxC, maxS, tcap, dcap, front_any, nq, true, replace_all);
        if (smem2 <= 227 * 1024) {
            e = raise_dyn_smem(fn, (int)smem2);
            if (e != cudaSuccess) return e;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kGThreads, (size_t)smem2);
            if (e != cudaSuccess) return e;
            if (occ >= 2) {
                dbuf = true;
                smem = smem2;
            }
        }
    }
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    e = raise_dyn_smem(fn, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kGThreads, (size_t)smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    int grid = group_grid(device, num_sms);
    if (grid > occ * num_sms) grid = occ * num_sms;
    const int work = C_tot > R_tot ? C_tot : R_tot;
    if (grid > work) grid = work;
    if (grid < 1) grid = 1;
    if (nq == 1) {
        ga.q0 = hd[0];
    } else {
        ga.qs = dd;
        ga.chunk_base = dbase;
        ga.range_base = dbase + nq + 1;
    }
    ga.nq = nq;
    ga.C_tot = C_tot;
    ga.R_tot = R_tot;
    ga.grid = grid;
    ga.maxP = maxP;
    ga.maxC = maxC;
    ga.tcap = tcap;
    ga.dcap = dcap;
    ga.maxS = maxS;
    ga.dbuf = dbuf ? 1 : 0;
    ga.replace_all = replace_all ? 1 : 0;
    ga.bar = bar;
    ga.trace = (trace && trace_slots >= (int64_t)grid * 8) ? trace : nullptr;
    void *args[] = {&ga};
    if (nq == 1) {   /* single query: monotonic barrier counter, no copies */
        ga.bar_target = *bar_base + (unsigned long long)grid;
        e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kGThreads), args, (size_t)smem, stream);
        if (e != cudaSuccess) return e;
        *bar_base += (unsigned long long)grid;
        return cudaSuccess;
    }
    /* several queries: reset the counter, copy descriptors, run; the counter
     * ends at `grid`, where a following single-query launch counts on */
    ga.bar_target = (unsigned long long)grid;
    *bar_base = (unsigned long long)grid;
    auto enqueue = [&]() -> cudaError_t {
        cudaError_t r = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned long long), stream);   /* barrier, range draws */
        if (r == cudaSuccess) r = cudaMemcpyAsync(dd, hd, sizeof(QDesc) * nq, cudaMemcpyHostToDevice, stream);
        if (r == cudaSuccess)
            r = cudaMemcpyAsync(dbase, hbase, sizeof(int) * 2 * (nq + 1), cudaMemcpyHostToDevice, stream);
        if (r == cudaSuccess)
            r = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kGThreads), args, (size_t)smem, stream);
        return r;
    };
    if (!gc || gc->unsupported || ga.trace) return enqueue();
    const int shape[10] = {nq, C_tot, R_tot, maxP, maxC, tcap, dcap, (int)front_any + 2 * (int)replace_all, grid,
                           (int)smem + (maxS << 18)};
    const bool repeated = memcmp(shape, gc->last, sizeof(shape)) == 0;
    memcpy(gc->last, shape, sizeof(shape));
    if (gc->exec && memcmp(shape, gc->shape, sizeof(shape)) == 0) return cudaGraphLaunch(gc->exec, stream);
    if (!repeated) return enqueue();
    {
        if (gc->exec) {
            cudaGraphExecDestroy(gc->exec);
            gc->exec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t r = enqueue();
            e = cudaStreamEndCapture(stream, &graph);
            if (r != cudaSuccess) e = r;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&gc->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {   /* capture not available: launch directly from now on */
            cudaGetLastError();
            gc->exec = nullptr;
            gc->unsupported = true;
            return enqueue();
        }
        memcpy(gc->shape, shape, sizeof(shape));
    }
    return cudaGraphLaunch(gc->exec, stream);
}

/* Whether the latest launch of `gc` was a graph replay or capture. */
bool graph_used(const GraphCache &gc) {
    return gc.exec && !gc.unsupported && memcmp(gc.shape, gc.last, sizeof(gc.shape)) == 0;
}

/* Where a group push sends a member's flip: a side stream, after the work
 * already on the query's stream (`pre` is recorded there), with `done`
 * recorded after it; `used` tells the caller that a flip went there. */
struct FlipRoute {
    cudaStream_t s;
    cudaEvent_t pre, done;
    bool used;
};

/* Host bookkeeping of a push of n tuples (flips are launched here, on the
 * query's stream or the route's side stream); fills the per-launch
 * arguments. */
cudaError_t prepare_push(cq_query *q, const int32_t *k_eff, const int32_t *v_eff, int64_t n, IngestArgs *a,
                         FlipRoute *route = nullptr) {
    const int64_t W = q->W, N = q->N;
    const int64_t n_eff = n < W ? n : W;
    const int64_t skip = n - n_eff;
    const int64_t H = N > W ? N - W : 0;
    const int64_t Hn = N + n > W ? N + n - W : 0;
    memset(a, 0, sizeof(*a));
    a->keys = k_eff;
    a->vals = v_eff;
    a->n = n_eff;
    a->slot0 = (N + skip) % W;
    a->hmod = H % W;
    a->old_len = N - H;
    a->fa = a->fb = 0;
    a->minmax = q->minmax;
    if (q->minmax) {
        if (Hn <= q->F) {
            a->fa = 0;
            a->fb = Hn - H;
        } else if (Hn >= N) {
            bump_epoch(q);
            q->F = Hn;
            q->resets++;
        } else {
            bump_epoch(q);
            cudaStream_t fs = q->stream;
            cudaError_t e = cudaSuccess;
            if (route) {
                fs = route->s;
                e = cudaEventRecord(route->pre, q->stream);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(fs, route->pre, 0);
                if (e != cudaSuccess) return e;
            }
            e = launch_flip(q->d, q->F % W, N - q->F, q->epoch, fs, &q->launches);
            if (e == cudaSuccess && route) {
                e = cudaEventRecord(route->done, fs);
                route->used = true;
            }
            if (e != cudaSuccess) return e;
            a->fa = q->F - H;
            a->fb = Hn - H;
            q->F = N;
            q->flips++;
        }
    }
    a->epoch = q->epoch;
    return cudaSuccess;
}

void commit_push(cq_query *q, int64_t n, int path) {
    q->N += n;
    q->pushes++;
    q->last_path = path;
    if (path == 1 || path == 3) q->hot_parity ^= 1;   /* the partitioned paths rotate the hot lists */
}

/* One push; (k_eff, v_eff) point at the last min(n, W) tuples of the batch. */
cq_status push_impl(cq_query *q, const int32_t *k_eff, const int32_t *v_eff, int64_t n) {
    IngestArgs a;
    cudaError_t e = prepare_push(q, k_eff, v_eff, n, &a);
    if (e != cudaSuccess) return fail_prepared(q, e);
    const bool front = q->minmax && a.fb > a.fa;
    int path = 2;
    bool wide = false;
    if (q->opt.path == 0 || q->opt.path == 1) {
        GPlan gp;
        const int grid = group_grid(q->device, q->num_sms);
        const bool replace = a.n == q->W && a.old_len > 0;
        if (group_plan(q, a.n, a.keys, a.vals, a.slot0, grid, true, &gp, replace) &&
            !(wide = prefer_wide_ranges(q, gp, a.n))) {
            QDesc dsc;
            e = group_desc(q, a, gp, front, 8, &dsc);
            if (e == cudaSuccess)
                e = launch_group(q->stream, q->device, q->num_sms, &dsc, 1, nullptr, nullptr, nullptr, q->d.bar,
                                 &q->bar_base, q->trace, q->trace_slots, front);
            if (e != cudaSuccess) return fail_prepared(q, e);
            path = 3;
            q->launches += 1;
        }
    }
    if (path == 2 && q->opt.path != 2) {
        PushPlan plan;
        if (make_plan(q, a.n, front, false, &plan, wide)) {
            e = launch_partitioned(q, a, plan, front);
            if (e != cudaSuccess) return fail_prepared(q, e);
            path = 1;
            q->launches += 1;
        }
    }
    if (path == 2) {
        e = launch_ingest(q->d, a, q->opt, q->num_sms, q->stream);
        if (e == cudaSuccess) e = launch_finalize(q->d, q->epoch, q->minmax, q->avg, q->num_sms, q->stream);
        if (e != cudaSuccess) return fail_prepared(q, e);
        q->launches += 2;
    }
    commit_push(q, n, path);
    return CQ_OK;
}

}  // namespace

extern "C" {

int64_t cq_footprint_bytes(int64_t groups, int64_t window, uint32_t aggs) {
    if (groups < 1 || groups > kMaxGroups || window < 1 || window > kMaxSize) return -1;
    int minmax = (aggs & (CQ_MIN | CQ_MAX)) != 0;
    int64_t b = 8 * window;                    /* ring */
    b += pad16(groups) * (8 + 4 + 4 + 4 + 8);  /* sum, count, min, max, avg */
    b += pad16(groups);                        /* touched */
    /* heavy-hitter lists, accumulators, flags */
    b += 8 * 4 * kMaxHot + (int64_t)sizeof(HotAcc) * kHotRep * (kMaxHot + kEmSlots) + 4 * kEmSlots + 8 + 64;
    if (minmax) {
        b += 40 * pad16(groups) + 8 * window;  /* tags, front pointers and departures, sorted suffixes */
        b += flip_scratch_bytes(window, groups);
    }
    return b;
}

cq_status cq_create(int64_t groups, int64_t window, uint32_t aggs, void *cuda_stream, cq_query **out) {
    if (!out) return CQ_EINVAL;
    *out = nullptr;
    if (groups < 1 || groups > kMaxGroups || window < 1 || window > kMaxSize) return CQ_EINVAL;
    if (aggs == 0 || (aggs & ~(uint32_t)CQ_ALL)) return CQ_EINVAL;
    cq_query *q = new (std::nothrow) cq_query();
    if (!q) return CQ_ENOMEM;
    q->G = groups;
    q->W = window;
    q->aggs = aggs;
    q->minmax = (aggs & (CQ_MIN | CQ_MAX)) != 0;
    q->avg = (aggs & CQ_AVG) != 0;
    cudaError_t e = cudaGetDevice(&q->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&q->num_sms, cudaDevAttrMultiProcessorCount, q->device);
    if (e == cudaSuccess) {
        if (cuda_stream) {
            q->stream = (cudaStream_t)cuda_stream;
        } else {
            e = cudaStreamCreateWithFlags(&q->stream, cudaStreamNonBlocking);
            q->own_stream = e == cudaSuccess;
        }
    }
    DeviceState &d = q->d;
    d.G = groups;
    d.W = window;
    d.Gpad = pad16(groups);
    if (e == cudaSuccess) e = dmalloc(q, &d.ring_k, window);
    if (e == cudaSuccess) e = dmalloc(q, &d.ring_v, window);
    if (e == cudaSuccess) e = dmalloc(q, &d.sum, d.Gpad);
    if (e == cudaSuccess) e = dmalloc(q, &d.cnt, d.Gpad);
    if (e == cudaSuccess) e = dmalloc(q, &d.rmin, d.Gpad);
    if (e == cudaSuccess) e = dmalloc(q, &d.rmax, d.Gpad);
    if (e == cudaSuccess) e = dmalloc(q, &d.ravg, d.Gpad);
    if (e == cudaSuccess) e = dmalloc(q, &d.touched, d.Gpad);
    if (e == cudaSuccess) e = dmalloc(q, &d.err, 1);
    if (e == cudaSuccess) e = dmalloc(q, &d.hotlist, 4 * kMaxHot);
    if (e == cudaSuccess) e = dmalloc(q, &d.hotlist_n, 4);
    if (e == cudaSuccess) e = dmalloc(q, &d.hotlist_cnt, 4 * kMaxHot);
    if (e == cudaSuccess) e = dmalloc(q, (HotAcc **)&d.hotacc, (int64_t)kHotRep * kMaxHot);
    if (e == cudaSuccess) e = dmalloc(q, &d.emkey, kEmSlots);
    if (e == cudaSuccess) e = dmalloc(q, (HotAcc **)&d.emacc, (int64_t)kHotRep * kEmSlots);
    if (e == cudaSuccess) e = dmalloc(q, &d.emfolds, 1);
    if (e == cudaSuccess) e = dmalloc(q, &d.bar, 2);
    if (e == cudaSuccess) e = dmalloc(q, &q->bad, 1);
    if (q->minmax) {
        if (e == cudaSuccess) e = dmalloc(q, &d.bmin, d.Gpad);
        if (e == cudaSuccess) e = dmalloc(q, &d.bmax, d.Gpad);
        if (e == cudaSuccess) e = dmalloc(q, &d.fmin, d.Gpad);
        if (e == cudaSuccess) e = dmalloc(q, &d.fmax, d.Gpad);
        if (e == cudaSuccess) e = dmalloc(q, &d.sufs, window);
        if (e == cudaSuccess) e = dmalloc(q, &d.fptr, d.Gpad);
        if (e == cudaSuccess) e = dmalloc(q, &d.fdep, d.Gpad);
        if (e == cudaSuccess) e = cudaMemsetAsync(d.fdep, 0, sizeof(int32_t) * d.Gpad, q->stream);
        if (e == cudaSuccess) {
            e = flip_alloc(d, q->stream);
            if (e == cudaSuccess) q->device_bytes += flip_scratch_bytes(window, groups);
        }
    }
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&q->h_err, sizeof(int), cudaHostAllocMapped);
    if (e == cudaSuccess) {
        *(volatile int *)q->h_err = 0;
        e = cudaHostGetDevicePointer((void **)&d.err_host, q->h_err, 0);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(d.touched, 0, (size_t)d.Gpad, q->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.err, 0, sizeof(int), q->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.hotlist_n, 0, 4 * sizeof(int), q->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.bar, 0, 2 * sizeof(unsigned long long), q->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(q->bad, 0, sizeof(int), q->stream);
    for (int r = 0; r < kHotRep && e == cudaSuccess; r++)
        e = cudaMemcpyAsync((HotAcc *)d.hotacc + (int64_t)r * kMaxHot, hot_acc_identity(), sizeof(HotAcc) * kMaxHot,
                            cudaMemcpyHostToDevice, q->stream);
    for (int r = 0; r < kHotRep && e == cudaSuccess; r++)
        e = cudaMemcpyAsync((HotAcc *)d.emacc + (int64_t)r * kEmSlots, hot_acc_identity(), sizeof(HotAcc) * kEmSlots,
                            cudaMemcpyHostToDevice, q->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.emkey, 0xFF, sizeof(int32_t) * kEmSlots, q->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.emfolds, 0, sizeof(unsigned long long), q->stream);
    if (e == cudaSuccess) e = launch_init_state(d, q->minmax, q->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(q->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_all(q);
        delete q;
        return cuda_status(e);
    }
    *out = q;
    return CQ_OK;
}

cq_status cq_push(cq_query *q, const int32_t *d_keys, const int32_t *d_vals, int64_t n) {
    if (!q) return CQ_EINVAL;
    cq_status st = poison_status(q);
    if (st != CQ_OK) return st;
    if (n < 0) return CQ_EINVAL;
    if (n == 0) return CQ_OK;
    if (!d_keys || !d_vals) return CQ_EINVAL;
    set_device(q);
    int64_t skip = n > q->W ? n - q->W : 0;
    return push_impl(q, d_keys + skip, d_vals + skip, n);
}

cq_status cq_push_host(cq_query *q, const int32_t *h_keys, const int32_t *h_vals, int64_t n) {
    if (!q) return CQ_EINVAL;
    cq_status st = poison_status(q);
    if (st != CQ_OK) return st;
    if (n < 0) return CQ_EINVAL;
    if (n == 0) return CQ_OK;
    if (!h_keys || !h_vals) return CQ_EINVAL;
    set_device(q);
    int64_t n_eff = n < q->W ? n : q->W;
    int64_t skip = n - n_eff;
    cudaError_t e = cudaSuccess;
    if (!q->h2d) {
        e = cudaStreamCreateWithFlags(&q->h2d, cudaStreamNonBlocking);
        for (int b = 0; b < 2 && e == cudaSuccess; b++) {
            e = cudaEventCreateWithFlags(&q->ev_staged[b], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&q->ev_consumed[b], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return cuda_status(e);
    }
    if (q->stage_cap < n_eff) {   /* growing: both slots idle first */
        e = cudaStreamSynchronize(q->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(q->h2d);
        if (e != cudaSuccess) return cuda_status(e);
        for (int b = 0; b < 2; b++) {
            cudaFree(q->stage_k[b]);
            cudaFree(q->stage_v[b]);
            q->stage_k[b] = q->stage_v[b] = nullptr;
        }
        q->stage_cap = 0;
        for (int b = 0; b < 2 && e == cudaSuccess; b++) {
            e = cudaMalloc((void **)&q->stage_k[b], sizeof(int32_t) * n_eff);
            if (e == cudaSuccess) e = cudaMalloc((void **)&q->stage_v[b], sizeof(int32_t) * n_eff);
            if (e == cudaSuccess) e = cudaEventRecord(q->ev_consumed[b], q->stream);
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            for (int b = 0; b < 2; b++) {
                cudaFree(q->stage_k[b]);
                cudaFree(q->stage_v[b]);
                q->stage_k[b] = q->stage_v[b] = nullptr;
            }
            return CQ_ENOMEM;
        }
        q->stage_cap = n_eff;
    }
    /* the slot's previous batch has been pushed; copy this one up on the copy
       stream (it overlaps the pushes and result reads before it); the push waits */
    const int sl = q->stage_slot;
    q->stage_slot ^= 1;
    e = cudaStreamWaitEvent(q->h2d, q->ev_consumed[sl], 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(q->stage_k[sl], h_keys + skip, sizeof(int32_t) * n_eff, cudaMemcpyHostToDevice, q->h2d);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(q->stage_v[sl], h_vals + skip, sizeof(int32_t) * n_eff, cudaMemcpyHostToDevice, q->h2d);
    if (e == cudaSuccess) e = cudaEventRecord(q->ev_staged[sl], q->h2d);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(q->stream, q->ev_staged[sl], 0);
    if (e != cudaSuccess) return cuda_status(e);
    const cq_status pst = push_impl(q, q->stage_k[sl], q->stage_v[sl], n);
    e = cudaEventRecord(q->ev_consumed[sl], q->stream);
    if (pst != CQ_OK) return pst;
    return e == cudaSuccess ? CQ_OK : cuda_status(e);
}

cq_status cq_sync(cq_query *q) {
    if (!q) return CQ_EINVAL;
    set_device(q);
    cudaError_t e = cudaStreamSynchronize(q->stream);
    if (e != cudaSuccess) return cuda_status(e);
    return poison_status(q);
}

cq_status cq_results(cq_query *q, cq_result_view *out) {
    if (!q || !out) return CQ_EINVAL;
    cq_status st = cq_sync(q);
    if (st != CQ_OK) return st;
    out->groups = q->G;
    out->sum = (const int64_t *)q->d.sum;
    out->count = q->d.cnt;
    out->min = q->d.rmin;
    out->max = q->d.rmax;
    out->avg = q->d.ravg;
    return CQ_OK;
}

cq_status cq_results_copy_async(cq_query *q, int64_t *h_sum, int32_t *h_count, int32_t *h_min, int32_t *h_max,
                                double *h_avg) {
    if (!q) return CQ_EINVAL;
    cq_status st = poison_status(q);
    if (st != CQ_OK) return st;
    set_device(q);
    const size_t G = (size_t)q->G;
    cudaError_t e = cudaSuccess;
    if (h_sum && e == cudaSuccess) e = cudaMemcpyAsync(h_sum, q->d.sum, 8 * G, cudaMemcpyDeviceToHost, q->stream);
    if (h_count && e == cudaSuccess) e = cudaMemcpyAsync(h_count, q->d.cnt, 4 * G, cudaMemcpyDeviceToHost, q->stream);
    if (h_min && e == cudaSuccess) e = cudaMemcpyAsync(h_min, q->d.rmin, 4 * G, cudaMemcpyDeviceToHost, q->stream);
    if (h_max && e == cudaSuccess) e = cudaMemcpyAsync(h_max, q->d.rmax, 4 * G, cudaMemcpyDeviceToHost, q->stream);
    if (h_avg && e == cudaSuccess) e = cudaMemcpyAsync(h_avg, q->d.ravg, 8 * G, cudaMemcpyDeviceToHost, q->stream);
    return e == cudaSuccess ? CQ_OK : cuda_status(e);
}

cq_status cq_results_copy(cq_query *q, int64_t *h_sum, int32_t *h_count, int32_t *h_min, int32_t *h_max,
                          double *h_avg) {
    if (!q) return CQ_EINVAL;
    cq_status st = poison_status(q);
    if (st != CQ_OK) return st;
    set_device(q);
    const size_t G = (size_t)q->G;
    cudaError_t e = cudaSuccess;
    if (h_sum && e == cudaSuccess) e = cudaMemcpyAsync(h_sum, q->d.sum, 8 * G, cudaMemcpyDeviceToHost, q->stream);
    if (h_count && e == cudaSuccess) e = cudaMemcpyAsync(h_count, q->d.cnt, 4 * G, cudaMemcpyDeviceToHost, q->stream);
    if (h_min && e == cudaSuccess) e = cudaMemcpyAsync(h_min, q->d.rmin, 4 * G, cudaMemcpyDeviceToHost, q->stream);
    if (h_max && e == cudaSuccess) e = cudaMemcpyAsync(h_max, q->d.rmax, 4 * G, cudaMemcpyDeviceToHost, q->stream);
    if (h_avg && e == cudaSuccess) e = cudaMemcpyAsync(h_avg, q->d.ravg, 8 * G, cudaMemcpyDeviceToHost, q->stream);
    if (e != cudaSuccess) return cuda_status(e);
    return cq_sync(q);
}

void cq_destroy(cq_query *q) {
    if (!q) return;
    set_device(q);
    if (q->stream) cudaStreamSynchronize(q->stream);
    free_all(q);
    delete q;
}

const char *cq_strerror(cq_status s) {
    switch (s) {
        case CQ_OK: return "ok";
        case CQ_EINVAL: return "invalid argument";
        case CQ_ENOMEM: return "out of memory";
        case CQ_EKEY: return "key outside [0, groups); query poisoned";
        case CQ_ECUDA: return "CUDA runtime error";
        case CQ_ETIMEOUT: return "bounded device wait timed out";
        case CQ_EBUSY: return "resource busy";
        case CQ_EPOISONED: return "query poisoned by an earlier bad key";
        case CQ_EBUDGET: return "device-memory budget exhausted";
        case CQ_ESCRATCH: return "batch needs more scratch than the fixed no-allocation area holds";
    }
    return "unknown status";
}

cq_status cq_set_option(cq_query *q, cq_option opt, int64_t v) {
    if (!q) return CQ_EINVAL;
    switch (opt) {
        case CQ_OPT_HOT_KEYS:
            if (v < 0 || v > kMaxHot) return CQ_EINVAL;
            if (v != q->opt.hot_keys) {
                /* the lists were written under the old cap: start empty */
                cudaError_t e = cudaMemsetAsync(q->d.hotlist_n, 0, 4 * sizeof(int), q->stream);
                if (e != cudaSuccess) return cuda_status(e);
            }
            q->opt.hot_keys = (int)v;
            return CQ_OK;
        case CQ_OPT_HOT_THRESHOLD:
            if (v < 0 || v > kMaxSize) return CQ_EINVAL;
            q->opt.hot_threshold = (int)v;
            return CQ_OK;
        case CQ_OPT_WARP_AGG:
            if (v != 0 && v != 1) return CQ_EINVAL;
            q->opt.warp_agg = (int)v;
            return CQ_OK;
        case CQ_OPT_CTAS_PER_SM:
            if (v < 1 || v > 8) return CQ_EINVAL;
            q->opt.ctas_per_sm = (int)v;
            return CQ_OK;
        case CQ_OPT_PARTITION_BITS:
            if (v < 0 || v > kMaxRBits) return CQ_EINVAL;
            q->opt.partition_bits = (int)v;
            return CQ_OK;
        case CQ_OPT_PATH:
            if (v < 0 || v > 3) return CQ_EINVAL;
            q->opt.path = (int)v;
            return CQ_OK;
        case CQ_OPT_WAIT_LIMIT_US:
            if (v < 1 || v > 60000000) return CQ_EINVAL;
            q->sm.wait_us = v;
            return CQ_OK;
        case CQ_OPT_STALL_BATCH:
            if (v < -1 || v >= kSMaxBatches) return CQ_EINVAL;
            q->sm.stall_batch = (int)v;
            return CQ_OK;
        case CQ_OPT_STREAM_PRODUCERS:
            if (v < -1 || v > 4096) return CQ_EINVAL;
            q->sm.pp_opt = (int)v;
            return CQ_OK;
    }
    return CQ_EINVAL;
}

cq_status cq_get_option(const cq_query *q, cq_option opt, int64_t *v) {
    if (!q || !v) return CQ_EINVAL;
    switch (opt) {
        case CQ_OPT_HOT_KEYS: *v = q->opt.hot_keys; return CQ_OK;
        case CQ_OPT_HOT_THRESHOLD: *v = q->opt.hot_threshold; return CQ_OK;
        case CQ_OPT_WARP_AGG: *v = q->opt.warp_agg; return CQ_OK;
        case CQ_OPT_CTAS_PER_SM: *v = q->opt.ctas_per_sm; return CQ_OK;
        case CQ_OPT_PARTITION_BITS: *v = q->opt.partition_bits; return CQ_OK;
        case CQ_OPT_PATH: *v = q->opt.path; return CQ_OK;
        case CQ_OPT_WAIT_LIMIT_US: *v = q->sm.wait_us; return CQ_OK;
        case CQ_OPT_STALL_BATCH: *v = q->sm.stall_batch; return CQ_OK;
        case CQ_OPT_STREAM_PRODUCERS: *v = q->sm.pp_opt; return CQ_OK;
    }
    return CQ_EINVAL;
}

cq_status cq_trace(cq_query *q, uint64_t *d_stamps, int64_t slots) {
    if (!q || slots < 0 || (d_stamps && slots == 0)) return CQ_EINVAL;
    q->trace = (unsigned long long *)d_stamps;
    q->trace_slots = d_stamps ? slots : 0;
    return CQ_OK;
}


cq_status cq_autotune(cq_query *q, const int32_t *d_keys, const int32_t *d_vals, int64_t n, int trials,
                      double *best_us) {
    if (!q || n <= 0 || !d_keys || !d_vals || trials < 1 || trials > 1000) return CQ_EINVAL;
    cq_status st = poison_status(q);
    if (st != CQ_OK) return st;
    set_device(q);
    cudaError_t e = cudaStreamSynchronize(q->stream);
    if (e != cudaSuccess) return cuda_status(e);
    /* candidate settings around the automatic choice */
    int r_auto = 2;
    while (r_auto <= 10 && ((q->G + ((int64_t)1 << r_auto) - 1) >> r_auto) > kGMaxParts) r_auto++;
    struct Cand {
        int path, rbits, hot_keys, hot_thr, cps;
    } cands[32];
    int nc = 0;
    const int thr_auto = 0;
    const int64_t n_eff = n < q->W ? n : q->W;
    /* a path the caller pinned (CQ_OPT_PATH != 0) is kept: a query pushed
       in group launches is tuned for the group kernel only (path 1) */
    const int paths[2] = {q->opt.path != 0 ? q->opt.path : 0, 3};
    const int npaths = q->opt.path != 0 ? 1 : 2;
    for (int pi = 0; pi < npaths; pi++)
        for (int dr : {0, 1, 2})
            for (int hk : {0, 128})
                for (int quarter : {0, 1}) {
                    if (hk == 0 && quarter) continue;
                    const int r = dr == 0 ? 0 : r_auto + dr;
                    if (r > 11) continue;
                    int thr = thr_auto;
                    if (quarter) {
                        int64_t P = (q->G + ((int64_t)1 << (r ? r : r_auto)) - 1) >> (r ? r : r_auto);
                        int64_t t = n_eff / (4 * (P > 0 ? P : 1));
                        thr = (int)(t < 16 ? 16 : t);
                    }
                    cands[nc++] = Cand{paths[pi], r, hk, thr, q->opt.ctas_per_sm};
                    /* the register-staged kernel also at one CTA per SM
                       (its whole shared memory for larger key ranges) */
                    if (paths[pi] == 3 && q->opt.ctas_per_sm != 1) cands[nc++] = Cand{paths[pi], r, hk, thr, 1};
                }
    cq_query *shadow = nullptr;
    double best = 1e30;
    int bi = -1;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int c = 0; c < nc && e == cudaSuccess; c++) {
        st = cq_create(q->G, q->W, q->aggs, nullptr, &shadow);
        if (st != CQ_OK) break;
        shadow->opt = q->opt;
        shadow->opt.path = cands[c].path;
        shadow->opt.partition_bits = cands[c].rbits;
        shadow->opt.hot_keys = cands[c].hot_keys;
        shadow->opt.hot_threshold = cands[c].hot_thr;
        shadow->opt.ctas_per_sm = cands[c].cps;
        /* two warm-up pushes (the second sees the heavy hitters of the first) */
        st = cq_push(shadow, d_keys, d_vals, n);
        if (st == CQ_OK) st = cq_push(shadow, d_keys, d_vals, n);
        if (st == CQ_OK) e = cudaEventRecord(e0, shadow->stream);
        for (int t = 0; t < trials && st == CQ_OK && e == cudaSuccess; t++) st = cq_push(shadow, d_keys, d_vals, n);
        if (st == CQ_OK && e == cudaSuccess) e = cudaEventRecord(e1, shadow->stream);
        if (st == CQ_OK && e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0;
        if (st == CQ_OK && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        const bool ok = st == CQ_OK && e == cudaSuccess && cq_sync(shadow) == CQ_OK;
        cq_destroy(shadow);
        shadow = nullptr;
        if (!ok) break;
        const double us = 1e3 * ms / trials;
        if (us < best) {
            best = us;
            bi = c;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_status(e);
    if (st != CQ_OK) return st;
    if (bi < 0) return CQ_ECUDA;
    q->opt.path = cands[bi].path;
    q->opt.partition_bits = cands[bi].rbits;
    if (q->opt.hot_keys != cands[bi].hot_keys) cq_set_option(q, CQ_OPT_HOT_KEYS, cands[bi].hot_keys);
    q->opt.hot_threshold = cands[bi].hot_thr;
    q->opt.ctas_per_sm = cands[bi].cps;
    if (best_us) *best_us = best;
    return CQ_OK;
}

cq_status cq_hot_list(const cq_query *q, int32_t *keys, int32_t *counts, int cap, int *n) {
    if (!q || !n || cap < 0 || (cap > 0 && !keys)) return CQ_EINVAL;
    *n = 0;
    if (!q->d.hotlist) return CQ_OK;
    set_device(q);
    const int par = q->hot_parity;
    int tier_n[2] = {0, 0};
    int32_t k[2 * kMaxHot], c[2 * kMaxHot];
    cudaError_t e = cudaMemcpyAsync(tier_n, q->d.hotlist_n + 2 * par, sizeof(tier_n), cudaMemcpyDeviceToHost,
                                    q->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(k, q->d.hotlist + par * 2 * kMaxHot, sizeof(k), cudaMemcpyDeviceToHost, q->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c, q->d.hotlist_cnt + par * 2 * kMaxHot, sizeof(c), cudaMemcpyDeviceToHost, q->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(q->stream);
    if (e != cudaSuccess) return cuda_status(e);
    const int hc = q->opt.hot_keys;
    const int n1 = tier_n[0] < hc ? tier_n[0] : hc;
    const int n2 = tier_n[1] < hc - n1 ? tier_n[1] : hc - n1;
    *n = n1 + n2;
    for (int h = 0; h < n1 + n2 && h < cap; h++) {
        const int at = h < n1 ? h : kMaxHot + (h - n1);
        keys[h] = k[at];
        if (counts) counts[h] = c[at];
    }
    return CQ_OK;
}

cq_status cq_stats(const cq_query *q, cq_query_stats *out) {
    if (!q || !out) return CQ_EINVAL;
    out->tuples_seen = q->N;
    out->window_len = q->N < q->W ? q->N : q->W;
    out->pushes = q->pushes;
    out->flips = q->flips;
    out->resets = q->resets;
    /* the heavy hitters the last push detected (the next push's set), read
       from the device once the query's stream is idle */
    int n_tier[2] = {0, 0};
    if (q->d.hotlist_n) {
        cudaError_t e = cudaMemcpyAsync(n_tier, q->d.hotlist_n + 2 * q->hot_parity, sizeof(n_tier),
                                        cudaMemcpyDeviceToHost, q->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(q->stream);
        if (e != cudaSuccess) return cuda_status(e);
    }
    /* the keys sure of a slot first, then the others up to the cap */
    const int cap = q->opt.hot_keys;
    const int n1 = n_tier[0] < cap ? n_tier[0] : cap;
    out->hot_keys = n1 + (n_tier[1] < cap - n1 ? n_tier[1] : cap - n1);
    out->device_bytes = q->device_bytes;
    unsigned long long folds = 0;
    if (q->d.emfolds) {
        cudaError_t e = cudaMemcpyAsync(&folds, q->d.emfolds, sizeof(folds), cudaMemcpyDeviceToHost, q->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(q->stream);
        if (e != cudaSuccess) return cuda_status(e);
    }
    out->heavy_folds = (int64_t)folds;
    out->kernel_launches = q->launches;
    out->last_path = q->last_path;
    return CQ_OK;
}

}  /* extern "C" */

/* ---- groups ---- */

/* Descriptor buffers of one in-flight group launch: the pinned host copy is
 * rewritten by the host for the launch and read by its copy to the device. */
struct GroupSlot {
    int cap = 0;
    QDesc *h_desc = nullptr, *d_desc = nullptr;
    int *h_base = nullptr, *d_base = nullptr;
    unsigned long long *bar = nullptr;
    unsigned long long bar_base = 0;   /* arrivals on `bar` so far */
    cudaEvent_t ev = nullptr;          /* recorded after the slot's last launch */
    GraphCache graph;
};

constexpr int kFlipStreams = 4;

struct cq_group {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0, num_sms = 148;
    GroupSlot slot[2];                 /* two launches may be in flight */
    int next_slot = 0;
    cudaEvent_t ev = nullptr;          /* recorded after the latest launch */
    int64_t launches = 0, graph_launches = 0;
    /* the members' flips run side by side on these streams, the launch waits
       for them (created at the first group push that flips) */
    cudaStream_t fs[kFlipStreams] = {};
    cudaEvent_t fdone[kFlipStreams] = {};
    cudaEvent_t fpre = nullptr;
};

namespace {

void slot_free(GroupSlot &sl) {
    if (sl.h_desc) cudaFreeHost(sl.h_desc);
    if (sl.h_base) cudaFreeHost(sl.h_base);
    cudaFree(sl.d_desc);
    cudaFree(sl.d_base);
    sl.h_desc = sl.d_desc = nullptr;
    sl.h_base = sl.d_base = nullptr;
    sl.cap = 0;
}

/* Buffers of a slot for nq descriptors (the slot's last launch has finished). */
cudaError_t slot_reserve(GroupSlot &sl, int nq) {
    if (sl.cap >= nq) return cudaSuccess;
    slot_free(sl);
    int cap = 64;
    while (cap < nq) cap *= 2;
    cudaError_t e = cudaHostAlloc((void **)&sl.h_desc, sizeof(QDesc) * cap, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&sl.h_base, sizeof(int) * 2 * (cap + 1), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaMalloc((void **)&sl.d_desc, sizeof(QDesc) * cap);
    if (e == cudaSuccess) e = cudaMalloc((void **)&sl.d_base, sizeof(int) * 2 * (cap + 1));
    if (e == cudaSuccess) sl.cap = cap;
    return e;
}

}  // namespace

extern "C" {

cq_status cqg_create(void *cuda_stream, cq_group **out) {
    if (!out) return CQ_EINVAL;
    *out = nullptr;
    cq_group *g = new (std::nothrow) cq_group();
    if (!g) return CQ_ENOMEM;
    cudaError_t e = cudaGetDevice(&g->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
    if (e == cudaSuccess) {
        if (cuda_stream) {
            g->stream = (cudaStream_t)cuda_stream;
        } else {
            e = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking);
            g->own_stream = e == cudaSuccess;
        }
    }
    for (int i = 0; i < 2 && e == cudaSuccess; i++) {
        GroupSlot &sl = g->slot[i];
        e = cudaMalloc((void **)&sl.bar, 2 * sizeof(unsigned long long));   /* barrier, range draws */
        if (e == cudaSuccess) e = cudaMemsetAsync(sl.bar, 0, sizeof(unsigned long long), g->stream);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(sl.ev, g->stream);
        if (e == cudaSuccess) e = slot_reserve(sl, 64);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cqg_destroy(g);
        return cuda_status(e);
    }
    *out = g;
    return CQ_OK;
}

void cqg_destroy(cq_group *g) {
    if (!g) return;
    if (g->stream) cudaStreamSynchronize(g->stream);
    for (int i = 0; i < 2; i++) {
        GroupSlot &sl = g->slot[i];
        slot_free(sl);
        cudaFree(sl.bar);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.graph.exec) cudaGraphExecDestroy(sl.graph.exec);
    }
    if (g->ev) cudaEventDestroy(g->ev);
    for (int i = 0; i < kFlipStreams; i++) {
        if (g->fs[i]) {
            cudaStreamSynchronize(g->fs[i]);
            cudaStreamDestroy(g->fs[i]);
        }
        if (g->fdone[i]) cudaEventDestroy(g->fdone[i]);
    }
    if (g->fpre) cudaEventDestroy(g->fpre);
    if (g->own_stream && g->stream) cudaStreamDestroy(g->stream);
    delete g;
}

cq_status cqg_stats(const cq_group *g, int64_t *launches, int64_t *graph_launches) {
    if (!g) return CQ_EINVAL;
    if (launches) *launches = g->launches;
    if (graph_launches) *graph_launches = g->graph_launches;
    return CQ_OK;
}

cq_status cqg_sync(cq_group *g) {
    if (!g) return CQ_EINVAL;
    return cuda_status(cudaStreamSynchronize(g->stream));
}

cq_status cqg_push(cq_group *g, int nq, cq_query *const *queries, const int32_t *const *d_keys,
                   const int32_t *const *d_vals, const int64_t *n, cq_status *status) {
    if (!g || nq < 0 || (nq > 0 && (!queries || !d_keys || !d_vals || !n))) return CQ_EINVAL;
    if (nq == 0) return CQ_OK;
    for (int i = 0; i < nq; i++) {
        if (!queries[i] || queries[i]->device != g->device) return CQ_EINVAL;
        for (int j = 0; j < i; j++)
            if (queries[j] == queries[i]) return CQ_EINVAL;
    }
    GroupSlot &sl = g->slot[g->next_slot];
    /* the launch before last used this slot's buffers: wait for it only */
    cudaError_t e = cudaEventSynchronize(sl.ev);
    if (e == cudaSuccess) e = slot_reserve(sl, nq);
    if (e != cudaSuccess) return cuda_status(e);
    struct Item {
        cq_query *q;
        int64_t n;
        IngestArgs a;
        GPlan plan;
        bool front, grouped, wide;
        bool done;     /* launched and committed */
        int flip_on;   /* side stream of the member's flip, or -1 */
    };
    if (!g->fpre) {   /* the side streams of the members' flips */
        int cur = -1;
        if (cudaGetDevice(&cur) == cudaSuccess && cur != g->device) cudaSetDevice(g->device);
        e = cudaEventCreateWithFlags(&g->fpre, cudaEventDisableTiming);
        for (int i = 0; i < kFlipStreams && e == cudaSuccess; i++) {
            e = cudaStreamCreateWithFlags(&g->fs[i], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->fdone[i], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return cuda_status(e);
    }
    int next_fs = 0;
    Item *items = (Item *)malloc(sizeof(Item) * nq);
    if (!items) return CQ_ENOMEM;
    int m = 0;
    bool front_any = false;
    const int grid = group_grid(g->device, g->num_sms);
    cq_status ret = CQ_OK;
    for (int i = 0; i < nq && ret == CQ_OK; i++) {
        cq_query *q = queries[i];
        cq_status st = poison_status(q);
        if (st == CQ_OK && n[i] < 0) st = CQ_EINVAL;
        if (st == CQ_OK && n[i] > 0 && (!d_keys[i] || !d_vals[i])) st = CQ_EINVAL;
        if (status) status[i] = st;
        if (st != CQ_OK || n[i] == 0) continue;
        const int64_t skip = n[i] > q->W ? n[i] - q->W : 0;
        Item &it = items[m];
        it.q = q;
        it.n = n[i];
        /* a flip goes to the next side stream: the members' flips overlap */
        FlipRoute route{g->fs[next_fs], g->fpre, g->fdone[next_fs], false};
        it.done = false;
        e = prepare_push(q, d_keys[i] + skip, d_vals[i] + skip, n[i], &it.a, &route);
        if (e != cudaSuccess) {
            ret = fail_prepared(q, e);
            if (status) status[i] = ret;
            break;
        }
        it.flip_on = route.used ? next_fs : -1;
        if (route.used) next_fs = (next_fs + 1) % kFlipStreams;
        it.front = q->minmax && it.a.fb > it.a.fa;
        it.grouped = q->opt.path <= 1 && group_plan(q, it.a.n, it.a.keys, it.a.vals, it.a.slot0, grid, false, &it.plan);
        it.wide = false;   /* a group launch keeps every member it can take */
        if (it.grouped && it.front) front_any = true;
        m++;
    }
    if (ret == CQ_OK) {
        /* each member's stream waits for its flip, once every flip is out */
        for (int i = 0; i < m && e == cudaSuccess; i++)
            if (items[i].flip_on >= 0) e = cudaStreamWaitEvent(items[i].q->stream, g->fdone[items[i].flip_on], 0);
        /* order after everything already enqueued on the queries' streams */
        for (int i = 0; i < m && e == cudaSuccess; i++) {
            cq_query *q = items[i].q;
            if (q->stream == g->stream || !items[i].grouped) continue;
            if (!q->ev) e = cudaEventCreateWithFlags(&q->ev, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventRecord(q->ev, q->stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(g->stream, q->ev, 0);
        }
        /* members with the most deltas per key range first: their ranges are
           drawn first, and the cheap ones fill in behind them */
        int *order = (int *)malloc(sizeof(int) * (m > 0 ? m : 1));
        if (!order) e = cudaErrorMemoryAllocation;
        int k = 0;
        for (int i = 0; i < m && e == cudaSuccess; i++)
            if (items[i].grouped) order[k++] = i;
        if (e == cudaSuccess)
            std::stable_sort(order, order + k, [&](int x, int y) {
                return items[x].a.n * (int64_t)items[y].plan.R > items[y].a.n * (int64_t)items[x].plan.R;
            });
        for (int j = 0; j < k && e == cudaSuccess; j++) {
            const Item &it = items[order[j]];
            e = group_desc(it.q, it.a, it.plan, it.front, 8, &sl.h_desc[j]);
        }
        free(order);
        if (e == cudaSuccess && k > 0) {
            e = launch_group(g->stream, g->device, g->num_sms, sl.h_desc, k, sl.d_desc, sl.h_base, sl.d_base, sl.bar,
                             &sl.bar_base, items[0].q->trace, items[0].q->trace_slots, front_any, &sl.graph);
            g->launches++;
            if (k > 1 && graph_used(sl.graph)) g->graph_launches++;
        }
        if (e == cudaSuccess) e = cudaEventRecord(sl.ev, g->stream);
        if (e == cudaSuccess) e = cudaEventRecord(g->ev, g->stream);
        g->next_slot ^= 1;
        for (int i = 0; i < m && e == cudaSuccess; i++) {
            cq_query *q = items[i].q;
            if (!items[i].grouped) continue;
            if (q->stream != g->stream) e = cudaStreamWaitEvent(q->stream, g->ev, 0);
            q->launches += 1;
            commit_push(q, items[i].n, 3);
            items[i].done = true;
        }
        /* queries the group kernel cannot take are pushed on their own */
        for (int i = 0; i < m && e == cudaSuccess; i++) {
            if (items[i].grouped) continue;
            cq_query *q = items[i].q;
            const bool front = items[i].front;
            int path = 2;
            PushPlan plan;
            if (q->opt.path != 2 && make_plan(q, items[i].a.n, front, false, &plan, items[i].wide)) {
                e = launch_partitioned(q, items[i].a, plan, front);
                path = 1;
                q->launches += 1;
            } else {
                e = launch_ingest(q->d, items[i].a, q->opt, q->num_sms, q->stream);
                if (e == cudaSuccess)
                    e = launch_finalize(q->d, q->epoch, q->minmax, q->avg, q->num_sms, q->stream);
                q->launches += 2;
            }
            if (e == cudaSuccess) {
                commit_push(q, items[i].n, path);
                items[i].done = true;
            }
        }
        if (e != cudaSuccess) ret = cuda_status(e);
    }
    /* members prepared but not launched are left inconsistent: poisoned */
    if (ret != CQ_OK)
        for (int i = 0; i < m; i++)
            if (!items[i].done) {
                fail_prepared(items[i].q, e);
                if (status)
                    for (int j = 0; j < nq; j++)
                        if (queries[j] == items[i].q) status[j] = (cq_status)items[i].q->poison;
            }
    free(items);
    return ret;
}

}  /* extern "C" */

/* ---- hooks of the serving loop ---- */

namespace cq {

int64_t group_scratch_bound(int64_t groups, int64_t window, int64_t max_batch) {
    if (groups < 1 || window < 1 || max_batch < 1) return -1;
    int r = 2;
    while (r <= 10 && ((groups + ((int64_t)1 << r) - 1) >> r) > kGMaxParts) r++;
    if (r > 10) return -1;
    const int64_t P = (groups + ((int64_t)1 << r) - 1) >> r;
    const int64_t n = max_batch < window ? max_batch : window;
    /* a group launch cuts n tuples into at most ceil(n / kGChunk) chunks of at
     * most kGChunk tuples; a chunk region holds 2 deltas a tuple plus the
     * partition padding, 16 bytes a delta at most */
    const int64_t C = (n + kGChunk - 1) / kGChunk;
    return C * (2 * kGChunk + P + 4) * 16 + P * (C + 1) * 8;
}

cudaError_t reserve_group_scratch(cq_query *q, int64_t max_batch) {
    if (group_scratch_bound(q->G, q->W, max_batch) < 0) return cudaErrorInvalidValue;
    int r = 2;
    while (((q->G + ((int64_t)1 << r) - 1) >> r) > kGMaxParts) r++;
    const int64_t P = (q->G + ((int64_t)1 << r) - 1) >> r;
    const int64_t n = max_batch < q->W ? max_batch : q->W;
    const int64_t C = (n + kGChunk - 1) / kGChunk;
    DeviceState &st = q->d;
    set_device(q);
    cudaError_t e = ensure_buffer(q, &st.stage, &st.stage_bytes, C * (2 * kGChunk + P + 4) * 16);
    if (e == cudaSuccess) e = ensure_buffer(q, (void **)&st.off, &st.off_bytes, P * (C + 1) * 8);
    return e;
}

cudaStream_t query_stream(const cq_query *q) { return q->stream; }

void group_disable_graphs(cq_group *g) {
    for (int i = 0; i < 2; i++) g->slot[i].graph.unsupported = true;
}

}  // namespace cq

/* ---- cq_push_many: the persistent multi-batch launch (cq_stream.cu) ----
 *
 * The host does each batch's window bookkeeping (as prepare_push: effective
 * batch, leaving tuples, front and flips), in order, into a list of batch
 * descriptors.  The list is launched as one persistent launch whenever a
 * flip is due (the flip is launched between two launches, on the query's
 * stream), when it is full, and at the end. */

namespace {

/* Key ranges of the persistent launch: R ranges (one per consumer), key k in
 * range __umulhi(k, M), tcap the largest range. */
struct SRanges {
    int R = 0;
    uint32_t M = 1;
    int tcap = 0;
};

SRanges stream_ranges(int64_t G, int nB) {
    SRanges r;
    r.R = (int)std::min<int64_t>(nB, G);
    unsigned long long m = ((unsigned long long)r.R << 32) / (unsigned long long)G;
    if (m > 0xFFFFFFFFull) m = 0xFFFFFFFFull;
    if (m < 1) m = 1;
    r.M = (uint32_t)m;
    for (int i = 0; i < r.R; i++) {
        const int64_t w = stream_range_lo((uint32_t)i + 1, r.M, G) - stream_range_lo((uint32_t)i, r.M, G);
        if (w > r.tcap) r.tcap = (int)w;
    }
    return r;
}

/* Tuples per chunk of a batch of n_eff tuples: two chunks per producer,
 * within [kSMinChunk, cap], a multiple of 4. */
int64_t stream_chunk(int64_t n_eff, int nA, int cap) {
    int64_t S = (n_eff + 2 * nA - 1) / (2 * (int64_t)nA);
    S = (S + 3) / 4 * 4;
    if (S < kSMinChunk) S = kSMinChunk;
    if (S > cap) S = cap;
    return S;
}

int g_stream_ok[kMaxDevices];   /* 0 unknown, 1 launchable, -1 not (per device) */
std::mutex g_stream_mu;

/* Whether cq_push_many can take the persistent launch for these batches:
 * automatic path, two launch CTAs per SM, and a consumer's key range that
 * fits its shared memory in the most demanding mode (old tuples read) with
 * the run-table row these batches need. */
bool stream_supported(cq_query *q, const SRanges &rg, int k, const int64_t *n, int nA) {
    if (q->opt.path != 0 || rg.R < 1 || q->device < 0 || q->device >= kMaxDevices) return false;
    if (nA > 1024 || q->num_sms > kSSmSlots) return false;   /* the launch's per-producer flags and SM counts */
    {
        std::lock_guard<std::mutex> lock(g_stream_mu);
        int &ok = g_stream_ok[q->device];
        if (ok == 0) ok = stream_launchable() ? 1 : -1;
        if (ok < 0) return false;
    }
    const int ds = 8;
    const int cap = stream_max_chunk(rg.R, true, ds);
    if (cap < kSMinChunk) return false;
    int64_t cmax = 1;
    for (int j = 0; j < k; j++) {
        const int64_t ne = n[j] < q->W ? n[j] : q->W;
        if (ne <= 0) continue;
        const int64_t S = stream_chunk(ne, nA, cap);
        const int64_t C = (ne + S - 1) / S;
        if (C > cmax) cmax = C;
    }
    const int Cpad = (int)((cmax + 1) & ~1);
    return rg.tcap <= stream_max_range(Cpad, 1024, ds, q->minmax != 0);
}

/* Batches gathered for one launch. */
struct ManySeg {
    std::vector<SBatch> b;
    std::vector<int64_t> first;   /* stream index of each batch's first effective tuple */
    std::vector<int64_t> end;     /* stream index after its last tuple */
    int call_index = 0;           /* the call's index of the launch's first batch */
    uint32_t epoch0 = 0;
};

/* Launch the gathered batches; the list is emptied. */
cudaError_t stream_flush(cq_query *q, ManySeg &sg, const SRanges &rg, const cq_many_out *out, int k, int nA,
                         int nB) {
    const int nb = (int)sg.b.size();
    if (nb == 0) return cudaSuccess;
    auto &sm = q->sm;
    bool ring_any = false;
    for (const SBatch &b : sg.b)
        if (b.flags & SB_RING) ring_any = true;
    const int ds = 8;
    const int cap = stream_max_chunk(rg.R, ring_any, ds);
    int64_t smax = 4, cmax = 1;
    for (SBatch &b : sg.b) {
        if (b.n <= 0) {
            b.S = kSMinChunk;
            b.C = 0;
            continue;
        }
        const int64_t S = stream_chunk(b.n, nA, cap);
        b.S = (int32_t)S;
        b.C = (int32_t)((b.n + S - 1) / S);
        if (S > smax) smax = S;
        if (b.C > cmax) cmax = b.C;
    }
    const int Cpad = (int)((cmax + 1) & ~1);
    /* the gather round: as many deltas as the consumer's shared memory holds
       beside its range (at most 8192, a multiple of 256), so that a batch's
       runs come in as few rounds as possible */
    int dcap = 8192;
    while (dcap > 1024 && stream_max_range(Cpad, dcap, ds, q->minmax != 0) < rg.tcap) dcap -= 256;
    if (stream_max_range(Cpad, dcap, ds, q->minmax != 0) < rg.tcap) return cudaErrorInvalidConfiguration;
    if (stream_smem_bytes((int)smax, rg.R, rg.tcap, Cpad, dcap, ring_any, ds, q->minmax != 0) < 0)
        return cudaErrorInvalidConfiguration;
    const int64_t stride = ((ring_any ? 2 : 1) * smax + rg.R + 2 + 1) & ~1LL;
    const int64_t stage_slot = cmax * stride;
    const int64_t pairs_slot = (int64_t)rg.R * Cpad;
    const int64_t ctl_words = SC_END;
    const int64_t list_n_bytes = (int64_t)kSListN * 2 * sizeof(int);
    cudaError_t e = ensure_buffer(q, &sm.stage, &sm.stage_bytes, kSSlots * stage_slot * ds);
    if (e == cudaSuccess) e = ensure_buffer(q, &sm.pairs, &sm.pairs_bytes, kSSlots * pairs_slot * 8);
    if (e == cudaSuccess && !sm.hotpart)
        e = dmalloc(q, &sm.hotpart, (int64_t)kSSlots * 2 * q->num_sms * kMaxHot);   /* up to two producers an SM */
    if (e == cudaSuccess && !sm.lists) e = dmalloc(q, &sm.lists, (int64_t)2 * kSListSlots * 2 * kMaxHot);
    if (e == cudaSuccess && !sm.ctl)
        e = dmalloc(q, &sm.ctl, ctl_words + (list_n_bytes + 7) / 8);
    if (e == cudaSuccess && !sm.d_desc) e = dmalloc(q, &sm.d_desc, kSMaxBatches);
    for (int s = 0; s < 2 && e == cudaSuccess; s++) {
        if (!sm.h_desc[s]) e = cudaHostAlloc((void **)&sm.h_desc[s], sizeof(SBatch) * kSMaxBatches, cudaHostAllocDefault);
        if (e == cudaSuccess && !sm.ev_desc[s]) e = cudaEventCreateWithFlags(&sm.ev_desc[s], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return e;
    /* descriptors up (the pinned slot is rewritten once its last copy is done) */
    const int ds_slot = sm.desc_slot;
    e = cudaEventSynchronize(sm.ev_desc[ds_slot]);
    if (e != cudaSuccess) return e;
    memcpy(sm.h_desc[ds_slot], sg.b.data(), sizeof(SBatch) * nb);
    e = cudaMemcpyAsync(sm.d_desc, sm.h_desc[ds_slot], sizeof(SBatch) * nb, cudaMemcpyHostToDevice, q->stream);
    if (e == cudaSuccess) e = cudaEventRecord(sm.ev_desc[ds_slot], q->stream);
    sm.desc_slot ^= 1;
    int *list_n = (int *)(sm.ctl + ctl_words);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(sm.ctl, 0, ctl_words * 8 + list_n_bytes, q->stream);
    if (e != cudaSuccess) return e;
    DeviceState &d = q->d;
    SArgs a;
    memset(&a, 0, sizeof(a));
    a.b = sm.d_desc;
    a.nb = nb;
    a.G = q->G;
    a.W = q->W;
    a.minmax = q->minmax;
    a.avg = q->avg;
    a.nA = nA;
    a.nB = nB;
    a.R = rg.R;
    a.M = rg.M;
    a.tcap = rg.tcap;
    a.Smax = (int)smax;
    a.Cpad = Cpad;
    a.stride = stride;
    a.dcap = dcap;
    a.ring_any = ring_any ? 1 : 0;
    a.epoch0 = sg.epoch0;
    a.stage_slot = stage_slot;
    a.pairs_slot = pairs_slot;
    a.ring_k = d.ring_k;
    a.ring_v = d.ring_v;
    a.sufs = d.sufs;
    a.fptr = d.fptr;
    a.sum = d.sum;
    a.cnt = d.cnt;
    a.bmin = d.bmin;
    a.bmax = d.bmax;
    a.fmin = d.fmin;
    a.fmax = d.fmax;
    a.rmin = d.rmin;
    a.rmax = d.rmax;
    a.ravg = d.ravg;
    a.stage = sm.stage;
    a.pairs = (uint2 *)sm.pairs;
    a.hotpart = sm.hotpart;
    a.lists = sm.lists;
    a.list_cnt = sm.lists + kSListSlots * 2 * kMaxHot;
    a.list_n = list_n;
    const int cur = q->hot_parity, nxt = cur ^ 1;
    a.q_hot = d.hotlist + cur * 2 * kMaxHot;
    a.q_hot_cnt = d.hotlist_cnt + cur * 2 * kMaxHot;
    a.q_hot_n = d.hotlist_n + 2 * cur;
    a.hot_cap = q->opt.hot_keys;
    a.ctl = sm.ctl;
    a.err = d.err;
    a.err_host = d.err_host;
    a.wait_ns = (unsigned long long)sm.wait_us * 1000ULL;
    a.stall_batch = sm.stall_batch;
    if (out && out->sum) {
        const int64_t o = (int64_t)sg.call_index * q->G;
        a.snap_sum = out->sum + o;
        a.snap_cnt = out->count + o;
        a.snap_min = out->min + o;
        a.snap_max = out->max + o;
        a.snap_avg = out->avg + o;
    }
    if (out && out->stamps) {
        a.stamp_begin = (unsigned long long *)out->stamps + sg.call_index;
        a.stamp_end = (unsigned long long *)out->stamps + k + sg.call_index;
    }
    /* phase stamps into the cq_trace buffer when it is large enough */
    if (q->trace && q->trace_slots >= (int64_t)(nA + nB) * nb * 12) a.trace = q->trace;
    e = launch_stream(a, ds, q->stream);
    if (e != cudaSuccess) return e;
    q->launches += 1;
    /* the heavy hitters the last batch found (list slot 2) become the query's list */
    const int ls = 2;
    e = cudaMemcpyAsync(d.hotlist + nxt * 2 * kMaxHot, a.lists + (int64_t)ls * 2 * kMaxHot,
                        sizeof(int32_t) * 2 * kMaxHot, cudaMemcpyDeviceToDevice, q->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d.hotlist_cnt + nxt * 2 * kMaxHot, a.list_cnt + (int64_t)ls * 2 * kMaxHot,
                            sizeof(int32_t) * 2 * kMaxHot, cudaMemcpyDeviceToDevice, q->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d.hotlist_n + 2 * nxt, list_n + 2 * (int64_t)(kSListN - 1), 2 * sizeof(int),
                            cudaMemcpyDeviceToDevice, q->stream);
    if (e != cudaSuccess) return e;
    q->hot_parity = nxt;
    sg.b.clear();
    sg.first.clear();
    sg.end.clear();
    return cudaSuccess;
}

/* Copy the query's current results into row j of the caller's per-batch arrays. */
cudaError_t copy_results_row(cq_query *q, const cq_many_out *out, int j) {
    const int64_t G = q->G, o = (int64_t)j * G;
    const DeviceState &d = q->d;
    cudaError_t e = cudaMemcpyAsync(out->sum + o, d.sum, 8 * G, cudaMemcpyDeviceToDevice, q->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out->count + o, d.cnt, 4 * G, cudaMemcpyDeviceToDevice, q->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out->min + o, d.rmin, 4 * G, cudaMemcpyDeviceToDevice, q->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out->max + o, d.rmax, 4 * G, cudaMemcpyDeviceToDevice, q->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out->avg + o, d.ravg, 8 * G, cudaMemcpyDeviceToDevice, q->stream);
    return e;
}

}  // namespace

extern "C" cq_status cq_push_many(cq_query *q, int k, const int32_t *const *d_keys, const int32_t *const *d_vals,
                                  const int64_t *n, const cq_many_out *out) {
    if (!q || k < 0) return CQ_EINVAL;
    if (k > 0 && (!d_keys || !d_vals || !n)) return CQ_EINVAL;
    cq_status st = poison_status(q);
    if (st != CQ_OK) return st;
    for (int j = 0; j < k; j++) {
        if (n[j] < 0) return CQ_EINVAL;
        if (n[j] > 0 && (!d_keys[j] || !d_vals[j])) return CQ_EINVAL;
    }
    const bool snap = out && (out->sum || out->count || out->min || out->max || out->avg);
    if (snap && !(out->sum && out->count && out->min && out->max && out->avg)) return CQ_EINVAL;
    if (k == 0) return CQ_OK;
    set_device(q);
    cudaError_t e = cudaSuccess;
    if (out && out->stamps) {
        e = cudaMemsetAsync(out->stamps, 0xFF, sizeof(uint64_t) * k, q->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(out->stamps + k, 0, sizeof(uint64_t) * k, q->stream);
        if (e != cudaSuccess) return cuda_status(e);
    }
    /* the roles: a producer and a consumer CTA on every SM, or two producers
       on pp of them; fewer consumers take wider key ranges, so a key space
       their shared memory cannot hold falls back to pp = 0 */
    int pp = q->sm.pp_opt >= 0 ? q->sm.pp_opt : 0;
    if (pp > q->num_sms - 1) pp = q->num_sms - 1;
    SRanges rg = stream_ranges(q->G, q->num_sms - pp);
    if (pp > 0 && !stream_supported(q, rg, k, n, q->num_sms + pp)) {
        pp = 0;
        rg = stream_ranges(q->G, q->num_sms);
    }
    const int nA = q->num_sms + pp, nB = q->num_sms - pp;
    if (!stream_supported(q, rg, k, n, nA)) {
        /* batch by batch, with cq_push's kernels */
        for (int j = 0; j < k; j++) {
            if (n[j] > 0) {
                const int64_t skip = n[j] > q->W ? n[j] - q->W : 0;
                st = push_impl(q, d_keys[j] + skip, d_vals[j] + skip, n[j]);
                if (st != CQ_OK) return st;
            }
            if (snap && (e = copy_results_row(q, out, j)) != cudaSuccess) return fail_prepared(q, e);
        }
        return CQ_OK;
    }
    ManySeg sg;
    sg.b.reserve(k < kSMaxBatches ? k : kSMaxBatches);
    const int64_t W = q->W;
    for (int j = 0; j < k; j++) {
        if ((int)sg.b.size() == kSMaxBatches && (e = stream_flush(q, sg, rg, out, k, nA, nB)) != cudaSuccess)
            return fail_prepared(q, e);
        SBatch b;
        memset(&b, 0, sizeof(b));
        b.ring_dep = -1;
        const int64_t N = q->N;
        if (n[j] > 0) {
            const int64_t n_eff = n[j] < W ? n[j] : W;
            const int64_t skip = n[j] - n_eff;
            const int64_t H = N > W ? N - W : 0;
            const int64_t Hn = N + n[j] > W ? N + n[j] - W : 0;
            int64_t fa = 0, fb = 0;
            const bool flip = q->minmax && Hn > q->F && Hn < N;
            const bool reset = q->minmax && Hn > q->F && Hn >= N;
            if (flip) {
                /* the back becomes the front between two launches */
                if ((e = stream_flush(q, sg, rg, out, k, nA, nB)) != cudaSuccess) return fail_prepared(q, e);
                bump_epoch(q);
                e = launch_flip(q->d, q->F % W, N - q->F, q->epoch, q->stream, &q->launches);
                if (e != cudaSuccess) return fail_prepared(q, e);
                fa = q->F - H;
                fb = Hn - H;
                q->F = N;
                q->flips++;
            } else if (q->minmax && Hn <= q->F) {
                fa = 0;
                fb = Hn - H;
            }
            /* an epoch wrap rewrites every tag first: the launch so far goes before it */
            if (reset && q->epoch >= 0xFFFFFFFEu && (e = stream_flush(q, sg, rg, out, k, nA, nB)) != cudaSuccess)
                return fail_prepared(q, e);
            const uint32_t e_before = q->epoch;
            if (reset) {
                bump_epoch(q);
                q->F = Hn;
                q->resets++;
            }
            if (sg.b.empty()) {
                sg.epoch0 = e_before;
                sg.call_index = j;
            }
            const int64_t old_len = N - H;
            const bool replace = n_eff == W && old_len > 0;
            const bool ring = !replace && old_len > 0 && Hn > H;
            const bool front = ring && q->minmax && fb > fa;
            b.keys = d_keys[j] + skip;
            b.vals = d_vals[j] + skip;
            b.n = (int32_t)n_eff;
            b.slot0 = (int32_t)((N + skip) % W);
            b.hmod = (int32_t)(H % W);
            b.old_len = (int32_t)old_len;
            b.fa = (int32_t)fa;
            b.fb = (int32_t)fb;
            b.epoch = q->epoch;
            const bool aligned = ((uintptr_t)b.keys % 16 == 0) && ((uintptr_t)b.vals % 16 == 0) &&
                                 (b.slot0 % 4 == 0) && (W % 4 == 0);
            b.flags = (replace ? SB_REPLACE : 0) | (ring ? SB_RING : 0) | (front ? SB_FRONT : 0) |
                      (aligned ? SB_ALIGNED : 0);
            /* the latest batch of this launch whose ring slots this batch
               touches: one whose first effective tuple is more than W
               before this batch's end */
            const int64_t my_first = N + skip, my_end = N + n[j];
            for (int p = (int)sg.b.size() - 1; p >= 0; p--) {
                if (sg.b[p].n <= 0) continue;
                if (my_end - sg.first[p] > W) {
                    b.ring_dep = p;
                    break;
                }
            }
            /* a run of window-replacing batches rewrites every slot each
               batch and reads none: only the run's last batch must write
               after the others (its slots are the ones that stay), so an
               earlier batch of the run drops its wait once the next batch
               turns out to replace the window too -- unless the batch it
               waits for reads the ring (retracts): those reads must come
               before its writes */
            if (replace)
                for (int p = (int)sg.b.size() - 1; p >= 0; p--) {
                    if (sg.b[p].n <= 0) continue;
                    const int d = sg.b[p].ring_dep;
                    if ((sg.b[p].flags & SB_REPLACE) && (d < 0 || (sg.b[d].flags & SB_REPLACE))) sg.b[p].ring_dep = -1;
                    break;
                }
            const int64_t deltas = n_eff * (ring ? 2 : 1);
            int64_t thr = q->opt.hot_threshold;
            if (thr <= 0) {
                /* a quarter of a consumer's fair share of the batch's deltas:
                   the consumers privatise the two busiest keys of their range
                   themselves, so lighter keys need not be listed; measured on
                   the skew sweep, an eighth (without that privatisation the
                   best) and a half were slower, a sixteenth overfilled the
                   producers' records (and the 128-key list at s = 1) */
                thr = deltas / (4 * (int64_t)rg.R);
                if (thr < 64) thr = 64;
            }
            b.hot_threshold = (uint32_t)(thr > 0x7FFFFFFF ? 0x7FFFFFFF : thr);
            b.hot_gthr = hot_guarantee(n_eff, q->opt.hot_keys);
            sg.first.push_back(my_first);
            sg.end.push_back(my_end);
            q->N += n[j];
            q->pushes++;
        } else {
            if (sg.b.empty()) {
                sg.epoch0 = q->epoch;
                sg.call_index = j;
            }
            b.epoch = q->epoch;
            b.hot_threshold = 0x7FFFFFFF;
            b.hot_gthr = 0xFFFFFFFFu;
            sg.first.push_back(N);
            sg.end.push_back(N);
        }
        sg.b.push_back(b);
    }
    if ((e = stream_flush(q, sg, rg, out, k, nA, nB)) != cudaSuccess) return fail_prepared(q, e);
    q->last_path = 4;
    return CQ_OK;
}

/* ---- push without allocation ----
 *
 * For callers that may not allocate while they push: a server that admitted
 * the query against a fixed device-memory budget (the query's footprint does
 * not count push scratch), and latency-bound loops with other streams in
 * flight, which cudaFree (and possibly cudaMalloc) would stall by waiting for
 * the whole device.  The partitioned kernel's scratch then comes from the
 * fixed array below instead of the query's growable buffers. */

/* One per device: a module-scope device array exists in every context that
 * loads this module.  No kernel lives in this file, so the module (and the
 * array's memory) is loaded at the first address lookup, not at start-up. */
static __device__ __align__(256) unsigned char g_noalloc_scratch[CQ_NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices];   /* the array's address on each device, once looked up */

/* The array's address on `device`, which must be current.  The first lookup
 * per device loads the module; later calls return the cached address. */
cudaError_t noalloc_scratch(int device, unsigned char **out) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e;
        }
        g_noalloc_ptr[device] = p;
    }
    *out = (unsigned char *)g_noalloc_ptr[device];
    return cudaSuccess;
}

/* Byte offsets of a launch's scratch inside the array: the barrier counter at
 * 0, then staged deltas (16 bytes a staged slot, twice a delta's 8, which
 * keeps the limits cq.h states) and the run table, each 256-byte aligned. */
struct NoallocLayout {
    int64_t stage, off, end;
};

int64_t align256(int64_t x) { return (x + 255) / 256 * 256; }

NoallocLayout noalloc_layout(const GPlan &pl) {
    NoallocLayout L;
    L.stage = 256;
    L.off = align256(L.stage + (int64_t)pl.C * pl.stride * 16);
    L.end = L.off + group_pair_bytes(pl);
    return L;
}

}  // namespace

extern "C" cq_status cq_push_noalloc(cq_query *q, const int32_t *d_keys, const int32_t *d_vals, int64_t n) {
    if (!q) return CQ_EINVAL;
    cq_status st = poison_status(q);
    if (st != CQ_OK) return st;
    if (n < 0) return CQ_EINVAL;
    if (n == 0) return CQ_OK;
    if (!d_keys || !d_vals) return CQ_EINVAL;
    set_device(q);
    unsigned char *area = nullptr;
    cudaError_t e = noalloc_scratch(q->device, &area);
    if (e != cudaSuccess) return cuda_status(e);
    /* plan and size check before any state changes */
    const int64_t n_eff = n < q->W ? n : q->W;
    const int64_t skip = n - n_eff;
    const int32_t *k = d_keys + skip, *v = d_vals + skip;
    GPlan gp;
    if (!group_plan(q, n_eff, k, v, (q->N + skip) % q->W, group_grid(q->device, q->num_sms), true, &gp,
                    n_eff == q->W && q->N > 0))
        return CQ_ESCRATCH;
    const NoallocLayout L = noalloc_layout(gp);
    if (L.end > CQ_NOALLOC_SCRATCH_BYTES) return CQ_ESCRATCH;
    IngestArgs a;
    e = prepare_push(q, k, v, n, &a);
    if (e != cudaSuccess) return fail_prepared(q, e);
    const bool front = q->minmax && a.fb > a.fa;
    QDesc dsc;
    group_desc_fill(q, a, gp, front, &dsc);
    dsc.stage = area + L.stage;
    dsc.off = (uint32_t *)(area + L.off);

    unsigned long long *bar = (unsigned long long *)area;
    unsigned long long bar_base = 0;
    e = cudaMemsetAsync(bar, 0, sizeof(*bar), q->stream);
    if (e == cudaSuccess)
        e = launch_group(q->stream, q->device, q->num_sms, &dsc, 1, nullptr, nullptr, nullptr, bar, &bar_base, nullptr,
                         0, front);
    if (e != cudaSuccess) return fail_prepared(q, e);
    q->launches += 1;
    commit_push(q, n, 3);
    return CQ_OK;
}
