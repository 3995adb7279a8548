/*
 * cq_serve.cu -- the serving loop: many standing queries fed by requests
 * that arrive over time (cqs_* in cq.h).
 *
 * Threads.  Callers submit batches from any thread (cqs_submit); one
 * dispatcher thread takes, for every query with pending batches, its oldest
 * pending batch and pushes all of them in one group launch (continuous
 * batching: a launch holds at most one batch per query, so a query's batches
 * stay in arrival order); one completion thread waits for each launch's event
 * and stamps its batches' completion time.  The group keeps two launches in
 * flight, so the dispatcher prepares launch i+1 while launch i runs.
 *
 * Admission.  A query is admitted only if its device footprint (state, from
 * cq_footprint_bytes, plus the push scratch that batches up to its declared
 * maximum can need, reserved at admission) fits in what is left of the
 * server's budget; serving itself then allocates no device memory.
 *
 * Latency of a batch = completion stamp - arrival stamp, both on the host's
 * monotonic clock (cqs_now_ns).
 */
#include <cuda_runtime.h>
#include <stdint.h>
#include <time.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "cq.h"
#include "cq_host.h"

namespace {

int64_t mono_ns() {
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (int64_t)ts.tv_sec * 1000000000LL + ts.tv_nsec;
}

constexpr int kEvents = 4;   /* launches the completion thread may trail by */

struct Batch {
    int member;
    const int32_t *keys, *vals;
    int64_t n;
    int64_t arrival, done_at;
    cq_status status;
    bool done;
};

struct Member {
    cq_query *q;
    int64_t max_batch, reserved;
    std::deque<int64_t> pending;   /* tickets in arrival order */
    bool queued;                   /* listed in cqs_server::ready */
};

struct Flight {
    cudaEvent_t ev;
    std::vector<int64_t> tickets;
    cq_status status;              /* the launch's own status */
};

}  // namespace

struct cqs_server {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cq_group *group = nullptr;
    int64_t budget = 0, reserved = 0;

    std::mutex mu;
    std::condition_variable cv_work;     /* dispatcher: batches ready, or stop */
    std::condition_variable cv_flight;   /* completion thread: a launch in flight, or stop */
    std::condition_variable cv_event;    /* dispatcher: an event came back */
    std::condition_variable cv_done;     /* waiters: batches completed */
    std::vector<Member> members;
    std::unordered_map<const cq_query *, int> index;
    std::vector<Batch> batches;          /* by ticket */
    std::deque<int> ready;               /* members with pending batches, round robin */
    std::deque<Flight> flights;
    std::vector<cudaEvent_t> events;     /* free events */
    bool stop = false, dispatcher_done = false;
    int64_t submitted = 0, completed = 0, tuples = 0, launches = 0, batches_launched = 0;
    int64_t first_arrival = INT64_MAX, last_done = 0;
    std::vector<double> latency_us;      /* of completed batches since the last reset */
    cq_status fatal = CQ_OK;             /* a failed launch: later launches are refused */

    std::thread dispatcher, completer;
};

namespace {

void dispatch_loop(cqs_server *s) {
    cudaSetDevice(s->device);
    std::vector<cq_query *> qs;
    std::vector<const int32_t *> ks, vs;
    std::vector<int64_t> ns, tickets;
    std::vector<cq_status> st;
    for (;;) {
        cudaEvent_t ev = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || !s->ready.empty(); });
            if (s->ready.empty()) break;
            s->cv_event.wait(lk, [&] { return !s->events.empty(); });
            ev = s->events.back();
            s->events.pop_back();
            qs.clear();
            ks.clear();
            vs.clear();
            ns.clear();
            tickets.clear();
            const size_t nr = s->ready.size();
            for (size_t i = 0; i < nr; i++) {
                const int m = s->ready.front();
                s->ready.pop_front();
                Member &mb = s->members[m];
                const int64_t t = mb.pending.front();
                mb.pending.pop_front();
                const Batch &b = s->batches[t];
                qs.push_back(mb.q);
                ks.push_back(b.keys);
                vs.push_back(b.vals);
                ns.push_back(b.n);
                tickets.push_back(t);
                if (mb.pending.empty()) mb.queued = false;
                else s->ready.push_back(m);
            }
        }
        st.assign(qs.size(), CQ_OK);
        cq_status r = CQ_ECUDA;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            r = s->fatal;
        }
        if (r == CQ_OK) r = cqg_push(s->group, (int)qs.size(), qs.data(), ks.data(), vs.data(), ns.data(), st.data());
        if (r == CQ_OK && cudaEventRecord(ev, s->stream) != cudaSuccess) r = CQ_ECUDA;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            Flight f;
            f.ev = ev;
            f.tickets = tickets;
            f.status = r;
            for (size_t i = 0; i < tickets.size(); i++) s->batches[tickets[i]].status = r != CQ_OK ? r : st[i];
            if (r != CQ_OK && s->fatal == CQ_OK) s->fatal = r;
            s->flights.push_back(std::move(f));
            s->launches++;
            s->batches_launched += (int64_t)tickets.size();
        }
        s->cv_flight.notify_one();
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->dispatcher_done = true;
    s->cv_flight.notify_one();
}

void complete_loop(cqs_server *s) {
    cudaSetDevice(s->device);
    for (;;) {
        cudaEvent_t ev;
        cq_status launch_status;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_flight.wait(lk, [&] { return !s->flights.empty() || s->dispatcher_done; });
            if (s->flights.empty()) return;
            ev = s->flights.front().ev;
            launch_status = s->flights.front().status;
        }
        cudaError_t e = launch_status == CQ_OK ? cudaEventSynchronize(ev) : cudaSuccess;
        const int64_t now = mono_ns();
        {
            std::lock_guard<std::mutex> lk(s->mu);
            Flight f = std::move(s->flights.front());
            s->flights.pop_front();
            for (int64_t t : f.tickets) {
                Batch &b = s->batches[t];
                if (e != cudaSuccess) b.status = CQ_ECUDA;
                b.done = true;
                b.done_at = now;
                s->completed++;
                s->tuples += b.n;
                s->latency_us.push_back((double)(now - b.arrival) * 1e-3);
            }
            if (e != cudaSuccess && s->fatal == CQ_OK) s->fatal = CQ_ECUDA;
            s->last_done = now;
            s->events.push_back(f.ev);
        }
        s->cv_event.notify_one();
        s->cv_done.notify_all();
    }
}

double percentile(std::vector<double> &v, double p) {
    /* nearest rank: the smallest value with at least p of the samples at or below it */
    if (v.empty()) return 0.0;
    size_t r = (size_t)(p * (double)v.size() + 0.999999999);
    if (r < 1) r = 1;
    if (r > v.size()) r = v.size();
    std::nth_element(v.begin(), v.begin() + (r - 1), v.end());
    return v[r - 1];
}

}  // namespace

extern "C" {

int64_t cqs_now_ns(void) { return mono_ns(); }

cq_status cqs_create(int64_t budget_bytes, void *cuda_stream, cqs_server **out) {
    if (!out) return CQ_EINVAL;
    *out = nullptr;
    if (budget_bytes < 0) return CQ_EINVAL;
    cqs_server *s = new (std::nothrow) cqs_server();
    if (!s) return CQ_ENOMEM;
    s->budget = budget_bytes;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) {
        if (cuda_stream) {
            s->stream = (cudaStream_t)cuda_stream;
        } else {
            e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
            s->own_stream = e == cudaSuccess;
        }
    }
    for (int i = 0; i < kEvents && e == cudaSuccess; i++) {
        cudaEvent_t ev;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) s->events.push_back(ev);
    }
    cq_status st = e == cudaSuccess ? cqg_create(s->stream, &s->group) : CQ_ECUDA;
    /* launch shapes rarely repeat here, and admissions from other threads
     * enqueue work on the same stream, which a capture would take in */
    if (st == CQ_OK) cq::group_disable_graphs(s->group);
    if (st != CQ_OK) {
        cudaGetLastError();
        for (cudaEvent_t ev : s->events) cudaEventDestroy(ev);
        if (s->own_stream) cudaStreamDestroy(s->stream);
        delete s;
        return st;
    }
    s->dispatcher = std::thread(dispatch_loop, s);
    s->completer = std::thread(complete_loop, s);
    *out = s;
    return CQ_OK;
}

cq_status cqs_admit(cqs_server *s, int64_t groups, int64_t window, uint32_t aggs, int64_t max_batch, cq_query **out) {
    if (!s || !out) return CQ_EINVAL;
    *out = nullptr;
    if (max_batch < 1) return CQ_EINVAL;
    const int64_t state = cq_footprint_bytes(groups, window, aggs);
    const int64_t scratch = cq::group_scratch_bound(groups, window, max_batch);
    if (state < 0 || scratch < 0 || aggs == 0 || (aggs & ~(uint32_t)CQ_ALL)) return CQ_EINVAL;
    const int64_t need = state + scratch;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->reserved + need > s->budget) return CQ_EBUDGET;
        s->reserved += need;
    }
    cudaSetDevice(s->device);
    cq_query *q = nullptr;
    cq_status st = cq_create(groups, window, aggs, s->stream, &q);
    if (st == CQ_OK && cq::reserve_group_scratch(q, max_batch) != cudaSuccess) {
        cudaGetLastError();
        cq_destroy(q);
        q = nullptr;
        st = CQ_ENOMEM;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (st != CQ_OK) {
        s->reserved -= need;
        return st;
    }
    Member m;
    m.q = q;
    m.max_batch = max_batch;
    m.reserved = need;
    m.queued = false;
    s->index[q] = (int)s->members.size();
    s->members.push_back(std::move(m));
    *out = q;
    return CQ_OK;
}

cq_status cqs_submit(cqs_server *s, cq_query *q, const int32_t *d_keys, const int32_t *d_vals, int64_t n,
                     int64_t arrival_ns, int64_t *ticket) {
    if (!s || !q || n < 0 || (n > 0 && (!d_keys || !d_vals))) return CQ_EINVAL;
    const int64_t arrival = arrival_ns >= 0 ? arrival_ns : mono_ns();
    int64_t t;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->index.find(q);
        if (it == s->index.end()) return CQ_EINVAL;
        Member &mb = s->members[it->second];
        if (n > mb.max_batch) return CQ_EINVAL;
        if (s->stop) return CQ_EBUSY;
        t = (int64_t)s->batches.size();
        Batch b;
        b.member = it->second;
        b.keys = d_keys;
        b.vals = d_vals;
        b.n = n;
        b.arrival = arrival;
        b.done_at = 0;
        b.status = CQ_OK;
        b.done = false;
        s->batches.push_back(b);
        mb.pending.push_back(t);
        if (!mb.queued) {
            mb.queued = true;
            s->ready.push_back(it->second);
        }
        s->submitted++;
        if (arrival < s->first_arrival) s->first_arrival = arrival;
    }
    s->cv_work.notify_one();
    if (ticket) *ticket = t;
    return CQ_OK;
}

cq_status cqs_wait(cqs_server *s, int64_t ticket) {
    if (!s) return CQ_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    if (ticket < 0 || ticket >= (int64_t)s->batches.size()) return CQ_EINVAL;
    s->cv_done.wait(lk, [&] { return s->batches[ticket].done; });
    return s->batches[ticket].status;
}

cq_status cqs_drain(cqs_server *s) {
    if (!s) return CQ_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] { return s->completed == s->submitted; });
    return s->fatal;
}

cq_status cqs_replay(cqs_server *s, int64_t nb, cq_query *const *queries, const int64_t *arrival_ns,
                     const int32_t *const *d_keys, const int32_t *const *d_vals, const int64_t *n) {
    if (!s || nb < 0 || (nb > 0 && (!queries || !arrival_ns || !d_keys || !d_vals || !n))) return CQ_EINVAL;
    for (int64_t i = 1; i < nb; i++)
        if (arrival_ns[i] < arrival_ns[i - 1]) return CQ_EINVAL;
    const int64_t t0 = mono_ns() + 1000000;   /* 1 ms lead */
    cq_status ret = CQ_OK;
    for (int64_t i = 0; i < nb && ret == CQ_OK; i++) {
        const int64_t at = t0 + arrival_ns[i];
        for (;;) {   /* open loop: submit at the scheduled time, whatever the backlog */
            const int64_t now = mono_ns();
            if (now >= at) break;
            if (at - now > 200000) std::this_thread::sleep_for(std::chrono::microseconds((at - now) / 2000));
        }
        ret = cqs_submit(s, queries[i], d_keys[i], d_vals[i], n[i], at, nullptr);
    }
    cq_status d = cqs_drain(s);
    return ret != CQ_OK ? ret : d;
}

cq_status cqs_stats(cqs_server *s, cqs_server_stats *out) {
    if (!s || !out) return CQ_EINVAL;
    std::vector<double> lat;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        out->queries = (int64_t)s->members.size();
        out->reserved_bytes = s->reserved;
        out->budget_bytes = s->budget;
        out->submitted = s->submitted;
        out->completed = s->completed;
        out->tuples = s->tuples;
        out->launches = s->launches;
        out->batches_launched = s->batches_launched;
        out->busy_s = s->completed > 0 && s->last_done > s->first_arrival
                          ? (double)(s->last_done - s->first_arrival) * 1e-9 : 0.0;
        lat = s->latency_us;
    }
    double sum = 0.0, mx = 0.0;
    for (double x : lat) {
        sum += x;
        mx = x > mx ? x : mx;
    }
    out->latency_mean_us = lat.empty() ? 0.0 : sum / (double)lat.size();
    out->latency_max_us = mx;
    out->latency_p50_us = percentile(lat, 0.50);
    out->latency_p99_us = percentile(lat, 0.99);
    return CQ_OK;
}

cq_status cqs_reset_stats(cqs_server *s) {
    if (!s) return CQ_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->completed != s->submitted) return CQ_EBUSY;
    s->latency_us.clear();
    s->submitted = s->completed = s->tuples = s->launches = s->batches_launched = 0;
    s->first_arrival = INT64_MAX;
    s->last_done = 0;
    s->batches.clear();
    return CQ_OK;
}

void cqs_destroy(cqs_server *s) {
    if (!s) return;
    cqs_drain(s);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    s->dispatcher.join();
    s->completer.join();
    for (Member &m : s->members) cq_destroy(m.q);
    cqg_destroy(s->group);
    for (cudaEvent_t ev : s->events) cudaEventDestroy(ev);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
}

}  /* extern "C" */
