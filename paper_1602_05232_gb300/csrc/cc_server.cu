// Serving form: a continuous-batching request loop over one forest (the
// cc_server_* entry points of include/cc.h).
//
// Threads and streams:
//  - callers enqueue requests (any thread); each gets a ticket and an arrival
//    time;
//  - one worker thread cuts the arrived, not yet launched requests into
//    groups of consecutive same-kind requests (up to kMaxBatch groups at a
//    time), reserves a contiguous range of its kind's device staging ring for
//    each group (one ring for update edges, one for query pairs), copies the
//    host data in on the h2d stream, and launches ONE Bulk-Update or
//    Bulk-Query per group over its range on the compute stream, after the
//    copy that carried its data. Requests whose host data follow one another
//    and land next to each other in their ring share one copy, also across
//    groups: with the two kinds in separate rings, the update groups of a
//    batch that alternates updates and queries still fill one run of the
//    update ring, so the copies stay large when the groups are small. Query
//    answers go back on the d2h stream. An event recorded after the group's
//    last operation is watched by a completion thread, which stamps the
//    completion time and frees the group's ring range;
//  - groups compute in arrival order on the single compute stream, so a
//    query sees exactly the updates that arrived before it. Merging adjacent
//    updates is exact because the graph is the union of the edge sets.
// Neither thread holds the lock while it calls CUDA, so neither can wait on
// the other.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "cc.h"
#include "cc_internal.cuh"

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Req {
    int32_t kind;
    const int32_t* data;
    int64_t k;
    uint8_t* out;
    double t_arrive = 0, t_done = -1;
    int64_t off = 0;  // ring position (pairs)
    bool done = false;
};

struct Group {
    cc_server* srv;
    int64_t first, last;  // requests [first, last)
    int32_t kind;         // CC_OP_UPDATE or CC_OP_QUERY: which ring
    int64_t b, e;         // ring range [b, e) in pairs
    cudaEvent_t ev = nullptr;  // recorded after the group's last operation
    bool launched = false;     // ev has been recorded
    bool done = false;
};

// A staging ring of pairs on the device: FIFO ranges, see ring_alloc.
struct Ring {
    int32_t* buf = nullptr;  // 2 * cap ints
    int64_t head = 0;
    int64_t used = 0;        // pairs held by in-flight groups of this ring's kind
};

constexpr int kMaxBatch = 64;                     // groups formed per pass of the worker
constexpr int64_t kMaxRunPairs = (int64_t)1 << 22;  // 32 MiB: a longer copy run only delays its first group

}  // namespace

struct cc_server {
    cc_ctx* ctx = nullptr;
    cudaStream_t prev_stream = nullptr;
    int device = 0;
    cudaStream_t compute = nullptr, h2d = nullptr, d2h = nullptr;
    cudaEvent_t ev_q = nullptr;
    std::vector<cudaEvent_t> run_ev;   // one per copy run of a batch (worker thread only)
    Ring ring[2];                      // [CC_OP_UPDATE], [CC_OP_QUERY]
    uint8_t* ring_out = nullptr;       // query answers, at the query ring's offsets
    int64_t cap = 0, max_group = 0;    // cap: pairs per ring
    bool merge = true;

    std::mutex mu;
    // one condition per kind of waiter, so that a notification wakes only
    // the thread that can act on it
    std::condition_variable cv_work;  // worker: new requests, ring space, stop
    std::condition_variable cv_reap;  // completion thread: launched groups, stop
    std::condition_variable cv_done;  // cc_server_wait / drain / destroy: completions
    std::deque<Req> reqs;
    int64_t next_launch = 0, completed = 0, groups = 0;
    int64_t n_upd = 0, n_qry = 0, edges = 0, pairs = 0;
    std::deque<Group*> inflight;
    bool stop = false;
    cc_status err = CC_OK;
    std::string errmsg;
    std::thread worker;
    std::thread reaper;                 // completion thread
    std::vector<cudaEvent_t> spare_events;
};

namespace {

void fail_worker(cc_server* s, cudaError_t e, const char* what) {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->err == CC_OK) {
        s->err = CC_ERR_CUDA;
        s->errmsg = std::string(what) + ": " + cudaGetErrorString(e);
    }
    s->cv_work.notify_all();
    s->cv_reap.notify_all();
    s->cv_done.notify_all();
}

// A group's work is complete: stamp its requests, free ring ranges in order.
// Called with the lock held.
void mark_done(cc_server* s, Group* g, double t) {
    for (int64_t i = g->first; i < g->last; i++) {
        s->reqs[i].t_done = t;
        s->reqs[i].done = true;
    }
    s->completed += g->last - g->first;
    g->done = true;
    while (!s->inflight.empty() && s->inflight.front()->done) {
        Group* f = s->inflight.front();
        s->ring[f->kind].used -= f->e - f->b;
        s->spare_events.push_back(f->ev);
        delete f;
        s->inflight.pop_front();
    }
    s->cv_done.notify_all();
    s->cv_work.notify_one();  // ring space for a group that did not fit
}

// Completion thread: takes the oldest launched group that is not done under
// the lock, then polls its event with the lock released (the worker and the
// enqueuing threads never wait behind the poll), so the time from completion
// to notice stays at a few microseconds. Groups complete in launch order
// except that an update group may finish while an earlier query group's
// answers are still being copied out; such a group is noticed right after
// that copy. Only this thread marks groups done, and a group is freed only
// once done, so the pointer stays valid while it is polled.
void reaper_loop(cc_server* s) {
    cudaSetDevice(s->device);
    for (;;) {
        Group* g = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            auto oldest = [&]() -> Group* {
                for (Group* x : s->inflight)
                    if (!x->done) return x->launched ? x : nullptr;
                return nullptr;
            };
            s->cv_reap.wait(lk, [&] {
                if (s->err != CC_OK || oldest()) return true;
                return s->stop && s->next_launch >= (int64_t)s->reqs.size() && s->inflight.empty();
            });
            if (s->err != CC_OK) return;
            g = oldest();
            if (!g) return;  // stopping, nothing left
        }
        // poll every ~2 us: often enough for latency, rarely enough that the
        // driver calls of the worker thread do not queue behind the queries
        cudaError_t q;
        while ((q = cudaEventQuery(g->ev)) == cudaErrorNotReady) {
            const double t_next = now_s() + 2e-6;
            while (now_s() < t_next) std::this_thread::yield();
        }
        if (q != cudaSuccess) {
            fail_worker(s, q, "serve: completion");
            return;
        }
        const double t = now_s();
        std::lock_guard<std::mutex> lk(s->mu);
        mark_done(s, g, t);
    }
}

// Reserve [b, b+k) of the ring of `kind` (FIFO). Called with the lock held.
//
// Groups of a kind take ranges of its ring in launch order and free them in
// the same order, so the occupied part is one arc from the oldest non-empty
// in-flight group's start (tail) to head, possibly wrapping past the end.
// Emptiness is decided by the number of pairs held, not by head == tail: a
// group of zero pairs sits at head without occupying anything, and when it is
// the oldest in flight while later groups have filled the ring all the way
// round, head == tail means full.
bool ring_alloc(cc_server* s, int32_t kind, int64_t k, int64_t* b) {
    Ring& r = s->ring[kind];
    if (r.used == 0) r.head = 0;
    if (k == 0) {
        *b = r.head;
        return true;
    }
    if (r.used == 0) {
        if (k > s->cap) return false;
        *b = 0;
        return true;
    }
    int64_t tail = r.head;
    for (const Group* g : s->inflight)
        if (g->kind == kind && g->e > g->b) {
            tail = g->b;
            break;
        }
    if (r.head > tail) {
        // occupied [tail, head): free space at the end, then at the start
        if (s->cap - r.head >= k) { *b = r.head; return true; }
        if (tail >= k) { *b = 0; return true; }
        return false;
    }
    // wrapped: occupied [tail, cap) and [0, head); free [head, tail)
    if (tail - r.head >= k) { *b = r.head; return true; }
    return false;
}


// One group of a batch, as the worker's device-work section sees it.
struct Planned {
    Group* g;
    int64_t r0, r1;  // its requests: batch[r0, r1)
    int need;        // the last copy run that carries its data, or -1
};

// A copy of host data that follow one another into consecutive ring slots.
struct Run {
    int32_t kind;
    const int32_t* src;
    int64_t dst, pairs;   // ring offset and length, in pairs
    int64_t r0, r1;       // the batch requests it covers
};

void worker_loop(cc_server* s) {
    cudaSetDevice(s->device);
    std::vector<Req> batch;
    std::vector<Planned> plan;
    std::vector<Run> runs;
    std::vector<int> run_of;  // batch request -> run, or -1 (empty request)
    for (;;) {
        plan.clear();
        batch.clear();
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || s->err != CC_OK || s->next_launch < (int64_t)s->reqs.size(); });
            if (s->err != CC_OK) return;
            if (s->next_launch >= (int64_t)s->reqs.size()) return;  // stop, nothing left
            while ((int)plan.size() < kMaxBatch && s->next_launch < (int64_t)s->reqs.size()) {
                // the longest run of same-kind requests that fits one launch
                const int64_t first = s->next_launch;
                const int32_t kind = s->reqs[first].kind;
                int64_t last = first, total = 0, b = 0;
                while (last < (int64_t)s->reqs.size() && s->reqs[last].kind == kind &&
                       (last == first || (s->merge && total + s->reqs[last].k <= s->max_group))) {
                    total += s->reqs[last].k;
                    last++;
                }
                // shrink it until its staging range fits; else launch what the
                // batch has, or wait for room
                while (!ring_alloc(s, kind, total, &b) && last - first > 1) total -= s->reqs[--last].k;
                if (!ring_alloc(s, kind, total, &b)) {
                    if (!plan.empty()) break;
                    s->cv_work.wait(lk);
                    if (s->err != CC_OK) return;
                    continue;
                }
                Group* g = new Group{s, first, last, kind, b, b + total};
                if (!s->spare_events.empty()) {
                    g->ev = s->spare_events.back();
                    s->spare_events.pop_back();
                }
                s->inflight.push_back(g);
                s->ring[kind].head = b + total;
                s->ring[kind].used += total;
                s->next_launch = last;
                s->groups++;
                const int64_t r0 = (int64_t)batch.size();
                int64_t off = b;
                for (int64_t i = first; i < last; i++) {
                    s->reqs[i].off = off;
                    off += s->reqs[i].k;
                    batch.push_back(s->reqs[i]);
                }
                plan.push_back({g, r0, (int64_t)batch.size(), -1});
            }
        }
        // --- device work for the batch (no lock held) ---
        cudaError_t e = cudaSuccess;
        for (Planned& p : plan)
            if (!p.g->ev && e == cudaSuccess) e = cudaEventCreateWithFlags(&p.g->ev, cudaEventDisableTiming);
        // copy runs: a request extends the open run of its kind when its host
        // data and its ring slots both follow on; runs are numbered in the
        // order of their first request, which is the order they are copied
        runs.clear();
        run_of.assign(batch.size(), -1);
        int open[2] = {-1, -1};
        for (Planned& p : plan) {
            const int32_t kind = p.g->kind;
            for (int64_t i = p.r0; i < p.r1; i++) {
                const Req& r = batch[i];
                if (r.k == 0) continue;
                int o = open[kind];
                if (o >= 0 && runs[o].src + 2 * runs[o].pairs == r.data && runs[o].dst + runs[o].pairs == r.off &&
                    runs[o].pairs + r.k <= kMaxRunPairs) {
                    runs[o].pairs += r.k;
                    runs[o].r1 = i + 1;
                } else {
                    runs.push_back({kind, r.data, r.off, r.k, i, i + 1});
                    o = open[kind] = (int)runs.size() - 1;
                }
                run_of[i] = o;
                if (o > p.need) p.need = o;
            }
        }
        while (s->run_ev.size() < runs.size() && e == cudaSuccess) {
            cudaEvent_t ev = nullptr;
            e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e == cudaSuccess) s->run_ev.push_back(ev);
        }
        // copy in, run by run; if the driver refuses a run (it spans two
        // separate host allocations), copy its requests one by one
        for (size_t ri = 0; ri < runs.size() && e == cudaSuccess; ri++) {
            const Run& r = runs[ri];
            int32_t* dst = s->ring[r.kind].buf + 2 * r.dst;
            e = cudaMemcpyAsync(dst, r.src, sizeof(int32_t) * 2 * (size_t)r.pairs, cudaMemcpyHostToDevice, s->h2d);
            if (e == cudaErrorInvalidValue && r.r1 - r.r0 > 1) {
                cudaGetLastError();
                e = cudaSuccess;
                for (int64_t i = r.r0; i < r.r1 && e == cudaSuccess; i++)
                    if (run_of[i] == (int)ri)
                        e = cudaMemcpyAsync(s->ring[r.kind].buf + 2 * batch[i].off, batch[i].data,
                                            sizeof(int32_t) * 2 * (size_t)batch[i].k, cudaMemcpyHostToDevice, s->h2d);
            }
            if (e == cudaSuccess) e = cudaEventRecord(s->run_ev[ri], s->h2d);
        }
        if (e != cudaSuccess) { fail_worker(s, e, "serve: staging copy"); return; }
        // launch the groups in arrival order, each after the copy of its data
        int waited = -1;
        for (const Planned& p : plan) {
            Group* g = p.g;
            const int64_t total = g->e - g->b;
            if (p.need > waited) {
                e = cudaStreamWaitEvent(s->compute, s->run_ev[p.need], 0);
                waited = p.need;
            }
            if (e != cudaSuccess) break;
            if (g->kind == CC_OP_UPDATE) {
                cc_status st = total ? cc_bulk_update(s->ctx, s->ring[CC_OP_UPDATE].buf + 2 * g->b, total) : CC_OK;
                if (st != CC_OK) { fail_worker(s, cudaErrorUnknown, "serve: bulk update"); return; }
                e = cudaEventRecord(g->ev, s->compute);
            } else {
                cc_status st = total ? cc_bulk_query(s->ctx, s->ring[CC_OP_QUERY].buf + 2 * g->b, total,
                                                     s->ring_out + g->b)
                                     : CC_OK;
                if (st != CC_OK) { fail_worker(s, cudaErrorUnknown, "serve: bulk query"); return; }
                e = cudaEventRecord(s->ev_q, s->compute);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(s->d2h, s->ev_q, 0);
                for (int64_t i = p.r0; i < p.r1 && e == cudaSuccess;) {  // contiguous outputs: one copy
                    int64_t j = i + 1;
                    int64_t pairs = batch[i].k;
                    while (j < p.r1 && batch[j].out == batch[i].out + pairs) pairs += batch[j++].k;
                    if (pairs > 0) {
                        e = cudaMemcpyAsync(batch[i].out, s->ring_out + batch[i].off, (size_t)pairs,
                                            cudaMemcpyDeviceToHost, s->d2h);
                        if (e == cudaErrorInvalidValue && j > i + 1) {  // spans two allocations
                            cudaGetLastError();
                            e = cudaSuccess;
                            for (int64_t r = i; r < j && e == cudaSuccess; r++)
                                if (batch[r].k > 0)
                                    e = cudaMemcpyAsync(batch[r].out, s->ring_out + batch[r].off, (size_t)batch[r].k,
                                                        cudaMemcpyDeviceToHost, s->d2h);
                        }
                    }
                    i = j;
                }
                if (e == cudaSuccess) e = cudaEventRecord(g->ev, s->d2h);
            }
            if (e != cudaSuccess) break;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                g->launched = true;
                s->cv_reap.notify_one();
            }
        }
        if (e != cudaSuccess) { fail_worker(s, e, "serve: launch"); return; }
    }
}

cc_status server_fail(cc_status st, const char* msg) { return cc::record_error(st, msg); }

}  // namespace

extern "C" {

cc_status cc_server_create(cc_ctx* ctx, const cc_server_config* cfg, cc_server** out) {
    if (!ctx || !out) return server_fail(CC_ERR_ARG, "cc_server_create: null argument");
    *out = nullptr;
    if (cc::ctx_graphs(ctx) > 1) return server_fail(CC_ERR_UNSUPPORTED, "cc_server_create: segmented handle");
    cc_server* s = new (std::nothrow) cc_server();
    if (!s) return server_fail(CC_ERR_OOM, "cc_server_create: host allocation");
    s->ctx = ctx;
    s->device = cc::ctx_device(ctx);
    s->prev_stream = cc::ctx_stream(ctx);
    s->cap = (cfg && cfg->ring_pairs > 0) ? cfg->ring_pairs : (int64_t)1 << 25;
    s->max_group = (cfg && cfg->max_group_pairs > 0) ? cfg->max_group_pairs : (int64_t)1 << 22;
    s->merge = cfg ? cfg->merge != 0 : true;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    cudaError_t e = cudaStreamCreateWithFlags(&s->compute, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->h2d, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->d2h, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_q, cudaEventDisableTiming);
    for (int kind = 0; kind < 2 && e == cudaSuccess; kind++)
        e = cudaMalloc(&s->ring[kind].buf, sizeof(int32_t) * 2 * (size_t)s->cap);
    if (e == cudaSuccess) e = cudaMalloc(&s->ring_out, (size_t)s->cap);
    // the new streams do not wait for the handle's old stream: order them once
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->prev_stream);
    cudaSetDevice(prev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(s->ring[0].buf);
        cudaFree(s->ring[1].buf);
        cudaFree(s->ring_out);
        if (s->ev_q) cudaEventDestroy(s->ev_q);
        if (s->compute) cudaStreamDestroy(s->compute);
        if (s->h2d) cudaStreamDestroy(s->h2d);
        if (s->d2h) cudaStreamDestroy(s->d2h);
        delete s;
        return server_fail(e == cudaErrorMemoryAllocation ? CC_ERR_OOM : CC_ERR_CUDA, "cc_server_create: CUDA setup failed");
    }
    cc_set_stream(ctx, s->compute);
    s->worker = std::thread(worker_loop, s);
    s->reaper = std::thread(reaper_loop, s);
    *out = s;
    return CC_OK;
}

cc_status cc_server_enqueue(cc_server* s, int32_t kind, const int32_t* data, int64_t k,
                            uint8_t* out, uint64_t* ticket) {
    if (!s) return server_fail(CC_ERR_ARG, "cc_server_enqueue: null server");
    if (kind != CC_OP_UPDATE && kind != CC_OP_QUERY) return server_fail(CC_ERR_ARG, "cc_server_enqueue: unknown kind");
    if (k < 0 || k > s->cap || k > INT32_MAX) return server_fail(CC_ERR_ARG, "cc_server_enqueue: k out of range (larger than the staging ring?)");
    if (k > 0 && (!data || (kind == CC_OP_QUERY && !out))) return server_fail(CC_ERR_ARG, "cc_server_enqueue: null array");
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->err != CC_OK) return server_fail(s->err, s->errmsg.c_str());
    if (s->stop) return server_fail(CC_ERR_ARG, "cc_server_enqueue: server is stopping");
    Req r;
    r.kind = kind;
    r.data = data;
    r.k = k;
    r.out = out;
    r.t_arrive = now_s();
    s->reqs.push_back(r);
    if (kind == CC_OP_UPDATE) { s->n_upd++; s->edges += k; } else { s->n_qry++; s->pairs += k; }
    if (ticket) *ticket = (uint64_t)(s->reqs.size() - 1);
    s->cv_work.notify_one();
    return CC_OK;
}

cc_status cc_server_enqueue_many(cc_server* s, int64_t n, const int32_t* kinds,
                                 const int32_t* const* data, const int64_t* k, uint8_t* const* out,
                                 uint64_t* first_ticket) {
    if (!s) return server_fail(CC_ERR_ARG, "cc_server_enqueue_many: null server");
    if (n < 0) return server_fail(CC_ERR_ARG, "cc_server_enqueue_many: n < 0");
    if (n > 0 && (!kinds || !data || !k)) return server_fail(CC_ERR_ARG, "cc_server_enqueue_many: null array");
    char msg[160];
    for (int64_t i = 0; i < n; i++) {  // everything is checked before anything is accepted
        const char* why = nullptr;
        if (kinds[i] != CC_OP_UPDATE && kinds[i] != CC_OP_QUERY) why = "unknown kind";
        else if (k[i] < 0 || k[i] > s->cap || k[i] > INT32_MAX) why = "k out of range (larger than the staging ring?)";
        else if (k[i] > 0 && !data[i]) why = "null data";
        else if (k[i] > 0 && kinds[i] == CC_OP_QUERY && (!out || !out[i])) why = "null out for a query";
        if (why) {
            snprintf(msg, sizeof msg, "cc_server_enqueue_many: request %lld: %s", (long long)i, why);
            return server_fail(CC_ERR_ARG, msg);
        }
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->err != CC_OK) return server_fail(s->err, s->errmsg.c_str());
    if (s->stop) return server_fail(CC_ERR_ARG, "cc_server_enqueue_many: server is stopping");
    const double t = now_s();
    if (first_ticket) *first_ticket = (uint64_t)s->reqs.size();
    for (int64_t i = 0; i < n; i++) {
        Req r;
        r.kind = kinds[i];
        r.data = data[i];
        r.k = k[i];
        r.out = kinds[i] == CC_OP_QUERY ? out[i] : nullptr;
        r.t_arrive = t;
        s->reqs.push_back(r);
        if (r.kind == CC_OP_UPDATE) { s->n_upd++; s->edges += r.k; } else { s->n_qry++; s->pairs += r.k; }
    }
    if (n > 0) s->cv_work.notify_one();
    return CC_OK;
}

cc_status cc_server_wait(cc_server* s, uint64_t ticket, double* latency_s) {
    if (!s) return server_fail(CC_ERR_ARG, "cc_server_wait: null server");
    std::unique_lock<std::mutex> lk(s->mu);
    if (ticket >= s->reqs.size()) return server_fail(CC_ERR_ARG, "cc_server_wait: unknown ticket");
    s->cv_done.wait(lk, [&] { return s->reqs[ticket].done || s->err != CC_OK; });
    if (s->err != CC_OK) return server_fail(s->err, s->errmsg.c_str());
    if (latency_s) *latency_s = s->reqs[ticket].t_done - s->reqs[ticket].t_arrive;
    return CC_OK;
}

cc_status cc_server_drain(cc_server* s) {
    if (!s) return server_fail(CC_ERR_ARG, "cc_server_drain: null server");
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] { return s->completed == (int64_t)s->reqs.size() || s->err != CC_OK; });
    if (s->err != CC_OK) return server_fail(s->err, s->errmsg.c_str());
    return CC_OK;
}

cc_status cc_server_get_stats(cc_server* s, cc_server_stats* out) {
    if (!s || !out) return server_fail(CC_ERR_ARG, "cc_server_get_stats: null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    out->requests = (int64_t)s->reqs.size();
    out->updates = s->n_upd;
    out->queries = s->n_qry;
    out->completed = s->completed;
    out->groups = s->groups;
    out->edges = s->edges;
    out->pairs = s->pairs;
    return CC_OK;
}

cc_status cc_server_latencies(cc_server* s, double* out, int64_t n, int64_t* written) {
    if (!s || (n > 0 && !out)) return server_fail(CC_ERR_ARG, "cc_server_latencies: null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    const int64_t m = n < (int64_t)s->reqs.size() ? n : (int64_t)s->reqs.size();
    for (int64_t i = 0; i < m; i++)
        out[i] = s->reqs[i].done ? s->reqs[i].t_done - s->reqs[i].t_arrive : -1.0;
    if (written) *written = m;
    return CC_OK;
}

cc_status cc_server_destroy(cc_server* s) {
    if (!s) return CC_OK;
    cc_status st = CC_OK;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        s->cv_done.wait(lk, [&] { return s->completed == (int64_t)s->reqs.size() || s->err != CC_OK; });
        s->stop = true;
        s->cv_work.notify_all();
        s->cv_reap.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->cv_reap.notify_all();
    }
    if (s->reaper.joinable()) s->reaper.join();
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    if (cudaStreamSynchronize(s->compute) != cudaSuccess || cudaStreamSynchronize(s->d2h) != cudaSuccess)
        st = server_fail(CC_ERR_CUDA, "cc_server_destroy: sync");
    cudaStreamSynchronize(s->h2d);
    cc_set_stream(s->ctx, s->prev_stream);
    for (Group* g : s->inflight) {
        if (g->ev) cudaEventDestroy(g->ev);
        delete g;
    }
    for (cudaEvent_t ev : s->spare_events) cudaEventDestroy(ev);
    cudaFree(s->ring[0].buf);
    cudaFree(s->ring[1].buf);
    cudaFree(s->ring_out);
    for (cudaEvent_t ev : s->run_ev) cudaEventDestroy(ev);
    cudaEventDestroy(s->ev_q);
    cudaStreamDestroy(s->compute);
    cudaStreamDestroy(s->h2d);
    cudaStreamDestroy(s->d2h);
    cudaSetDevice(prev);
    if (s->err != CC_OK && st == CC_OK) st = server_fail(s->err, s->errmsg.c_str());
    delete s;
    return st;
}

}  // extern "C"
