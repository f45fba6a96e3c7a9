// The C-ABI of include/cc.h: argument checks, handle state, error reporting,
// per-kernel launch counters and CUDA-event profiling around the launchers.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <algorithm>
#include <mutex>
#include <vector>

#include "cc.h"
#include "cc_internal.cuh"

namespace {

thread_local std::string g_err;

cc_status fail(cc_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

cc_status cuda_fail(cudaError_t e, const char* what) {
    return fail(CC_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

struct Timed {
    int kind;
    cudaEvent_t a, b;
};

// Makes the handle's device current for the scope of an entry point.
struct DeviceScope {
    int prev = -1;
    cudaError_t err = cudaSuccess;
    explicit DeviceScope(int dev) {
        err = cudaGetDevice(&prev);
        if (err == cudaSuccess && prev != dev) err = cudaSetDevice(dev);
        else if (err == cudaSuccess) prev = -1;
    }
    ~DeviceScope() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Persisting-L2 bookkeeping per device (CC_OPT_L2_PERSIST). Handles with an
// access-policy window raise the context's persisting-L2 limit; when the last
// of them on a device lets go (option off, or destroyed) the limit found
// before the first one is put back and every persisting line is turned back
// into a normal one. Without that, lines of a freed forest stay persisting,
// and with the raised set-aside they keep that part of L2 from every later
// kernel in the process.
struct PersistState {
    int users = 0;
    size_t saved_limit = 0;  // the limit before the first user raised it
    size_t limit = 0;        // the limit as raised
};
std::mutex g_persist_mu;
PersistState g_persist[64];

cudaError_t persist_acquire(int dev, size_t want) {
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_persist_mu);
    PersistState& p = g_persist[dev];
    if (p.users == 0) {
        cudaError_t e = cudaDeviceGetLimit(&p.saved_limit, cudaLimitPersistingL2CacheSize);
        if (e != cudaSuccess) return e;
        p.limit = p.saved_limit;
    }
    if (want > p.limit) {
        cudaError_t e = cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want);
        if (e != cudaSuccess) return e;
        p.limit = want;
    }
    p.users++;
    return cudaSuccess;
}

// Called with the device current and the releasing handle's work finished.
void persist_release(int dev) {
    if (dev < 0 || dev >= 64) return;
    std::lock_guard<std::mutex> lk(g_persist_mu);
    PersistState& p = g_persist[dev];
    if (p.users <= 0 || --p.users > 0) return;
    cudaCtxResetPersistingL2Cache();
    cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, p.saved_limit);
    p.limit = p.saved_limit;
}

const int64_t kDefaults[CC_OPT__COUNT] = {256, 2, 1, CC_COMPRESS_ALL, 0, 0, 0, 0,
                                          512, 1, 65536, 1, 0, 0, 0, 0, 0, 1, 0, 0, 1, 0, 0, 0};

// Minibatches below this many edges are never reordered (CC_OPT_EDGE_ORDER):
// their parent reads are too few to share L2 lines.
constexpr int64_t kOrderMinEdges = 4096;

}  // namespace

struct cc_ctx {
    int device = 0;
    int64_t n = 0;
    int* parent = nullptr;
    cc::DevState* ds = nullptr;
    cudaStream_t stream = nullptr;
    int64_t opt[CC_OPT__COUNT];
    uint64_t launches[CC_K__COUNT] = {};
    double ms[CC_K__COUNT] = {};
    std::vector<Timed> pending;
    std::vector<cudaEvent_t> spare;
    uint64_t update_calls = 0;
    bool flat = true;  // every tree has height <= 1
    cudaAccessPolicyWindow window = {};  // L2 window over parent (num_bytes 0 = off)

    // batched form
    int32_t G = 1;
    std::vector<int64_t> seg_off_h;  // G + 1 offsets
    int64_t* seg_off = nullptr;      // device copy
    int64_t cap_ops = 0;             // capacity of the table buffers, in ops
    size_t table_bytes = 0;
    // pinned host tables, two: the host fills one while the graph launched
    // with the other (its copy and its kernel) may still be queued or running
    void* staging[2] = {nullptr, nullptr};
    void* tables = nullptr;          // device tables
    cudaEvent_t staging_free[2] = {nullptr, nullptr};  // recorded after the submit that used it
    bool staging_pending[2] = {false, false};
    int stage = 0;                   // the staging buffer the next submit fills
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t graph_exec[2] = {nullptr, nullptr};  // captured with staging[0] / staging[1]
    int64_t graph_key[2][5] = {{-1, -1, -1, -1, -1}, {-1, -1, -1, -1, -1}};
    std::vector<int> bucket_count, op_begin_h, order_h;
    std::vector<int64_t> work_h;

    // the paper's schedule (CC_OPT_UPDATE_SCHEDULE = 1)
    int* a2 = nullptr;            // A'': compacted pairs of distinct roots
    int64_t a2_cap = 0;           // in pairs
    int* comp = nullptr;          // component labels of A'' endpoints (n entries)
    unsigned* pcount = nullptr;   // device: [0] = |A''|, [1] = hooked flag, [2] = rounds (graph)
    cudaGraphExec_t sv_exec = nullptr;  // the hooking rounds as one graph (CC_OPT_SV_GRAPH)
    const int* sv_a2 = nullptr;         // ... built for this A'' buffer,
    int sv_grid = 0, sv_block = 0;      // ... and this launch shape
    bool stats_on_device = false;       // last_nonloop / last_rounds still to be read from pcount
    int64_t last_nonloop = 0;
    int32_t last_rounds = 0;

    // the two-pass Bulk-Update (update variant 4)
    int4* live = nullptr;           // open edges of the current minibatch
    int64_t live_cap = 0;           // in entries
    unsigned* live_count = nullptr; // the two alternating list counters
    uint64_t live_seq = 0;          // two-pass updates so far (selects the counter)

    // locality order of the edges (CC_OPT_EDGE_ORDER)
    int* order_buf = nullptr;       // the ordered copy of a minibatch (2 ints per edge)
    int64_t order_cap = 0;          // in edges
    int* order_hist = nullptr;      // bucket totals, fill counters and a done counter
    int64_t order_hist_cap = 0;     // in ints
    bool order_dirty = false;       // a failed launch may have left the counters non-zero

    // largest-component filter (CC_OPT_BIG_FILTER)
    unsigned* big = nullptr;        // n bits, written by full compression passes

    // union by size (CC_OPT_LINK = 1)
    int* size = nullptr;                 // tree sizes, meaningful at roots
    unsigned long long* best = nullptr;  // per-component vote of the join step
    bool fresh = true;                   // no edge since create / reset

    // Bulk-Find (CC_OPT_BULK_FIND, cc_bulk_find)
    cc::BulkFindState bf;
};

namespace {

cudaEvent_t take_event(cc_ctx* c) {
    if (!c->spare.empty()) {
        cudaEvent_t e = c->spare.back();
        c->spare.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Enqueue one kernel through `launch`, counting it and (when profiling) timing
// it with a pair of events on the handle's stream.
template <class F>
cc_status run(cc_ctx* c, int kind, const char* what, F&& launch) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (c->opt[CC_OPT_PROFILE]) {
        a = take_event(c);
        b = take_event(c);
        if (a && b) cudaEventRecord(a, c->stream);
    }
    cudaError_t e = launch();
    c->launches[kind]++;
    if (a && b) {
        cudaEventRecord(b, c->stream);
        c->pending.push_back({kind, a, b});
    }
    if (e != cudaSuccess) return cuda_fail(e, what);
    return CC_OK;
}

cc::Launch cfg_of(const cc_ctx* c) {
    return cc::Launch{(int)c->opt[CC_OPT_BLOCK], (int)c->opt[CC_OPT_EDGES_PER_THREAD],
                      (int)c->opt[CC_OPT_UPDATE_VARIANT], (int)c->opt[CC_OPT_QUERY_VARIANT],
                      c->window.num_bytes > 0 ? &c->window : nullptr, (int)c->opt[CC_OPT_PDL],
                      (int)c->opt[CC_OPT_QUERY_PAIRS_PER_THREAD], (int)(c->opt[CC_OPT_HOOK] == 1),
                      (int)c->opt[CC_OPT_HOOK_WARP], c->opt[CC_OPT_BIG_FILTER] > 0 ? c->big : nullptr};
}

// The largest-component bitmap no longer describes the forest (reset, or a
// forest loaded from outside): off until the next full compression pass.
cudaError_t big_invalidate(cc_ctx* c) {
    return cudaMemsetAsync(&c->ds->big_root, 0xff, sizeof(int), c->stream);
}

cc_status check_pairs(const int32_t* p, int64_t k, const char* name) {
    if (k < 0 || k > INT32_MAX) return fail(CC_ERR_ARG, "%s: k = %lld out of [0, 2^31-1]", name, (long long)k);
    if (k > 0 && !p) return fail(CC_ERR_ARG, "%s: null array with k > 0", name);
    if (k > 0 && reinterpret_cast<uintptr_t>(p) % 4 != 0) return fail(CC_ERR_ARG, "%s: array not 4-byte aligned", name);
    return CC_OK;
}

cc_status do_compress(cc_ctx* c, int scope, const int32_t* edges, int64_t k) {
    if (c->opt[CC_OPT_LINK] == 1) {  // union by size: only the full generic pass
        cc_status s = run(c, CC_K_COMPRESS_ALL, "compress(all, generic)", [&] {
            return cc::launch_compress_generic(c->parent, c->n, nullptr, nullptr, c->ds,
                                               (int)c->opt[CC_OPT_BLOCK], c->stream);
        });
        if (s == CC_OK) c->flat = true;
        return s;
    }
    if (scope == CC_COMPRESS_ALL) {
        unsigned* big = c->opt[CC_OPT_BIG_FILTER] > 0 ? c->big : nullptr;
        if (big) {
            cc_status s = run(c, CC_K_BIG_PICK, "compress(all): largest-tree pick", [&] {
                return cc::launch_big_pick(c->parent, c->n, (int)c->opt[CC_OPT_BIG_FILTER], c->ds, c->stream);
            });
            if (s != CC_OK) return s;
        }
        cc_status s = run(c, CC_K_COMPRESS_ALL, "compress(all)", [&] {
            return cc::launch_compress_all(c->parent, c->n, nullptr, c->ds, (int)c->opt[CC_OPT_BLOCK], c->stream, big);
        });
        if (s == CC_OK) c->flat = true;
        return s;
    }
    if (k == 0) return CC_OK;
    return run(c, CC_K_COMPRESS_TOUCHED, "compress(touched)", [&] {
        return cc::launch_compress_touched(c->parent, (int)c->n, edges, k, c->ds, cfg_of(c), c->stream);
    });
}

// Launch options of a Bulk-Update: CC_OPT_HOOK = 2 hooks with atomicMin only
// for the first Bulk-Update on an empty forest (`first`), CAS afterwards.
cc::Launch update_cfg(const cc_ctx* c, bool first) {
    cc::Launch cfg = cfg_of(c);
    if (c->opt[CC_OPT_HOOK] == 2) cfg.minhook = first ? 1 : 0;
    return cfg;
}

// One Bulk-Update as a filter pass and a live-edge pass (update variant 4).
// The list has room for k entries; growing it synchronises the stream once.
cc_status split_update(cc_ctx* c, const int32_t* edges, int64_t k, bool first, bool ordered, const int32_t* alt) {
    cudaError_t e = cudaSuccess;
    if (!c->live_count) {
        e = cudaMalloc(&c->live_count, 2 * sizeof(unsigned));
        if (e == cudaSuccess) e = cudaMemsetAsync(c->live_count, 0, 2 * sizeof(unsigned), c->stream);
        if (e != cudaSuccess) {
            cudaFree(c->live_count);
            c->live_count = nullptr;
            cudaGetLastError();
            return fail(CC_ERR_OOM, "update variant 4: list counters");
        }
    }
    if (k > c->live_cap) {
        int4* live = nullptr;
        e = cudaStreamSynchronize(c->stream);
        if (e == cudaSuccess) e = cudaMalloc(&live, sizeof(int4) * (size_t)k);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(CC_ERR_OOM, "update variant 4: list of %lld edges", (long long)k);
        }
        cudaFree(c->live);
        c->live = live;
        c->live_cap = k;
    }
    const int sel = (int)(c->live_seq & 1u);
    cc::Launch cfg = update_cfg(c, first);
    if (ordered && cfg.pdl == 2) cfg.pdl = 1;  // its edges were written by the kernel just before
    cfg.alt = alt;
    cc_status s = run(c, CC_K_UPDATE, "bulk_update (two passes)", [&] {
        return cc::launch_update_split(c->parent, (int)c->n, edges, k, c->ds, cfg, c->live,
                                       c->live_count, sel, c->stream);
    });
    if (s == CC_OK) {
        c->live_seq++;
        c->launches[CC_K_UPDATE]++;  // the second kernel
    }
    return s;
}

// CC_OPT_EDGE_ORDER: the minibatch bucketed by its smaller endpoints into the
// handle's scratch copy, which then replaces `edges` for the update. The
// scratch grows to the largest minibatch with one stream synchronisation;
// its bucket counters start at zero and every call leaves them at zero.
// skip_big: the largest-component bitmap when the update kernel that follows
// takes the caller's edges as BigArgs::alt; the order kernels then do nothing
// while the bitmap is in use.
cc_status order_edges(cc_ctx* c, const int32_t** edges, int64_t k, const unsigned* skip_big) {
    const int b = (int)c->opt[CC_OPT_EDGE_ORDER];
    const int64_t counters = cc::order_counter_ints(b);
    if (k > c->order_cap || counters > c->order_hist_cap || c->order_dirty) {
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(e, "edge order: sync");
        if (k > c->order_cap) {
            int* q = nullptr;
            e = cudaMalloc(&q, sizeof(int) * 2 * (size_t)k);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(CC_ERR_OOM, "edge order: copy of %lld edges", (long long)k);
            }
            cudaFree(c->order_buf);
            c->order_buf = q;
            c->order_cap = k;
        }
        if (counters > c->order_hist_cap) {
            int* q = nullptr;
            e = cudaMalloc(&q, sizeof(int) * (size_t)counters);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(CC_ERR_OOM, "edge order: bucket counters");
            }
            cudaFree(c->order_hist);
            c->order_hist = q;
            c->order_hist_cap = counters;
        }
        e = cudaMemsetAsync(c->order_hist, 0, sizeof(int) * (size_t)c->order_hist_cap, c->stream);
        if (e != cudaSuccess) return cuda_fail(e, "edge order: clear counters");
        c->order_dirty = false;
    }
    int kernels = 1;
    cc_status s = run(c, CC_K_ORDER, "edge order", [&] {
        return cc::launch_order_edges(*edges, k, (int)c->n, b, c->order_hist, c->order_buf,
                                      (int)c->opt[CC_OPT_PDL], c->stream, &kernels, skip_big, c->ds);
    });
    if (s != CC_OK) {
        c->order_dirty = true;  // the counters may be left non-zero
        return s;
    }
    c->launches[CC_K_ORDER] += kernels - 1;  // run() counted one
    *edges = c->order_buf;
    return s;
}

// Steps 2-3 of the paper's schedule without a host round trip: the hooking
// rounds as one graph launch (build_sv_loop), then the join, on a grid of 8
// CTAs per SM (the kernels stride over A'', whose size they read on the
// device). |A''| and the round count stay on the device until asked for.
cc_status paper_rounds_graph(cc_ctx* c, int block) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    const int grid = 8 * (sms > 0 ? sms : 1);
    if (!c->sv_exec || c->sv_a2 != c->a2 || c->sv_grid != grid || c->sv_block != block) {
        if (c->sv_exec) cudaGraphExecDestroy(c->sv_exec);
        c->sv_exec = nullptr;
        cudaError_t e = cc::build_sv_loop(c->a2, c->pcount, c->comp, c->ds, grid, block, &c->sv_exec);
        if (e != cudaSuccess) return cuda_fail(e, "schedule 1: building the rounds graph");
        c->sv_a2 = c->a2;
        c->sv_grid = grid;
        c->sv_block = block;
    }
    cc_status st = run(c, CC_K_UPDATE, "schedule 1: components rounds (graph)", [&] {
        return cudaGraphLaunch(c->sv_exec, c->stream);
    });
    if (st != CC_OK) return st;
    c->stats_on_device = true;
    if (c->opt[CC_OPT_LINK] == 1) {
        c->launches[CC_K_UPDATE]++;  // vote, then join
        return run(c, CC_K_UPDATE, "schedule 1: size join", [&] {
            return cc::launch_size_join(c->a2, c->pcount, c->comp, c->parent, c->size, c->best, c->ds,
                                        grid, block, c->stream);
        });
    }
    return run(c, CC_K_UPDATE, "schedule 1: join", [&] {
        return cc::launch_join(c->a2, c->pcount, c->comp, c->parent, c->ds, grid, block, c->stream);
    });
}

// The last update's |A''| and round count, from the device when the rounds
// ran as a graph. Synchronises the stream in that case.
cc_status refresh_schedule_stats(cc_ctx* c) {
    if (!c->stats_on_device) return CC_OK;
    unsigned h[3] = {0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(h, c->pcount, sizeof h, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "schedule 1: reading the round statistics");
    c->last_nonloop = h[0];
    c->last_rounds = (int32_t)h[2];
    c->stats_on_device = false;
    return CC_OK;
}

// Algorithm 2 as written, one Bulk-Update: relabel + filter, CC rounds, join.
cc_status paper_update(cc_ctx* c, const int32_t* edges, int64_t k) {
    cudaError_t e = cudaSuccess;
    if (!c->comp) {
        e = cudaMalloc(&c->comp, sizeof(int) * (size_t)c->n);
        if (e == cudaSuccess) e = cudaMalloc(&c->pcount, 4 * sizeof(unsigned));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(CC_ERR_OOM, "schedule 1: component array of %lld entries", (long long)c->n);
        }
    }
    if (k > c->a2_cap) {
        int* a2 = nullptr;
        e = cudaStreamSynchronize(c->stream);
        if (e == cudaSuccess) e = cudaMalloc(&a2, sizeof(int) * 2 * (size_t)k);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(CC_ERR_OOM, "schedule 1: A'' buffer of %lld pairs", (long long)k);
        }
        cudaFree(c->a2);
        c->a2 = a2;
        c->a2_cap = k;
    }
    const int block = (int)c->opt[CC_OPT_BLOCK];
    if (c->opt[CC_OPT_BULK_FIND] == 1) {  // relabel with one Bulk-Find over all 2k endpoints
        const uint64_t before = c->bf.launches;
        int64_t cres = c->bf.cap_res;
        if (2 * k > cres) {
            int* q = nullptr;
            e = cudaMalloc(&q, sizeof(int) * 2 * (size_t)k);
            if (e != cudaSuccess) { cudaGetLastError(); return fail(CC_ERR_OOM, "schedule 1: root buffer"); }
            cudaFree(c->bf.res);
            c->bf.res = q;
            c->bf.cap_res = 2 * k;
        }
        e = cc::bulk_find(c->bf, c->parent, (int)c->n, edges, 2 * k, c->bf.res, c->ds, c->stream);
        c->launches[CC_K_UPDATE] += c->bf.launches - before;
        if (e != cudaSuccess) return cuda_fail(e, "schedule 1: Bulk-Find relabel");
    }
    cc_status st = run(c, CC_K_UPDATE, "schedule 1: relabel", [&]() -> cudaError_t {
        cudaError_t e1 = cudaMemsetAsync(c->pcount, 0, 2 * sizeof(unsigned), c->stream);
        if (e1 != cudaSuccess) return e1;
        if (c->opt[CC_OPT_BULK_FIND] == 1)
            return cc::launch_filter_roots(c->bf.res, k, c->a2, c->pcount, c->comp,
                                           c->opt[CC_OPT_LINK] == 1 ? c->best : nullptr, block, c->stream);
        if (c->opt[CC_OPT_LINK] == 1)
            return cc::launch_relabel_generic(c->parent, (int)c->n, edges, k, c->a2, c->pcount, c->comp,
                                              c->best, c->ds, block, c->stream);
        return cc::launch_relabel(c->parent, (int)c->n, edges, k, c->a2, c->pcount, c->comp, c->ds, block, c->stream);
    });
    if (st != CC_OK) return st;
    if (c->opt[CC_OPT_SV_GRAPH] == 1) return paper_rounds_graph(c, block);
    c->stats_on_device = false;
    unsigned m2 = 0;
    e = cudaMemcpyAsync(&m2, c->pcount, sizeof m2, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "schedule 1: read |A''|");
    c->last_nonloop = m2;
    c->last_rounds = 0;
    if (m2 == 0) return CC_OK;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    int64_t g = (2 * (int64_t)m2 + block - 1) / block;
    const int grid = (int)(g < 8LL * sms ? g : 8LL * sms);
    // each round with a hook removes at least one component root, so at most
    // 2|A''| rounds can hook; the next one finds nothing to do
    const int64_t max_rounds = 2 * (int64_t)m2 + 1;
    for (int64_t r = 0;; r++) {
        if (r >= max_rounds) return fail(CC_ERR_CORRUPT, "schedule 1: connected components did not converge");
        unsigned hooked = 0;
        st = run(c, CC_K_UPDATE, "schedule 1: components round", [&]() -> cudaError_t {
            cudaError_t e1 = cudaMemsetAsync(c->pcount + 1, 0, sizeof(unsigned), c->stream);
            if (e1 != cudaSuccess) return e1;
            return cc::launch_sv_round(c->a2, c->pcount, c->comp, c->pcount + 1, grid, block, c->stream);
        });
        if (st != CC_OK) return st;
        c->launches[CC_K_UPDATE]++;  // a round is two kernels: hook, then jump
        e = cudaMemcpyAsync(&hooked, c->pcount + 1, sizeof hooked, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(e, "schedule 1: read round flag");
        c->last_rounds = (int32_t)(r + 1);
        if (!hooked) break;
    }
    if (c->opt[CC_OPT_LINK] == 1) {
        c->launches[CC_K_UPDATE]++;  // vote, then join
        return run(c, CC_K_UPDATE, "schedule 1: size join", [&] {
            return cc::launch_size_join(c->a2, c->pcount, c->comp, c->parent, c->size, c->best, c->ds,
                                        grid, block, c->stream);
        });
    }
    return run(c, CC_K_UPDATE, "schedule 1: join", [&] {
        return cc::launch_join(c->a2, c->pcount, c->comp, c->parent, c->ds, grid, block, c->stream);
    });
}

bool by_size(const cc_ctx* c) { return c->opt[CC_OPT_LINK] == 1; }

}  // namespace

namespace cc {
// Lets the other translation units leave a message for cc_last_error_string().
cc_status record_error(cc_status s, const char* msg) { return fail(s, "%s", msg); }
cudaStream_t ctx_stream(const cc_ctx* c) { return c->stream; }
int ctx_device(const cc_ctx* c) { return c->device; }
int32_t ctx_graphs(const cc_ctx* c) { return c->G; }
}  // namespace cc

#define CC_CHECK_CTX(c)                                            \
    do {                                                           \
        if (!(c)) return fail(CC_ERR_ARG, "null cc_ctx handle");   \
    } while (0)

#define CC_DEVICE(c)                                                       \
    DeviceScope scope_(c->device);                                         \
    if (scope_.err != cudaSuccess) return cuda_fail(scope_.err, "cudaSetDevice")

extern "C" {

const char* cc_status_string(cc_status s) {
    switch (s) {
        case CC_OK: return "CC_OK";
        case CC_ERR_ARG: return "CC_ERR_ARG";
        case CC_ERR_OOM: return "CC_ERR_OOM";
        case CC_ERR_CUDA: return "CC_ERR_CUDA";
        case CC_ERR_RANGE: return "CC_ERR_RANGE";
        case CC_ERR_CORRUPT: return "CC_ERR_CORRUPT";
        case CC_ERR_LABELS: return "CC_ERR_LABELS";
        case CC_ERR_UNSUPPORTED: return "CC_ERR_UNSUPPORTED";
    }
    return "CC_ERR_?";
}

const char* cc_last_error_string(void) { return g_err.c_str(); }

cc_status cc_create(int64_t n, cc_ctx** out) {
    if (!out) return fail(CC_ERR_ARG, "cc_create: out is null");
    *out = nullptr;
    if (n < 1 || n > INT32_MAX) return fail(CC_ERR_ARG, "cc_create: n = %lld out of [1, 2^31-1]", (long long)n);
    cc_ctx* c = new (std::nothrow) cc_ctx();
    if (!c) return fail(CC_ERR_OOM, "cc_create: host allocation failed");
    memcpy(c->opt, kDefaults, sizeof kDefaults);
    c->n = n;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "cc_create: cudaGetDevice");
    }
    e = cudaMalloc(&c->parent, (size_t)n * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->ds, sizeof(cc::DevState));
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(c->parent);
        delete c;
        return fail(e == cudaErrorMemoryAllocation ? CC_ERR_OOM : CC_ERR_CUDA,
                    "cc_create(%lld): %s", (long long)n, cudaGetErrorString(e));
    }
    e = cudaMemsetAsync(c->ds, 0, sizeof(cc::DevState), c->stream);
    if (e == cudaSuccess) e = big_invalidate(c);
    if (e == cudaSuccess) e = cc::launch_reset(c->parent, n, 256, c->stream);
    c->launches[CC_K_RESET]++;
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaFree(c->parent);
        cudaFree(c->ds);
        delete c;
        return cuda_fail(e, "cc_create: init");
    }
    *out = c;
    return CC_OK;
}

cc_status cc_destroy(cc_ctx* c) {
    if (!c) return CC_OK;
    cc_status s = CC_OK;
    {
        DeviceScope scope(c->device);
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) s = cuda_fail(e, "cc_destroy: sync");
        for (auto& t : c->pending) {
            cudaEventDestroy(t.a);
            cudaEventDestroy(t.b);
        }
        for (auto ev : c->spare) cudaEventDestroy(ev);
        for (int j = 0; j < 2; j++) {
            if (c->graph_exec[j]) cudaGraphExecDestroy(c->graph_exec[j]);
            if (c->staging_free[j]) cudaEventDestroy(c->staging_free[j]);
            if (c->staging[j]) cudaFreeHost(c->staging[j]);
        }
        if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
        cudaFree(c->tables);
        cudaFree(c->seg_off);
        cudaFree(c->a2);
        cudaFree(c->comp);
        cudaFree(c->pcount);
        if (c->sv_exec) cudaGraphExecDestroy(c->sv_exec);
        cudaFree(c->size);
        cudaFree(c->best);
        cudaFree(c->live);
        cudaFree(c->live_count);
        cudaFree(c->order_buf);
        cudaFree(c->order_hist);
        cudaFree(c->big);
        cc::bulk_find_free(c->bf);
        if (c->window.num_bytes > 0) persist_release(c->device);
        cudaFree(c->parent);
        cudaFree(c->ds);
    }
    delete c;
    return s;
}

cc_status cc_set_stream(cc_ctx* c, cc_stream_t stream) {
    CC_CHECK_CTX(c);
    c->stream = reinterpret_cast<cudaStream_t>(stream);
    return CC_OK;
}

cc_status cc_sync(cc_ctx* c) {
    CC_CHECK_CTX(c);
    CC_DEVICE(c);
    unsigned st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, &c->ds->status, sizeof st, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cc_sync");
    if (st) {
        e = cudaMemsetAsync(&c->ds->status, 0, sizeof(unsigned), c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cc_sync: clear status");
        if (st & cc::ST_CORRUPT) return fail(CC_ERR_CORRUPT, "a kernel found parent[v] > v");
        return fail(CC_ERR_RANGE, "an edge or query had an endpoint outside [0, %lld)", (long long)c->n);
    }
    return CC_OK;
}

cc_status cc_reset(cc_ctx* c) {
    CC_CHECK_CTX(c);
    CC_DEVICE(c);
    cudaError_t e = cudaMemsetAsync(&c->ds->unions, 0, sizeof(unsigned long long), c->stream);
    if (e == cudaSuccess) e = big_invalidate(c);
    if (e != cudaSuccess) return cuda_fail(e, "cc_reset");
    cc_status s = run(c, CC_K_RESET, "reset", [&] {
        return cc::launch_reset(c->parent, c->n, (int)c->opt[CC_OPT_BLOCK], c->stream);
    });
    if (s == CC_OK) {
        c->flat = true;
        c->update_calls = 0;
        c->fresh = true;
        if (c->size) {
            cudaError_t e2 = cc::launch_fill(c->size, c->n, 1, c->stream);
            if (e2 != cudaSuccess) return cuda_fail(e2, "cc_reset: sizes");
        }
    }
    return s;
}

cc_status cc_bulk_update(cc_ctx* c, const int32_t* edges, int64_t k) {
    CC_CHECK_CTX(c);
    cc_status s = check_pairs(edges, k, "cc_bulk_update");
    if (s != CC_OK) return s;
    if (c->G > 1) return fail(CC_ERR_UNSUPPORTED, "cc_bulk_update on a segmented handle: use cc_submit");
    if (k == 0) return CC_OK;
    CC_DEVICE(c);
    if (by_size(c) && c->opt[CC_OPT_UPDATE_SCHEDULE] != 1)
        return fail(CC_ERR_UNSUPPORTED, "union by size (CC_OPT_LINK = 1) needs CC_OPT_UPDATE_SCHEDULE = 1");
    const bool first = c->fresh;  // the forest has no edge yet
    const int32_t* given = edges;
    const bool fused = c->opt[CC_OPT_UPDATE_SCHEDULE] != 1;
    // the fused kernels read the caller's edges instead of an ordered copy
    // while the largest-component bitmap is in use (cc::BigArgs)
    const unsigned* big = fused ? cfg_of(c).big : nullptr;
    bool ordered = false;
    if (c->opt[CC_OPT_EDGE_ORDER] > 0 && k >= kOrderMinEdges) {
        s = order_edges(c, &edges, k, big);
        if (s != CC_OK) return s;
        ordered = true;
    }
    const int32_t* alt = ordered && big ? given : nullptr;
    c->fresh = false;
    if (!fused) {
        s = paper_update(c, edges, k);
    } else if (c->opt[CC_OPT_UPDATE_VARIANT] == 4) {
        s = split_update(c, edges, k, first, ordered, alt);
    } else {
        cc::Launch cfg = update_cfg(c, first);
        if (ordered && cfg.pdl == 2) cfg.pdl = 1;  // its edges were written by the kernel just before
        cfg.alt = alt;
        s = run(c, CC_K_UPDATE, "bulk_update", [&] {
            return cc::launch_update(c->parent, (int)c->n, edges, k, c->ds, cfg, c->stream);
        });
    }
    if (s != CC_OK) return s;
    c->flat = false;
    c->update_calls++;
    const int64_t every = c->opt[CC_OPT_COMPRESS_EVERY];
    if (every > 0 && c->update_calls % (uint64_t)every == 0)
        return do_compress(c, (int)c->opt[CC_OPT_COMPRESS_SCOPE], given, k);  // a set: same endpoints
    return CC_OK;
}

cc_status cc_bulk_query(cc_ctx* c, const int32_t* pairs, int64_t k, uint8_t* out) {
    CC_CHECK_CTX(c);
    cc_status s = check_pairs(pairs, k, "cc_bulk_query");
    if (s != CC_OK) return s;
    if (k > 0 && !out) return fail(CC_ERR_ARG, "cc_bulk_query: out is null");
    if (k == 0) return CC_OK;
    CC_DEVICE(c);
    if (c->opt[CC_OPT_BULK_FIND] == 1) {
        const uint64_t before = c->bf.launches;
        s = run(c, CC_K_QUERY, "bulk_query(Bulk-Find)", [&] {
            return cc::bulk_find_query(c->bf, c->parent, (int)c->n, pairs, k, out, c->ds, c->stream);
        });
        c->launches[CC_K_QUERY] += c->bf.launches - before - 1;  // run() counted one
        return s;
    }
    if (by_size(c)) {
        const bool flat = c->flat;
        s = run(c, CC_K_QUERY, "bulk_query(generic)", [&] {
            return cc::launch_query_generic(c->parent, (int)c->n, pairs, k, out, c->ds, flat,
                                            (int)c->opt[CC_OPT_BLOCK], c->stream);
        });
        if (s == CC_OK && !flat) c->flat = false;
        return s;
    }
    const int64_t qh = c->opt[CC_OPT_QUERY_HALVING];
    const int mode = c->flat ? 2 : (qh == 2 ? 3 : qh == 1 ? 1 : 0);
    s = run(c, CC_K_QUERY, "bulk_query", [&] {
        return cc::launch_query(c->parent, (int)c->n, pairs, k, out, c->ds, mode, cfg_of(c), c->stream);
    });
    return s;
}

cc_status cc_compress(cc_ctx* c, int32_t scope, const int32_t* edges, int64_t k) {
    CC_CHECK_CTX(c);
    if (scope != CC_COMPRESS_ALL && scope != CC_COMPRESS_TOUCHED)
        return fail(CC_ERR_ARG, "cc_compress: unknown scope %d", scope);
    if (scope == CC_COMPRESS_TOUCHED) {
        cc_status s = check_pairs(edges, k, "cc_compress");
        if (s != CC_OK) return s;
        if (c->G > 1) return fail(CC_ERR_UNSUPPORTED, "touched compression on a segmented handle");
    }
    CC_DEVICE(c);
    return do_compress(c, scope, edges, k);
}

cc_status cc_labels(cc_ctx* c, int32_t* out) {
    CC_CHECK_CTX(c);
    if (!out) return fail(CC_ERR_ARG, "cc_labels: out is null");
    if (reinterpret_cast<uintptr_t>(out) % 4 != 0) return fail(CC_ERR_ARG, "cc_labels: out not 4-byte aligned");
    CC_DEVICE(c);
    if (by_size(c)) {
        if (!c->comp) {
            cudaError_t e = cudaMalloc(&c->comp, sizeof(int) * (size_t)c->n);
            if (e != cudaSuccess) { cudaGetLastError(); return fail(CC_ERR_OOM, "cc_labels: scratch"); }
        }
        cc_status s = run(c, CC_K_LABELS, "labels(generic)", [&] {
            return cc::launch_compress_generic(c->parent, c->n, out, c->comp, c->ds,
                                               (int)c->opt[CC_OPT_BLOCK], c->stream);
        });
        if (s == CC_OK) c->flat = true;
        return s;
    }
    cc_status s = run(c, CC_K_LABELS, "labels", [&] {
        return cc::launch_compress_all(c->parent, c->n, out, c->ds, (int)c->opt[CC_OPT_BLOCK], c->stream);
    });
    if (s == CC_OK) c->flat = true;
    return s;
}

cc_status cc_load_labels(cc_ctx* c, const int32_t* labels) {
    CC_CHECK_CTX(c);
    if (!labels) return fail(CC_ERR_ARG, "cc_load_labels: labels is null");
    if (reinterpret_cast<uintptr_t>(labels) % 4 != 0) return fail(CC_ERR_ARG, "cc_load_labels: not 4-byte aligned");
    if (c->G > 1) return fail(CC_ERR_UNSUPPORTED, "cc_load_labels on a segmented handle");
    CC_DEVICE(c);
    cudaError_t e = cudaMemsetAsync(&c->ds->labels_bad, 0, sizeof(unsigned), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(&c->ds->roots, 0, sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cc_load_labels");
    cc_status s = run(c, CC_K_LOAD, "load_labels(validate)", [&] {
        return cc::launch_validate_labels(labels, c->n, c->ds, 256, c->stream);
    });
    if (s != CC_OK) return s;
    cc::DevState h;
    e = cudaMemcpyAsync(&h, c->ds, sizeof h, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cc_load_labels: read back");
    if (h.labels_bad) return fail(CC_ERR_LABELS, "cc_load_labels: not a minimum-id labelling (need 0 <= l[v] <= v, l[l[v]] == l[v])");
    unsigned long long unions = (unsigned long long)c->n - h.roots;
    e = cudaMemcpyAsync(c->parent, labels, (size_t)c->n * sizeof(int), cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&c->ds->unions, &unions, sizeof unions, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = big_invalidate(c);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cc_load_labels: copy");
    c->flat = true;
    c->update_calls = 0;
    c->fresh = false;
    if (by_size(c)) {
        e = cc::launch_size_count(c->parent, c->n, c->size, c->ds, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cc_load_labels: sizes");
    }
    return CC_OK;
}

cc_status cc_copy_parent(cc_ctx* c, int32_t* out) {
    CC_CHECK_CTX(c);
    if (!out) return fail(CC_ERR_ARG, "cc_copy_parent: out is null");
    CC_DEVICE(c);
    cudaError_t e = cudaMemcpyAsync(out, c->parent, (size_t)c->n * sizeof(int), cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cc_copy_parent");
    return CC_OK;
}

cc_status cc_components(cc_ctx* c, int64_t* out) {
    CC_CHECK_CTX(c);
    if (!out) return fail(CC_ERR_ARG, "cc_components: out is null");
    CC_DEVICE(c);
    unsigned long long u = 0;
    cudaError_t e = cudaMemcpyAsync(&u, &c->ds->unions, sizeof u, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cc_components");
    *out = c->n - (int64_t)u;
    return CC_OK;
}

cc_status cc_create_segmented(int32_t G, const int64_t* n_per_graph, cc_ctx** out) {
    if (!out) return fail(CC_ERR_ARG, "cc_create_segmented: out is null");
    *out = nullptr;
    if (G < 1 || !n_per_graph) return fail(CC_ERR_ARG, "cc_create_segmented: need G >= 1 and sizes");
    std::vector<int64_t> off((size_t)G + 1, 0);
    for (int32_t g = 0; g < G; g++) {
        if (n_per_graph[g] < 1) return fail(CC_ERR_ARG, "cc_create_segmented: graph %d has n < 1", g);
        off[g + 1] = off[g] + n_per_graph[g];
        if (off[g + 1] > INT32_MAX) return fail(CC_ERR_ARG, "cc_create_segmented: total vertices exceed 2^31-1");
    }
    cc_ctx* c = nullptr;
    cc_status s = cc_create(off[G], &c);
    if (s != CC_OK) return s;
    c->G = G;
    c->seg_off_h = std::move(off);
    cudaError_t e = cudaMalloc(&c->seg_off, sizeof(int64_t) * (size_t)(G + 1));
    if (e == cudaSuccess)
        e = cudaMemcpy(c->seg_off, c->seg_off_h.data(), sizeof(int64_t) * (size_t)(G + 1), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cc_destroy(c);
        return fail(e == cudaErrorMemoryAllocation ? CC_ERR_OOM : CC_ERR_CUDA, "cc_create_segmented: %s", cudaGetErrorString(e));
    }
    *out = c;
    return CC_OK;
}

namespace {

// Table layout in the staging and device buffers (fixed by the capacities,
// so a captured graph keeps valid pointers): [nactive, pad x3][ops][op_begin
// G+1][order G].
struct TableLayout {
    size_t ops, op_begin, order, bytes;
};

TableLayout table_layout(int64_t cap_ops, int32_t G) {
    TableLayout L;
    L.ops = 16;
    L.op_begin = L.ops + sizeof(cc::SegOp) * (size_t)cap_ops;
    L.order = L.op_begin + sizeof(int) * (size_t)(G + 1);
    L.bytes = (L.order + sizeof(int) * (size_t)G + 255) / 256 * 256;
    return L;
}

cc_status ensure_tables(cc_ctx* c, int64_t nops) {
    if (!c->seg_off) {  // a plain handle is one graph
        c->seg_off_h = {0, c->n};
        cudaError_t e = cudaMalloc(&c->seg_off, sizeof(int64_t) * 2);
        if (e == cudaSuccess) e = cudaMemcpy(c->seg_off, c->seg_off_h.data(), sizeof(int64_t) * 2, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "cc_submit: segment offsets");
    }
    for (int j = 0; j < 2; j++)
        if (!c->staging_free[j]) {
            cudaError_t e = cudaEventCreateWithFlags(&c->staging_free[j], cudaEventDisableTiming);
            if (e != cudaSuccess) return cuda_fail(e, "cc_submit: event");
        }
    if (nops <= c->cap_ops) return CC_OK;
    int64_t cap = c->cap_ops ? c->cap_ops : 1024;
    while (cap < nops) cap *= 2;
    for (int j = 0; j < 2; j++)
        if (c->staging_pending[j]) {
            cudaEventSynchronize(c->staging_free[j]);
            c->staging_pending[j] = false;
        }
    const TableLayout L = table_layout(cap, c->G);
    void* staging[2] = {nullptr, nullptr};
    void* tables = nullptr;
    cudaError_t e = cudaMallocHost(&staging[0], L.bytes);
    if (e == cudaSuccess) e = cudaMallocHost(&staging[1], L.bytes);
    if (e == cudaSuccess) e = cudaMalloc(&tables, L.bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (staging[0]) cudaFreeHost(staging[0]);
        if (staging[1]) cudaFreeHost(staging[1]);
        return fail(CC_ERR_OOM, "cc_submit: table buffers of %zu bytes", L.bytes);
    }
    cudaStreamSynchronize(c->stream);  // the old tables may still be read by a running submit
    for (int j = 0; j < 2; j++) {
        if (c->staging[j]) cudaFreeHost(c->staging[j]);
        c->staging[j] = staging[j];
        if (c->graph_exec[j]) {
            cudaGraphExecDestroy(c->graph_exec[j]);
            c->graph_exec[j] = nullptr;
        }
    }
    cudaFree(c->tables);
    c->tables = tables;
    c->cap_ops = cap;
    c->table_bytes = L.bytes;
    return CC_OK;
}

cc::SegLaunch seg_cfg(const cc_ctx* c) {
    cc::SegLaunch cfg;
    cfg.block = (int)c->opt[CC_OPT_SEG_BLOCK];
    cfg.ept = (int)c->opt[CC_OPT_SEG_EDGES_PER_THREAD];
    cfg.smem_cap = (int)c->opt[CC_OPT_SEG_SMEM_CAP];
    cfg.max_ctas = (int)c->opt[CC_OPT_SEG_MAX_CTAS];
    return cfg;
}

}  // namespace

cc_status cc_submit(cc_ctx* c, const cc_op* ops, int64_t nops) {
    CC_CHECK_CTX(c);
    if (nops < 0 || nops > INT32_MAX) return fail(CC_ERR_ARG, "cc_submit: nops out of range");
    if (nops == 0) return CC_OK;
    if (!ops) return fail(CC_ERR_ARG, "cc_submit: ops is null");
    if (by_size(c)) return fail(CC_ERR_UNSUPPORTED, "cc_submit with union by size");
    for (int64_t i = 0; i < nops; i++) {
        const cc_op& o = ops[i];
        if (o.graph < 0 || o.graph >= c->G) return fail(CC_ERR_ARG, "cc_submit: op %lld: graph %d out of [0, %d)", (long long)i, o.graph, c->G);
        if (o.kind != CC_OP_UPDATE && o.kind != CC_OP_QUERY) return fail(CC_ERR_ARG, "cc_submit: op %lld: unknown kind %d", (long long)i, o.kind);
        if (o.k < 0 || o.k > INT32_MAX) return fail(CC_ERR_ARG, "cc_submit: op %lld: k out of range", (long long)i);
        if (o.k > 0 && (!o.data || reinterpret_cast<uintptr_t>(o.data) % 4)) return fail(CC_ERR_ARG, "cc_submit: op %lld: data null or not 4-byte aligned", (long long)i);
        if (o.k > 0 && o.kind == CC_OP_QUERY && !o.out) return fail(CC_ERR_ARG, "cc_submit: op %lld: out is null", (long long)i);
    }
    CC_DEVICE(c);
    cc_status st = ensure_tables(c, nops);
    if (st != CC_OK) return st;
    const int j = c->stage;
    if (c->staging_pending[j]) {  // the submit before the previous one used this buffer
        cudaError_t e = cudaEventSynchronize(c->staging_free[j]);
        if (e != cudaSuccess) return cuda_fail(e, "cc_submit: wait for staging");
        c->staging_pending[j] = false;
    }
    // bucket the operations by graph, keeping their order within a graph
    const int32_t G = c->G;
    const TableLayout L = table_layout(c->cap_ops, G);
    char* base = static_cast<char*>(c->staging[j]);
    cc::SegOp* sops = reinterpret_cast<cc::SegOp*>(base + L.ops);
    int* op_begin = reinterpret_cast<int*>(base + L.op_begin);
    int* order = reinterpret_cast<int*>(base + L.order);
    c->bucket_count.assign((size_t)G + 1, 0);
    c->work_h.assign((size_t)G, 0);
    for (int64_t i = 0; i < nops; i++) {
        c->bucket_count[ops[i].graph + 1]++;
        c->work_h[ops[i].graph] += ops[i].k;
    }
    op_begin[0] = 0;
    for (int32_t g = 0; g < G; g++) op_begin[g + 1] = op_begin[g] + c->bucket_count[g + 1];
    c->op_begin_h.assign(op_begin, op_begin + G + 1);
    for (int64_t i = 0; i < nops; i++) {
        const cc_op& o = ops[i];
        cc::SegOp& d = sops[c->op_begin_h[o.graph]++];
        d.data = o.data;
        d.out = o.out;
        d.k = o.k;
        d.kind = o.kind;
        d.pad = 0;
    }
    // graphs with work, largest first (a graph's cost grows with its ops and its size)
    c->order_h.clear();
    for (int32_t g = 0; g < G; g++)
        if (c->bucket_count[g + 1]) {
            c->work_h[g] += c->seg_off_h[g + 1] - c->seg_off_h[g];
            c->order_h.push_back(g);
        }
    std::stable_sort(c->order_h.begin(), c->order_h.end(),
                     [&](int a, int b) { return c->work_h[a] > c->work_h[b]; });
    memcpy(order, c->order_h.data(), sizeof(int) * c->order_h.size());
    reinterpret_cast<int*>(base)[0] = (int)c->order_h.size();

    cc::SegLaunch cfg = seg_cfg(c);
    char* dbase = static_cast<char*>(c->tables);
    cc::SegTables t;
    t.ops = reinterpret_cast<const cc::SegOp*>(dbase + L.ops);
    t.op_begin = reinterpret_cast<const int*>(dbase + L.op_begin);
    t.order = reinterpret_cast<const int*>(dbase + L.order);
    t.nactive = reinterpret_cast<const int*>(dbase);
    const int64_t key[5] = {cfg.block, cfg.ept, cfg.smem_cap, cfg.max_ctas, c->cap_ops};
    const bool use_graph = c->opt[CC_OPT_SEG_GRAPH] != 0;
    st = run(c, CC_K_SEGMENTED, "submit", [&]() -> cudaError_t {
        cudaError_t e;
        if (use_graph) {
            if (!c->graph_exec[j] || memcmp(key, c->graph_key[j], sizeof key) != 0) {
                if (c->graph_exec[j]) {
                    cudaGraphExecDestroy(c->graph_exec[j]);
                    c->graph_exec[j] = nullptr;
                }
                e = cc::prepare_segmented(cfg);
                if (e != cudaSuccess) return e;
                if (!c->capture_stream) {
                    e = cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking);
                    if (e != cudaSuccess) return e;
                }
                cudaGraph_t graph = nullptr;
                e = cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal);
                if (e != cudaSuccess) return e;
                cudaError_t e1 = cudaMemcpyAsync(c->tables, c->staging[j], c->table_bytes, cudaMemcpyHostToDevice, c->capture_stream);
                if (e1 == cudaSuccess) e1 = cudaMemsetAsync(&c->ds->queue, 0, sizeof(unsigned), c->capture_stream);
                if (e1 == cudaSuccess) e1 = cc::launch_segmented(c->parent, c->seg_off, t, &c->ds->queue, c->ds, cfg, c->capture_stream);
                e = cudaStreamEndCapture(c->capture_stream, &graph);
                if (e1 != cudaSuccess) e = e1;
                if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph_exec[j], graph, 0);
                if (graph) cudaGraphDestroy(graph);
                if (e != cudaSuccess) {
                    c->graph_exec[j] = nullptr;
                    return e;
                }
                memcpy(c->graph_key[j], key, sizeof key);
            }
            e = cudaGraphLaunch(c->graph_exec[j], c->stream);
        } else {
            e = cc::prepare_segmented(cfg);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(c->tables, c->staging[j], L.order + sizeof(int) * c->order_h.size(), cudaMemcpyHostToDevice, c->stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(&c->ds->queue, 0, sizeof(unsigned), c->stream);
            if (e == cudaSuccess) e = cc::launch_segmented(c->parent, c->seg_off, t, &c->ds->queue, c->ds, cfg, c->stream);
        }
        if (e == cudaSuccess) e = cudaEventRecord(c->staging_free[j], c->stream);
        return e;
    });
    if (st == CC_OK) {
        c->staging_pending[j] = true;
        c->stage = j ^ 1;
    }
    c->flat = false;
    c->fresh = false;
    return st;
}

cc_status cc_set_option(cc_ctx* c, int32_t option, int64_t value) {
    CC_CHECK_CTX(c);
    switch (option) {
        case CC_OPT_BLOCK:
            if (value < 64 || value > 1024 || value % 32) return fail(CC_ERR_ARG, "block %lld: need 64..1024, multiple of 32", (long long)value);
            break;
        case CC_OPT_EDGES_PER_THREAD:
            if (value != 1 && value != 2 && value != 4) return fail(CC_ERR_ARG, "edges per thread %lld: need 1, 2 or 4", (long long)value);
            break;
        case CC_OPT_COMPRESS_EVERY:
            if (value < 0) return fail(CC_ERR_ARG, "compress_every must be >= 0");
            break;
        case CC_OPT_COMPRESS_SCOPE:
            if (value != CC_COMPRESS_ALL && value != CC_COMPRESS_TOUCHED) return fail(CC_ERR_ARG, "unknown compress scope");
            break;
        case CC_OPT_QUERY_HALVING:
            if (value < 0 || value > 2) return fail(CC_ERR_ARG, "query halving %lld: need 0, 1 or 2", (long long)value);
            break;
        case CC_OPT_PDL:
            if (value < 0 || value > 2) return fail(CC_ERR_ARG, "pdl %lld: need 0, 1 or 2", (long long)value);
            break;
        case CC_OPT_SV_GRAPH:
            if (value != 0 && value != 1) return fail(CC_ERR_ARG, "option %d takes 0 or 1", option);
            break;
        case CC_OPT_HOOK:
            if (value < 0 || value > 2) return fail(CC_ERR_ARG, "hook %lld: need 0 (CAS), 1 (atomicMin) or 2 (atomicMin on an empty forest only)", (long long)value);
            break;
        case CC_OPT_QUERY_PAIRS_PER_THREAD:
            if (value != 0 && value != 1 && value != 2 && value != 4) return fail(CC_ERR_ARG, "query pairs per thread %lld: need 0, 1, 2 or 4", (long long)value);
            break;
        case CC_OPT_PROFILE:
            if (value != 0 && value != 1) return fail(CC_ERR_ARG, "option %d takes 0 or 1", option);
            break;
        case CC_OPT_SEG_BLOCK:
            if (value < 64 || value > 1024 || value % 32) return fail(CC_ERR_ARG, "seg block %lld: need 64..1024, multiple of 32", (long long)value);
            break;
        case CC_OPT_SEG_EDGES_PER_THREAD:
            if (value != 1 && value != 2 && value != 4) return fail(CC_ERR_ARG, "seg edges per thread %lld: need 1, 2 or 4", (long long)value);
            break;
        case CC_OPT_SEG_SMEM_CAP:
            if (value < 0 || value > 65536) return fail(CC_ERR_ARG, "seg smem cap %lld: need 0..65536", (long long)value);
            break;
        case CC_OPT_SEG_GRAPH:
            if (value != 0 && value != 1) return fail(CC_ERR_ARG, "option %d takes 0 or 1", option);
            break;
        case CC_OPT_SEG_MAX_CTAS:
            if (value < 0 || value > (1 << 20)) return fail(CC_ERR_ARG, "seg max ctas %lld out of range", (long long)value);
            break;
        case CC_OPT_QUERY_VARIANT:
            if (value < 0 || value > 2) return fail(CC_ERR_ARG, "query variant %lld: need 0, 1 or 2", (long long)value);
            break;
        case CC_OPT_BULK_FIND:
            if (value != 0 && value != 1) return fail(CC_ERR_ARG, "option %d takes 0 or 1", option);
            break;
        case CC_OPT_LINK: {
            if (value != 0 && value != 1) return fail(CC_ERR_ARG, "link %lld: need 0 (index) or 1 (size)", (long long)value);
            if (value == c->opt[CC_OPT_LINK]) break;
            if (!c->fresh) return fail(CC_ERR_ARG, "the link rule can only change while the forest has no edges (after create or reset)");
            if (c->G > 1) return fail(CC_ERR_UNSUPPORTED, "union by size on a segmented handle");
            if (value == 1) {
                DeviceScope scope(c->device);
                cudaError_t e = cudaSuccess;
                if (!c->size) e = cudaMalloc(&c->size, sizeof(int) * (size_t)c->n);
                if (e == cudaSuccess && !c->best) e = cudaMalloc(&c->best, sizeof(unsigned long long) * (size_t)c->n);
                if (e == cudaSuccess) e = cc::launch_fill(c->size, c->n, 1, c->stream);
                if (e != cudaSuccess) { cudaGetLastError(); return fail(CC_ERR_OOM, "union by size: size arrays"); }
            }
            break;
        }
        case CC_OPT_UPDATE_SCHEDULE:
            if (value != 0 && value != 1) return fail(CC_ERR_ARG, "update schedule %lld: need 0 or 1", (long long)value);
            break;
        case CC_OPT_HOOK_WARP:
            if (value != 0 && value != 1) return fail(CC_ERR_ARG, "option %d takes 0 or 1", option);
            break;
        case CC_OPT_BIG_FILTER:
            if (value < 0 || value > cc::kBigSample)
                return fail(CC_ERR_ARG, "big filter %lld: need 0 (off) or 1..%d (least sampled share)", (long long)value, cc::kBigSample);
            if (value > 0 && c->G > 1) return fail(CC_ERR_UNSUPPORTED, "the largest-component filter on a segmented handle");
            if (value > 0 && !c->big) {
                DeviceScope scope(c->device);
                const size_t words = (size_t)((c->n + 31) / 32);
                cudaError_t e = cudaMalloc(&c->big, words * sizeof(unsigned));
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    c->big = nullptr;
                    return fail(CC_ERR_OOM, "big filter: bitmap of %zu words", words);
                }
            }
            break;
        case CC_OPT_EDGE_ORDER:
            if (value != 0 && (value < 6 || value > 9))
                return fail(CC_ERR_ARG, "edge order %lld: need 0 (off) or 6..9 (log2 of the bucket count)", (long long)value);
            break;
        case CC_OPT_UPDATE_VARIANT:
            if (value < 0 || value > 5) return fail(CC_ERR_ARG, "update variant %lld: need 0..5", (long long)value);
            break;
        case CC_OPT_L2_PERSIST: {
            if (value != 0 && value != 1) return fail(CC_ERR_ARG, "option %d takes 0 or 1", option);
            const bool had = c->window.num_bytes > 0;
            if (value && had) break;  // already on
            DeviceScope scope(c->device);
            if (!value) {
                if (had) {
                    cudaError_t e = cudaStreamSynchronize(c->stream);
                    if (e != cudaSuccess) return cuda_fail(e, "L2 persist off: sync");
                    c->window = cudaAccessPolicyWindow{};
                    persist_release(c->device);
                }
                break;
            }
            {
                int max_persist = 0, max_window = 0;
                cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, c->device);
                cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, c->device);
                if (max_persist <= 0 || max_window <= 0)
                    return fail(CC_ERR_UNSUPPORTED, "no persisting L2 on this device");
                const size_t bytes = (size_t)c->n * sizeof(int);
                const size_t limit = bytes < (size_t)max_persist ? bytes : (size_t)max_persist;
                cudaError_t e = persist_acquire(c->device, limit);
                if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSetLimit(persisting L2)");
                c->window.base_ptr = c->parent;
                c->window.num_bytes = bytes < (size_t)max_window ? bytes : (size_t)max_window;
                c->window.hitRatio = (float)((double)limit / (double)c->window.num_bytes);
                if (c->window.hitRatio > 1.f) c->window.hitRatio = 1.f;
                c->window.hitProp = cudaAccessPropertyPersisting;
                c->window.missProp = cudaAccessPropertyStreaming;
            }
            break;
        }
        default:
            return fail(CC_ERR_ARG, "unknown option %d", option);
    }
    c->opt[option] = value;
    return CC_OK;
}

cc_status cc_get_option(const cc_ctx* c, int32_t option, int64_t* value) {
    CC_CHECK_CTX(c);
    if (!value) return fail(CC_ERR_ARG, "cc_get_option: value is null");
    if (option < 0 || option >= CC_OPT__COUNT) return fail(CC_ERR_ARG, "unknown option %d", option);
    *value = c->opt[option];
    return CC_OK;
}

cc_status cc_kernel_stats(cc_ctx* c, uint64_t* launches, double* ms) {
    CC_CHECK_CTX(c);
    if (launches) memcpy(launches, c->launches, sizeof c->launches);
    if (!ms) return CC_OK;
    CC_DEVICE(c);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cc_kernel_stats: sync");
    for (auto& t : c->pending) {
        float dt = 0.f;
        if (cudaEventElapsedTime(&dt, t.a, t.b) == cudaSuccess) c->ms[t.kind] += dt;
        c->spare.push_back(t.a);
        c->spare.push_back(t.b);
    }
    c->pending.clear();
    memcpy(ms, c->ms, sizeof c->ms);
    memset(c->ms, 0, sizeof c->ms);
    return CC_OK;
}

int64_t cc_num_vertices(const cc_ctx* c) { return c ? c->n : 0; }

cc_status cc_schedule_stats(cc_ctx* c, int64_t* nonloop_edges, int32_t* rounds) {
    CC_CHECK_CTX(c);
    {
        CC_DEVICE(c);
        cc_status st = refresh_schedule_stats(c);
        if (st != CC_OK) return st;
    }
    if (nonloop_edges) *nonloop_edges = c->last_nonloop;
    if (rounds) *rounds = c->last_rounds;
    return CC_OK;
}

cc_status cc_copy_nonloop(cc_ctx* c, int32_t* out, int64_t cap, int64_t* count) {
    CC_CHECK_CTX(c);
    {
        CC_DEVICE(c);
        cc_status st = refresh_schedule_stats(c);
        if (st != CC_OK) return st;
    }
    if (count) *count = c->last_nonloop;
    const int64_t m = c->last_nonloop < cap ? c->last_nonloop : cap;
    if (m <= 0) return CC_OK;
    if (!out) return fail(CC_ERR_ARG, "cc_copy_nonloop: out is null");
    CC_DEVICE(c);
    cudaError_t e = cudaMemcpyAsync(out, c->a2, sizeof(int) * 2 * (size_t)m, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cc_copy_nonloop");
    return CC_OK;
}

cc_status cc_bulk_find(cc_ctx* c, const int32_t* S, int64_t k, int32_t* res) {
    CC_CHECK_CTX(c);
    if (k < 0 || k > INT32_MAX) return fail(CC_ERR_ARG, "cc_bulk_find: k out of range");
    if (k == 0) return CC_OK;
    if (!S || !res) return fail(CC_ERR_ARG, "cc_bulk_find: null array");
    if (reinterpret_cast<uintptr_t>(S) % 4 || reinterpret_cast<uintptr_t>(res) % 4)
        return fail(CC_ERR_ARG, "cc_bulk_find: arrays must be 4-byte aligned");
    CC_DEVICE(c);
    const uint64_t before = c->bf.launches;
    cudaError_t e = cc::bulk_find(c->bf, c->parent, (int)c->n, S, k, res, c->ds, c->stream);
    c->launches[CC_K_QUERY] += c->bf.launches - before;
    if (e != cudaSuccess) return cuda_fail(e, "cc_bulk_find");
    return CC_OK;
}

cc_status cc_bulk_find_stats(cc_ctx* c, int64_t* traversed, int32_t* levels_up, int32_t* levels_down) {
    CC_CHECK_CTX(c);
    if (traversed) *traversed = c->bf.traversed;
    if (levels_up) *levels_up = c->bf.levels_up;
    if (levels_down) *levels_down = c->bf.levels_down;
    return CC_OK;
}

cc_status cc_load_forest(cc_ctx* c, const int32_t* parent) {
    CC_CHECK_CTX(c);
    if (!parent || reinterpret_cast<uintptr_t>(parent) % 4) return fail(CC_ERR_ARG, "cc_load_forest: null or misaligned");
    if (c->G > 1 || by_size(c)) return fail(CC_ERR_UNSUPPORTED, "cc_load_forest needs the default link rule on a plain handle");
    CC_DEVICE(c);
    cudaError_t e = cudaMemsetAsync(&c->ds->labels_bad, 0, sizeof(unsigned), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(&c->ds->roots, 0, sizeof(unsigned long long), c->stream);
    if (e == cudaSuccess) e = cc::launch_validate_forest(parent, c->n, c->ds, 256, c->stream);
    cc::DevState h;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, c->ds, sizeof h, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cc_load_forest: validate");
    c->launches[CC_K_LOAD]++;
    if (h.labels_bad) return fail(CC_ERR_LABELS, "cc_load_forest: need 0 <= parent[v] <= v");
    unsigned long long unions = (unsigned long long)c->n - h.roots;
    e = cudaMemcpyAsync(c->parent, parent, sizeof(int) * (size_t)c->n, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&c->ds->unions, &unions, sizeof unions, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = big_invalidate(c);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cc_load_forest: copy");
    c->flat = false;
    c->fresh = false;
    c->update_calls = 0;
    return CC_OK;
}

cc_status cc_forest_depth(cc_ctx* c, int32_t* max_depth, double* mean_depth) {
    CC_CHECK_CTX(c);
    if (!max_depth) return fail(CC_ERR_ARG, "cc_forest_depth: max_depth is null");
    CC_DEVICE(c);
    cudaError_t e = cudaMemsetAsync(&c->ds->max_depth, 0, sizeof(unsigned), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(&c->ds->sum_depth, 0, sizeof(unsigned long long), c->stream);
    if (e == cudaSuccess) e = cc::launch_depth(c->parent, c->n, &c->ds->max_depth, &c->ds->sum_depth, c->ds, c->stream);
    cc::DevState h;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, c->ds, sizeof h, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cc_forest_depth");
    *max_depth = (int32_t)h.max_depth;
    if (mean_depth) *mean_depth = (double)h.sum_depth / (double)c->n;
    return CC_OK;
}

cc_status cc_big_filter_stats(cc_ctx* c, int32_t* root, int64_t* members) {
    CC_CHECK_CTX(c);
    if (!root || !members) return fail(CC_ERR_ARG, "cc_big_filter_stats: null output");
    CC_DEVICE(c);
    cc::DevState h;
    cudaError_t e = cudaMemcpyAsync(&h, c->ds, sizeof h, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess && h.big_root >= 0 && c->big) {  // count the marks
        e = cudaMemsetAsync(&c->ds->big_members, 0, sizeof(unsigned long long), c->stream);
        if (e == cudaSuccess) e = cc::launch_big_count(c->big, (c->n + 31) / 32, c->ds, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h, c->ds, sizeof h, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "cc_big_filter_stats");
    *root = h.big_root;
    *members = h.big_root >= 0 ? (int64_t)h.big_members : 0;
    return CC_OK;
}

cc_status cc_device_can_read(const void* p, int32_t* ok) {
    if (!ok) return fail(CC_ERR_ARG, "cc_device_can_read: ok is null");
    *ok = 0;
    if (!p) return CC_OK;
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return CC_OK;
    }
    if (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged) *ok = 1;
    else if (attr.type == cudaMemoryTypeHost && attr.devicePointer == p) *ok = 1;
    return CC_OK;
}

}  // extern "C"
