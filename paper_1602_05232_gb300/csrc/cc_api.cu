// The C-ABI of include/cc.h: argument checks, handle state, error reporting,
// per-kernel launch counters and CUDA-event profiling around the launchers.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
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

const int64_t kDefaults[CC_OPT__COUNT] = {256, 2, 1, CC_COMPRESS_ALL, 0, 0};

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
    return cc::Launch{(int)c->opt[CC_OPT_BLOCK], (int)c->opt[CC_OPT_EDGES_PER_THREAD]};
}

cc_status check_pairs(const int32_t* p, int64_t k, const char* name) {
    if (k < 0 || k > INT32_MAX) return fail(CC_ERR_ARG, "%s: k = %lld out of [0, 2^31-1]", name, (long long)k);
    if (k > 0 && !p) return fail(CC_ERR_ARG, "%s: null array with k > 0", name);
    if (k > 0 && reinterpret_cast<uintptr_t>(p) % 4 != 0) return fail(CC_ERR_ARG, "%s: array not 4-byte aligned", name);
    return CC_OK;
}

cc_status do_compress(cc_ctx* c, int scope, const int32_t* edges, int64_t k) {
    if (scope == CC_COMPRESS_ALL) {
        cc_status s = run(c, CC_K_COMPRESS_ALL, "compress(all)", [&] {
            return cc::launch_compress_all(c->parent, c->n, nullptr, c->ds, (int)c->opt[CC_OPT_BLOCK], c->stream);
        });
        if (s == CC_OK) c->flat = true;
        return s;
    }
    if (k == 0) return CC_OK;
    return run(c, CC_K_COMPRESS_TOUCHED, "compress(touched)", [&] {
        return cc::launch_compress_touched(c->parent, (int)c->n, edges, k, c->ds, cfg_of(c), c->stream);
    });
}

}  // namespace

namespace cc {
// Lets the other translation units leave a message for cc_last_error_string().
cc_status record_error(cc_status s, const char* msg) { return fail(s, "%s", msg); }
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
    if (e != cudaSuccess) return cuda_fail(e, "cc_reset");
    cc_status s = run(c, CC_K_RESET, "reset", [&] {
        return cc::launch_reset(c->parent, c->n, (int)c->opt[CC_OPT_BLOCK], c->stream);
    });
    if (s == CC_OK) {
        c->flat = true;
        c->update_calls = 0;
    }
    return s;
}

cc_status cc_bulk_update(cc_ctx* c, const int32_t* edges, int64_t k) {
    CC_CHECK_CTX(c);
    cc_status s = check_pairs(edges, k, "cc_bulk_update");
    if (s != CC_OK) return s;
    if (k == 0) return CC_OK;
    CC_DEVICE(c);
    s = run(c, CC_K_UPDATE, "bulk_update", [&] {
        return cc::launch_update(c->parent, (int)c->n, edges, k, c->ds, cfg_of(c), c->stream);
    });
    if (s != CC_OK) return s;
    c->flat = false;
    c->update_calls++;
    const int64_t every = c->opt[CC_OPT_COMPRESS_EVERY];
    if (every > 0 && c->update_calls % (uint64_t)every == 0)
        return do_compress(c, (int)c->opt[CC_OPT_COMPRESS_SCOPE], edges, k);
    return CC_OK;
}

cc_status cc_bulk_query(cc_ctx* c, const int32_t* pairs, int64_t k, uint8_t* out) {
    CC_CHECK_CTX(c);
    cc_status s = check_pairs(pairs, k, "cc_bulk_query");
    if (s != CC_OK) return s;
    if (k > 0 && !out) return fail(CC_ERR_ARG, "cc_bulk_query: out is null");
    if (k == 0) return CC_OK;
    CC_DEVICE(c);
    const int mode = c->flat ? 2 : (c->opt[CC_OPT_QUERY_HALVING] ? 1 : 0);
    s = run(c, CC_K_QUERY, "bulk_query", [&] {
        return cc::launch_query(c->parent, (int)c->n, pairs, k, out, c->ds, mode, cfg_of(c), c->stream);
    });
    if (s == CC_OK && mode == 1) c->flat = false;
    return s;
}

cc_status cc_compress(cc_ctx* c, int32_t scope, const int32_t* edges, int64_t k) {
    CC_CHECK_CTX(c);
    if (scope != CC_COMPRESS_ALL && scope != CC_COMPRESS_TOUCHED)
        return fail(CC_ERR_ARG, "cc_compress: unknown scope %d", scope);
    if (scope == CC_COMPRESS_TOUCHED) {
        cc_status s = check_pairs(edges, k, "cc_compress");
        if (s != CC_OK) return s;
    }
    CC_DEVICE(c);
    return do_compress(c, scope, edges, k);
}

cc_status cc_labels(cc_ctx* c, int32_t* out) {
    CC_CHECK_CTX(c);
    if (!out) return fail(CC_ERR_ARG, "cc_labels: out is null");
    if (reinterpret_cast<uintptr_t>(out) % 4 != 0) return fail(CC_ERR_ARG, "cc_labels: out not 4-byte aligned");
    CC_DEVICE(c);
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
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cc_load_labels: copy");
    c->flat = true;
    c->update_calls = 0;
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
        case CC_OPT_PROFILE:
            if (value != 0 && value != 1) return fail(CC_ERR_ARG, "option %d takes 0 or 1", option);
            break;
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

}  // extern "C"
