// cc_components_static: connected-component labels of one edge list, using
// no memory that has to be allocated.
//
// Some callers cannot call cudaMalloc: real-time loops that must not take the
// implicit device synchronisation and unbounded latency of an allocation, and
// plugins whose host framework owns all device memory and offers them no
// allocator. They can still label a graph: the working forest and the status
// word live in the file-scope device array below, which is part of the loaded
// module, not of any allocation. The caller passes only its inputs (the
// edges) and outputs (the labels, and optionally a status word).
//
// The array holds CC_STATIC_MAX_VERTICES vertices (16 MiB + 256 B) and every
// GPU that loads this library keeps it until the process exits. All calls
// share it: each call re-initialises what it uses before its kernels read it,
// and two calls whose work overlaps on the GPU (different streams, no
// ordering between them) race on it and give wrong labels.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "cc.h"
#include "cc_internal.cuh"

namespace {

constexpr int kHeaderInts = 64;  // 256 bytes: the DevState, then the forest
static_assert(sizeof(cc::DevState) <= kHeaderInts * sizeof(int32_t), "header too small");

// The scratch: [0, 256 B) DevState, then parent[0 .. CC_STATIC_MAX_VERTICES).
static __device__ __align__(256) int32_t g_static_scratch[kHeaderInts + CC_STATIC_MAX_VERTICES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;

// The address is cached per device together with the id of the context it
// was looked up in: if that context is destroyed (cudaDeviceReset) and a new
// one made, the module is loaded again, possibly elsewhere, and the lookup
// must be repeated. Context ids are never reused within a process.
struct ScratchAddr {
    unsigned long long ctx_id = 0;
    int32_t* ptr = nullptr;
};
ScratchAddr g_scratch[kMaxDevices];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Id of the calling thread's current context, or 0 if there is none or the
// driver cannot say. The two driver calls are reached through the runtime's
// entry-point query, so libcc does not link the driver library itself.
unsigned long long current_context_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
    });
    if (!get_current || !get_id) return 0;
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of the scratch on the current device. In host code the
// array's name is only a host-side stand-in; the kernels need this address.
// Looked up on the first call on a device (and again only if that device's
// context has been replaced since); make that first call before any stream
// capture.
cudaError_t scratch_address(int device, int32_t** out) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    ScratchAddr& a = g_scratch[device];
    const unsigned long long id = current_context_id();
    if (!a.ptr || id == 0 || id != a.ctx_id) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        a.ptr = static_cast<int32_t*>(p);
        a.ctx_id = current_context_id();  // the lookup made a context current if none was
    }
    *out = a.ptr;
    return cudaSuccess;
}

}  // namespace

extern "C" cc_status cc_components_static(const int32_t* edges, int64_t k, int64_t n,
                                          int32_t* labels, uint32_t* status,
                                          cc_stream_t stream) {
    if (n < 1 || n > CC_STATIC_MAX_VERTICES)
        return cc::record_error(CC_ERR_ARG, "cc_components_static: n must be in [1, "
                                "CC_STATIC_MAX_VERTICES = 4194304]; use cc_create for larger graphs");
    if (k < 0 || k > INT32_MAX || (k > 0 && !edges) || !labels)
        return cc::record_error(CC_ERR_ARG, "cc_components_static: bad k or null array");
    if (reinterpret_cast<uintptr_t>(edges) % 4 || reinterpret_cast<uintptr_t>(labels) % 4)
        return cc::record_error(CC_ERR_ARG, "cc_components_static: arrays must be 4-byte aligned");
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices)
        return cc::record_error(CC_ERR_CUDA, "cc_components_static: no usable current device");
    int32_t* scratch = nullptr;
    if (scratch_address(device, &scratch) != cudaSuccess)
        return cc::record_error(CC_ERR_CUDA, "cc_components_static: cudaGetSymbolAddress failed");

    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cc::DevState* ds = reinterpret_cast<cc::DevState*>(scratch);
    int* parent = scratch + kHeaderInts;
    const cc::Launch cfg{256, 2};
    // Start from n singletons with a clear status word, whatever the last call left.
    cudaError_t e = cudaMemsetAsync(ds, 0, sizeof(cc::DevState), s);
    if (e == cudaSuccess) e = cc::launch_reset(parent, n, 256, s);
    if (e == cudaSuccess) e = cc::launch_update(parent, (int)n, edges, k, ds, cfg, s);
    if (e == cudaSuccess) e = cc::launch_compress_all(parent, n, labels, ds, 256, s);
    if (e == cudaSuccess && status)
        e = cudaMemcpyAsync(status, &ds->status, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess)
        return cc::record_error(CC_ERR_CUDA, "cc_components_static: a launch or copy failed");
    return CC_OK;
}
