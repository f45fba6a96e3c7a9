// cc_components_static: connected-component labels of one edge list, using
// no memory that has to be allocated.
//
// Callers that cannot call cudaMalloc -- code running while its stream is
// captured into a CUDA graph, real-time loops that must not take the implicit
// device synchronisation and unbounded latency of an allocation, and plugins
// whose host framework owns all device memory and offers them no allocator --
// can still label a graph: the working forest and the status word live in the
// file-scope device array below, which is part of the loaded module, not of
// any allocation. The caller passes only its inputs (the edges) and outputs
// (the labels, and optionally a status word).
//
// The array holds CC_STATIC_MAX_VERTICES vertices (16 MiB + 256 B) and every
// GPU that loads this library keeps it until the process exits. All calls
// share it: each call re-initialises what it uses before its kernels read it,
// and two calls whose work overlaps on the GPU (different streams, no
// ordering between them) race on it and give wrong labels.
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
int32_t* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device. In host code the
// array's name is only a host-side stand-in; the kernels need this address.
// Looked up once per device (the first call on a device does it).
cudaError_t scratch_address(int device, int32_t** out) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[device] = static_cast<int32_t*>(p);
    }
    *out = g_scratch_ptr[device];
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
