// Kernels of the plain (one launch per bulk operation) path and their launchers.
#include <cstdint>

#include "cc_device.cuh"
#include "cc_internal.cuh"

namespace cc {

int pair_vec(const void* p) {
    uintptr_t a = reinterpret_cast<uintptr_t>(p);
    return (a % 16 == 0) ? 2 : (a % 8 == 0) ? 1 : 0;
}

static inline unsigned blocks_for(int64_t work, int64_t per_block) {
    return (unsigned)((work + per_block - 1) / per_block);
}

// Launch with per-launch attributes that apply to this kernel only (the
// stream is left as it is): an optional L2 access-policy window, and
// programmatic dependent launch, which lets the kernel's CTAs become resident
// while the kernel before it on the stream drains; the kernel then waits for
// that one in pdl_wait() (griddepcontrol.wait).
template <typename... Params, typename... Args>
static void launch_windowed(void (*kernel)(Params...), unsigned grid, int block, cudaStream_t s,
                            const cudaAccessPolicyWindow* window, bool pdl, Args... args) {
    if (!window && !pdl) {
        kernel<<<grid, block, 0, s>>>(args...);
        return;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    unsigned na = 0;
    if (window) {
        attr[na].id = cudaLaunchAttributeAccessPolicyWindow;
        attr[na].val.accessPolicyWindow = *window;
        na++;
    }
    if (pdl) {
        attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[na].val.programmaticStreamSerializationAllowed = 1;
        na++;
    }
    cfg.attrs = attr;
    cfg.numAttrs = na;
    cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Programmatic dependent launch, device side. pdl_trigger: the kernel launched
// after this one on the stream may start placing its CTAs (it still waits in
// pdl_wait before touching results). pdl_wait: returns once the kernel before
// this one has completed and its writes are visible; immediately when this
// kernel was not launched as a dependent.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

// A persistent grid for KERNEL at `block` threads (no dynamic shared memory):
// resident CTAs per SM x SMs of the current device. Cached per host thread,
// device and block size, so neither threads nor different GPUs share an entry.
template <auto KERNEL>
static int resident_grid(int block) {
    thread_local int cache[16][33] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    int* slot = (dev >= 0 && dev < 16 && block > 0 && block <= 1024) ? &cache[dev][block / 32] : nullptr;
    if (slot && *slot) return *slot;
    int per_sm = 0, sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, KERNEL, block, 0);
    const int c = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
    if (slot) *slot = c;
    return c;
}

// ------------------------------------------------------------------ reset

// parent[v] = v: n singletons, the empty graph G_0.
__global__ void k_reset(int* __restrict__ parent, int64_t n) {
    int64_t v0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (v0 + 4 <= n) {
        int x = (int)v0;
        reinterpret_cast<int4*>(parent)[v0 / 4] = make_int4(x, x + 1, x + 2, x + 3);
    } else {
        for (int64_t v = v0; v < n; v++) parent[v] = (int)v;
    }
}

cudaError_t launch_reset(int* parent, int64_t n, int block, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_reset<<<blocks_for(n, 4LL * block), block, 0, s>>>(parent, n);
    return cudaGetLastError();
}

// ------------------------------------------------------------ Bulk-Update

// One fused pass of Algorithm 2 over E edges: the first parent reads of both
// endpoints of all E edges are issued together; equal parents mean the edge
// joins a tree to itself and is dropped at once (the common case once trees
// are flat, and the self-loop filter of Algorithm 2). The other endpoints are
// walked to their roots -- VARIANT 0 one edge at a time with path halving,
// VARIANTs 1 and 2 all 2E walks in lockstep with path splitting -- and the
// roots are hooked. Returns the number of links made.
template <int E, int VARIANT, bool WARP = false>
__device__ __forceinline__ int update_edges(int* __restrict__ parent, int n,
                                            const int (&u)[E], const int (&v)[E], int64_t e0,
                                            int64_t k, DevState* __restrict__ ds, int minhook,
                                            const unsigned* bits) {
    bool ok[E];
    bool bad = false;
    int made = 0;
#pragma unroll
    for (int i = 0; i < E; i++) {
        ok[i] = e0 + i < k;
        if (ok[i] && !(in_range(u[i], n) && in_range(v[i], n))) {
            ok[i] = false;
            bad = true;
        }
    }
    if (bad) flag(ds, ST_RANGE);
    if (bits) {  // both endpoints in the marked tree: already joined
#pragma unroll
        for (int i = 0; i < E; i++)
            if (ok[i] && big_member(bits, u[i]) && big_member(bits, v[i])) ok[i] = false;
    }
    if constexpr (VARIANT == 0) {
        int pu[E], pv[E];
#pragma unroll
        for (int i = 0; i < E; i++) {
            pu[i] = ok[i] ? parent[u[i]] : 0;
            pv[i] = ok[i] ? parent[v[i]] : 0;
        }
#pragma unroll
        for (int i = 0; i < E; i++) {
            if (!ok[i] || pu[i] == pv[i]) continue;
            int ru = pu[i] == u[i] ? u[i] : find_from(parent, u[i], pu[i], ds);
            int rv = pv[i] == v[i] ? v[i] : find_from(parent, v[i], pv[i], ds);
            made += hook_as(parent, ru, rv, ds, minhook);
        }
        return made;
    } else {
        // lockstep: chain c = 2i (u side) and 2i+1 (v side); finished when p >= x
        int x[2 * E], p[2 * E];
#pragma unroll
        for (int i = 0; i < E; i++) {
            x[2 * i] = ok[i] ? u[i] : 0;
            x[2 * i + 1] = ok[i] ? v[i] : 0;
        }
#pragma unroll
        for (int c = 0; c < 2 * E; c++) p[c] = ok[c / 2] ? parent[x[c]] : x[c];
        bool live[E];
#pragma unroll
        for (int i = 0; i < E; i++) {
            live[i] = ok[i] && p[2 * i] != p[2 * i + 1];
            if (!live[i]) {  // nothing to walk for this edge
                p[2 * i] = x[2 * i];
                p[2 * i + 1] = x[2 * i + 1];
            }
        }
        walk_split<2 * E>(parent, x, p, ds);
        if constexpr (WARP) {  // every lane of the warp is here (see the kernels)
            int a[E], b[E];
#pragma unroll
            for (int i = 0; i < E; i++) {
                a[i] = x[2 * i];
                b[i] = x[2 * i + 1];
            }
            made = hook_warp<E>(parent, live, a, b, ds, minhook);
        } else {
#pragma unroll
            for (int i = 0; i < E; i++)
                if (live[i]) made += hook_as(parent, x[2 * i], x[2 * i + 1], ds, minhook);
        }
        return made;
    }
}

// early: the first edges are read before the wait for the previous kernel
// (programmatic dependent launch; see launch_windowed), else after it.
// warphook (lockstep variants only): the hooks of a warp are grouped by
// target (hook_warp), so every lane of a warp that has any edge left goes
// through each round of the loop, with no edges of its own if it has none.
template <int E, int VARIANT, bool WARP>
__global__ void __launch_bounds__(1024)
k_update(int* __restrict__ parent, int n, const int* __restrict__ edges, int64_t k, int vec,
         DevState* __restrict__ ds, int early, int minhook, BigArgs fb) {
    pdl_trigger();
    if (!early) pdl_wait();
    if (fb.alt && big_active(fb.big, ds)) {  // the filter is on: the edges were not ordered
        edges = fb.alt;
        vec = pair_vec_dev(fb.alt);
    }
    int made = 0;
    int64_t e0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * E;
    if (VARIANT < 2) {
        // with warphook, every lane goes in if any lane of its warp has edges
        bool warp_busy = false;
        if constexpr (WARP) warp_busy = __any_sync(0xffffffffu, e0 < k);
        if (e0 < k || warp_busy) {
            int u[E], v[E];
            load_pairs<E>(edges, e0, k, vec, u, v);
            if (early) pdl_wait();
            made = update_edges<E, VARIANT, WARP>(parent, n, u, v, e0, k, ds, minhook, big_active(fb.big, ds));
        }
    } else {
        // persistent grid: loop over chunks, loading the next chunk's edges
        // before walking the current one so their latency overlaps
        const int64_t stride = (int64_t)gridDim.x * blockDim.x * E;
        int u[E], v[E];
        if (e0 < k) load_pairs<E>(edges, e0, k, vec, u, v);
        if (early) pdl_wait();
        const unsigned* bits = big_active(fb.big, ds);
        while (WARP ? __any_sync(0xffffffffu, e0 < k) : e0 < k) {
            const int64_t nx = e0 + stride;
            int nu[E] = {}, nv[E] = {};
            if (nx < k) load_pairs<E>(edges, nx, k, vec, nu, nv);
            made += update_edges<E, 1, WARP>(parent, n, u, v, e0, k, ds, minhook, bits);
#pragma unroll
            for (int i = 0; i < E; i++) {
                u[i] = nu[i];
                v[i] = nv[i];
            }
            e0 = nx;
        }
    }
    made = __reduce_add_sync(0xffffffffu, made);
    if ((threadIdx.x & 31) == 0 && made) atomicAdd(&ds->unions, (unsigned long long)made);
}

// --- VARIANT 3: the persistent grid with a two-stage prefetch -------------

// Bit i set when this thread's edge i at e0 exists and has both endpoints in
// range, and (with a largest-component bitmap) they are not both marked;
// range errors are flagged here, once per chunk.
template <int E>
__device__ __forceinline__ unsigned edge_mask(int n, const int (&u)[E], const int (&v)[E], int64_t e0,
                                              int64_t k, DevState* __restrict__ ds, const unsigned* bits) {
    unsigned m = 0;
    bool bad = false;
#pragma unroll
    for (int i = 0; i < E; i++) {
        if (e0 + i >= k) continue;
        if (in_range(u[i], n) && in_range(v[i], n)) m |= 1u << i;
        else bad = true;
    }
    if (bad) flag(ds, ST_RANGE);
    if (bits) {
#pragma unroll
        for (int i = 0; i < E; i++)
            if (((m >> i) & 1u) && big_member(bits, u[i]) && big_member(bits, v[i])) m &= ~(1u << i);
    }
    return m;
}

// The first parent reads of the edges in m, all issued together (an edge not
// in m reads nothing and keeps its endpoints as their own parents).
template <int E>
__device__ __forceinline__ void gather_parents(const int* parent, unsigned m, const int (&u)[E],
                                               const int (&v)[E], int (&pu)[E], int (&pv)[E]) {
#pragma unroll
    for (int i = 0; i < E; i++) {
        const bool on = (m >> i) & 1u;
        pu[i] = on ? parent[u[i]] : u[i];
        pv[i] = on ? parent[v[i]] : v[i];
    }
}

// The rest of the fused pass for edges whose first parents pu, pv were read
// earlier, possibly before other links of this minibatch: a parent read then
// is still an ancestor now (links only put roots under roots, and splitting
// only repoints a node at an ancestor), so walking on from it reaches the
// current root, and equal values still prove the endpoints joined.
template <int E, bool WARP = false>
__device__ __forceinline__ int walk_and_hook(int* parent, unsigned m, const int (&u)[E], const int (&v)[E],
                                             const int (&pu)[E], const int (&pv)[E], DevState* ds,
                                             int minhook) {
    int x[2 * E], p[2 * E];
    bool live[E];
#pragma unroll
    for (int i = 0; i < E; i++) {
        live[i] = ((m >> i) & 1u) && pu[i] != pv[i];
        x[2 * i] = u[i];
        x[2 * i + 1] = v[i];
        p[2 * i] = live[i] ? pu[i] : u[i];
        p[2 * i + 1] = live[i] ? pv[i] : v[i];
    }
    walk_split<2 * E>(parent, x, p, ds);
    int made = 0;
    if constexpr (WARP) {  // every lane of the warp is here (see the kernels)
        int a[E], b[E];
#pragma unroll
        for (int i = 0; i < E; i++) {
            a[i] = x[2 * i];
            b[i] = x[2 * i + 1];
        }
        made = hook_warp<E>(parent, live, a, b, ds, minhook);
    } else {
#pragma unroll
        for (int i = 0; i < E; i++)
            if (live[i]) made += hook_as(parent, x[2 * i], x[2 * i + 1], ds, minhook);
    }
    return made;
}

// Persistent grid over chunks of E edges per thread. While the walks and
// hooks of chunk c run, the first parent reads of chunk c+1 and the edge
// loads of chunk c+2 are already in flight, so a warp waiting on its deepest
// walk still has the next chunk's gathers outstanding. early: as for k_update.
template <int E, bool WARP>
__global__ void __launch_bounds__(1024)
k_update_deep(int* __restrict__ parent, int n, const int* __restrict__ edges, int64_t k, int vec,
              DevState* __restrict__ ds, int early, int minhook, BigArgs fb) {
    pdl_trigger();
    if (!early) pdl_wait();
    if (fb.alt && big_active(fb.big, ds)) {  // as in k_update
        edges = fb.alt;
        vec = pair_vec_dev(fb.alt);
    }
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * E;
    int64_t e0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * E;
    int made = 0;
    int u0[E] = {}, v0[E] = {}, u1[E] = {}, v1[E] = {};
    if (e0 < k) load_pairs<E>(edges, e0, k, vec, u0, v0);
    if (e0 + stride < k) load_pairs<E>(edges, e0 + stride, k, vec, u1, v1);
    if (early) pdl_wait();
    const unsigned* bits = big_active(fb.big, ds);
    unsigned m0 = e0 < k ? edge_mask<E>(n, u0, v0, e0, k, ds, bits) : 0u;
    int pu0[E], pv0[E];
    gather_parents<E>(parent, m0, u0, v0, pu0, pv0);
    while (WARP ? __any_sync(0xffffffffu, e0 < k) : e0 < k) {
        const int64_t e1 = e0 + stride, e2 = e1 + stride;
        const unsigned m1 = e1 < k ? edge_mask<E>(n, u1, v1, e1, k, ds, bits) : 0u;
        int pu1[E], pv1[E];
        gather_parents<E>(parent, m1, u1, v1, pu1, pv1);
        int u2[E] = {}, v2[E] = {};
        if (e2 < k) load_pairs<E>(edges, e2, k, vec, u2, v2);
        made += walk_and_hook<E, WARP>(parent, m0, u0, v0, pu0, pv0, ds, minhook);
#pragma unroll
        for (int i = 0; i < E; i++) {
            u0[i] = u1[i]; v0[i] = v1[i]; pu0[i] = pu1[i]; pv0[i] = pv1[i];
            u1[i] = u2[i]; v1[i] = v2[i];
        }
        m0 = m1;
        e0 = e1;
    }
    made = __reduce_add_sync(0xffffffffu, made);
    if ((threadIdx.x & 31) == 0 && made) atomicAdd(&ds->unions, (unsigned long long)made);
}

template <int E>
static void update_deep_inst(const int* edges, int64_t k, int vec, int* parent, int n, DevState* ds,
                             int block, const cudaAccessPolicyWindow* window, int pdl, int minhook,
                             int warphook, BigArgs fb, cudaStream_t s) {
    int64_t g = (k + (int64_t)E * block - 1) / ((int64_t)E * block);
    if (warphook) {
        const int64_t cap = resident_grid<k_update_deep<E, true>>(block);
        if (g > cap) g = cap;
        launch_windowed(k_update_deep<E, true>, (unsigned)g, block, s, window, pdl != 0, parent, n, edges, k,
                        vec, ds, (int)(pdl == 2), minhook, fb);
        return;
    }
    const int64_t cap = resident_grid<k_update_deep<E, false>>(block);
    if (g > cap) g = cap;
    launch_windowed(k_update_deep<E, false>, (unsigned)g, block, s, window, pdl != 0, parent, n, edges, k, vec,
                    ds, (int)(pdl == 2), minhook, fb);
}

// --- VARIANT 5: per-CTA list of open edges ---------------------------------
//
// A persistent grid over tiles of blockDim * E edges. Every thread reads its
// E edges' first parents (independent loads, as in the filter pass of
// variant 4); the open edges (parents differ) go to a list in shared memory,
// and then all threads of the CTA walk and hook that list together, two
// listed edges per thread at a time, while the edge loads and first parent
// reads of the CTA's next tile are already in flight. So the walks of the few
// open edges are spread over every thread of the CTA instead of stalling the
// warp that happened to load them. Two barriers per tile; the list's counter
// is double-buffered so that a count is cleared only after every thread has
// read it.
template <int E>
__global__ void __launch_bounds__(1024, 1)  // without the minimum, E = 1 and 2 were held to 32 registers and spilled
k_update_tiles(int* __restrict__ parent, int n, const int* __restrict__ edges, int64_t k, int vec,
               DevState* __restrict__ ds, int early, int minhook, BigArgs fb) {
    extern __shared__ int4 open_list[];  // blockDim.x * E entries: (u, v, parent[u], parent[v])
    __shared__ unsigned n_open[2];
    pdl_trigger();
    if (!early) pdl_wait();
    if (fb.alt && big_active(fb.big, ds)) {  // as in k_update
        edges = fb.alt;
        vec = pair_vec_dev(fb.alt);
    }
    const int64_t T = (int64_t)blockDim.x * E;
    const int64_t tiles = (k + T - 1) / T;
    if (threadIdx.x == 0) n_open[0] = n_open[1] = 0u;
    int made = 0;
    int64_t t = blockIdx.x;
    int u[E] = {}, v[E] = {}, pu[E], pv[E];
    unsigned m = 0;
    int64_t e0 = t * T + (int64_t)threadIdx.x * E;
    if (t < tiles && e0 < k) load_pairs<E>(edges, e0, k, vec, u, v);
    if (early) pdl_wait();
    const unsigned* bits = big_active(fb.big, ds);
    if (t < tiles && e0 < k) m = edge_mask<E>(n, u, v, e0, k, ds, bits);
    gather_parents<E>(parent, m, u, v, pu, pv);
    __syncthreads();  // counters cleared
    const unsigned lane = threadIdx.x & 31u;
    for (int sel = 0; t < tiles; t += gridDim.x, sel ^= 1) {
        // append this thread's open edges (one atomic per warp)
        unsigned open = 0;
#pragma unroll
        for (int i = 0; i < E; i++)
            if (((m >> i) & 1u) && pu[i] != pv[i]) open |= 1u << i;
        const int mine = __popc(open);
        int incl = mine;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= (unsigned)d) incl += y;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        unsigned base = 0;
        if (lane == 31 && total) base = atomicAdd(&n_open[sel], (unsigned)total);
        base = __shfl_sync(0xffffffffu, base, 31) + (unsigned)(incl - mine);
#pragma unroll
        for (int i = 0; i < E; i++)
            if ((open >> i) & 1u) open_list[base++] = make_int4(u[i], v[i], pu[i], pv[i]);
        __syncthreads();  // A: the list of this tile is complete
        const unsigned cnt = n_open[sel];
        if (threadIdx.x == 0) n_open[sel ^ 1] = 0u;  // last read before the previous B
        // the next tile's edges and first parents, in flight during the walks
        const int64_t t1 = t + gridDim.x;
        const int64_t e1 = t1 * T + (int64_t)threadIdx.x * E;
        int nu[E] = {}, nv[E] = {};
        unsigned m1 = 0;
        if (t1 < tiles && e1 < k) {
            load_pairs<E>(edges, e1, k, vec, nu, nv);
            m1 = edge_mask<E>(n, nu, nv, e1, k, ds, bits);
        }
        int npu[E], npv[E];
        gather_parents<E>(parent, m1, nu, nv, npu, npv);
        // walk and hook the list, two entries per thread at a time
        for (unsigned j = 2u * threadIdx.x; j < cnt; j += 2u * blockDim.x) {
            const int4 a = open_list[j];
            const int4 b = j + 1 < cnt ? open_list[j + 1] : a;
            const unsigned on = j + 1 < cnt ? 3u : 1u;
            const int lu[2] = {a.x, b.x}, lv[2] = {a.y, b.y}, lpu[2] = {a.z, b.z}, lpv[2] = {a.w, b.w};
            made += walk_and_hook<2>(parent, on, lu, lv, lpu, lpv, ds, minhook);
        }
        __syncthreads();  // B: the list has been walked; it may be refilled
#pragma unroll
        for (int i = 0; i < E; i++) {
            u[i] = nu[i]; v[i] = nv[i]; pu[i] = npu[i]; pv[i] = npv[i];
        }
        m = m1;
    }
    made = __reduce_add_sync(0xffffffffu, made);
    if ((threadIdx.x & 31) == 0 && made) atomicAdd(&ds->unions, (unsigned long long)made);
}

template <int E>
static void update_tiles_inst(const int* edges, int64_t k, int vec, int* parent, int n, DevState* ds, int block,
                              const cudaAccessPolicyWindow* window, int pdl, int minhook, BigArgs fb,
                              cudaStream_t s) {
    const size_t smem = sizeof(int4) * (size_t)block * E;
    if (smem > 48 * 1024)  // the largest list (1024 threads x 4 edges) needs 64 KiB
        cudaFuncSetAttribute(k_update_tiles<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0, sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_update_tiles<E>, block, smem);
    int64_t g = (k + (int64_t)E * block - 1) / ((int64_t)E * block);
    const int64_t cap = (int64_t)(per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
    if (g > cap) g = cap;
    if (!window && !pdl) {
        k_update_tiles<E><<<(unsigned)g, block, smem, s>>>(parent, n, edges, k, vec, ds, 0, minhook, fb);
        return;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)g);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    unsigned na = 0;
    if (window) {
        attr[na].id = cudaLaunchAttributeAccessPolicyWindow;
        attr[na].val.accessPolicyWindow = *window;
        na++;
    }
    if (pdl) {
        attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[na].val.programmaticStreamSerializationAllowed = 1;
        na++;
    }
    cfg.attrs = attr;
    cfg.numAttrs = na;
    cudaLaunchKernelEx(&cfg, k_update_tiles<E>, parent, n, edges, k, vec, ds, (int)(pdl == 2), minhook, fb);
}

// --- VARIANT 4: filter pass + live-edge pass ------------------------------
//
// Once the forest is shallow, almost every edge of a minibatch already has
// parent[u] == parent[v] (its endpoints were joined before), and only a few
// percent need walks and a hook. Pass 1 streams all edges and does only those
// first parent reads -- every warp's loads are independent, so the pass runs
// at the rate of the gathers -- and appends each edge that is still open as
// (u, v, parent[u], parent[v]) to a compact list. Pass 2 walks and hooks only
// the listed edges, from the parents pass 1 read (still ancestors; see
// walk_and_hook). The two list counters alternate between minibatches: pass 1
// of minibatch i appends through count[sel] and zeroes count[sel ^ 1] for
// minibatch i + 1, after the wait that orders it behind everything before it.

template <int E>
__global__ void __launch_bounds__(1024)
k_update_filter(const int* __restrict__ parent, int n, const int* __restrict__ edges, int64_t k, int vec,
                int4* __restrict__ live, unsigned* __restrict__ count, int sel, DevState* __restrict__ ds,
                int early, BigArgs fb) {
    pdl_trigger();
    if (!early) pdl_wait();
    if (fb.alt && big_active(fb.big, ds)) {  // as in k_update
        edges = fb.alt;
        vec = pair_vec_dev(fb.alt);
    }
    const int64_t e0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * E;
    int u[E] = {}, v[E] = {};
    if (e0 < k) load_pairs<E>(edges, e0, k, vec, u, v);
    if (early) pdl_wait();
    if (blockIdx.x == 0 && threadIdx.x == 0) count[sel ^ 1] = 0u;
    const unsigned m = e0 < k ? edge_mask<E>(n, u, v, e0, k, ds, big_active(fb.big, ds)) : 0u;
    int pu[E], pv[E];
    gather_parents<E>(parent, m, u, v, pu, pv);
    unsigned open = 0;
#pragma unroll
    for (int i = 0; i < E; i++)
        if (((m >> i) & 1u) && pu[i] != pv[i]) open |= 1u << i;
    // one atomic per warp: an exclusive scan of the lanes' open counts
    const unsigned lane = threadIdx.x & 31u;
    const int mine = __popc(open);
    int incl = mine;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= (unsigned)d) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (total == 0) return;
    unsigned base = 0;
    if (lane == 31) base = atomicAdd(count + sel, (unsigned)total);
    base = __shfl_sync(0xffffffffu, base, 31) + (unsigned)(incl - mine);
#pragma unroll
    for (int i = 0; i < E; i++)
        if ((open >> i) & 1u) live[base++] = make_int4(u[i], v[i], pu[i], pv[i]);
}

// Pass 2: two listed edges per thread per step, their four walks in lockstep.
template <bool WARP>
__global__ void __launch_bounds__(1024)
k_update_live(int* __restrict__ parent, const int4* __restrict__ live, const unsigned* __restrict__ count,
              int sel, DevState* __restrict__ ds, int minhook) {
    pdl_trigger();
    pdl_wait();
    const int64_t m = count[sel];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * 2;
    int made = 0;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 2;
         WARP ? __any_sync(0xffffffffu, i < m) : i < m; i += stride) {
        const int4 zero = make_int4(0, 0, 0, 0);
        const int4 a = i < m ? live[i] : zero;
        const int4 b = i + 1 < m ? live[i + 1] : a;
        const unsigned on = i + 1 < m ? 3u : i < m ? 1u : 0u;
        const int u[2] = {a.x, b.x}, v[2] = {a.y, b.y}, pu[2] = {a.z, b.z}, pv[2] = {a.w, b.w};
        made += walk_and_hook<2, WARP>(parent, on, u, v, pu, pv, ds, minhook);
    }
    made = __reduce_add_sync(0xffffffffu, made);
    if ((threadIdx.x & 31) == 0 && made) atomicAdd(&ds->unions, (unsigned long long)made);
}

template <int E>
static void update_filter_inst(const int* edges, int64_t k, int vec, const int* parent, int n, int4* live,
                               unsigned* count, int sel, DevState* ds, int block,
                               const cudaAccessPolicyWindow* window, int pdl, BigArgs fb,
                               cudaStream_t s) {
    const int64_t g = (k + (int64_t)E * block - 1) / ((int64_t)E * block);
    launch_windowed(k_update_filter<E>, (unsigned)g, block, s, window, pdl != 0, parent, n, edges, k, vec,
                    live, count, sel, ds, (int)(pdl == 2), fb);
}

cudaError_t launch_update_split(int* parent, int n, const int* edges, int64_t k, DevState* ds, Launch cfg,
                                int4* live, unsigned* count, int sel, cudaStream_t s) {
    if (k <= 0) return cudaSuccess;
    const int vec = pair_vec(edges);
    switch (cfg.ept) {
        case 1: update_filter_inst<1>(edges, k, vec, parent, n, live, count, sel, ds, cfg.block, cfg.window, cfg.pdl, BigArgs{cfg.big, cfg.alt}, s); break;
        case 2: update_filter_inst<2>(edges, k, vec, parent, n, live, count, sel, ds, cfg.block, cfg.window, cfg.pdl, BigArgs{cfg.big, cfg.alt}, s); break;
        case 4: update_filter_inst<4>(edges, k, vec, parent, n, live, count, sel, ds, cfg.block, cfg.window, cfg.pdl, BigArgs{cfg.big, cfg.alt}, s); break;
        default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // pass 2 on a grid of resident CTAs, capped by the most it could have to do
    int64_t g = (k + 2LL * cfg.block - 1) / (2LL * cfg.block);
    if (cfg.warphook) {
        const int64_t cap = resident_grid<k_update_live<true>>(cfg.block);
        if (g > cap) g = cap;
        launch_windowed(k_update_live<true>, (unsigned)g, cfg.block, s, cfg.window, cfg.pdl != 0, parent,
                        (const int4*)live, (const unsigned*)count, sel, ds, cfg.minhook);
    } else {
        const int64_t cap = resident_grid<k_update_live<false>>(cfg.block);
        if (g > cap) g = cap;
        launch_windowed(k_update_live<false>, (unsigned)g, cfg.block, s, cfg.window, cfg.pdl != 0, parent,
                        (const int4*)live, (const unsigned*)count, sel, ds, cfg.minhook);
    }
    return cudaGetLastError();
}


template <int E, int VARIANT, bool WARP>
static void update_inst2(const int* edges, int64_t k, int vec, int* parent, int n, DevState* ds,
                         int block, const cudaAccessPolicyWindow* window, int pdl, int minhook,
                         BigArgs fb, cudaStream_t s) {
    int64_t g = (k + (int64_t)E * block - 1) / ((int64_t)E * block);
    if (VARIANT == 2) {
        const int64_t cap = resident_grid<k_update<E, VARIANT, WARP>>(block);
        if (g > cap) g = cap;
    }
    launch_windowed(k_update<E, VARIANT, WARP>, (unsigned)g, block, s, window, pdl != 0, parent, n, edges, k,
                    vec, ds, (int)(pdl == 2), minhook, fb);
}

// warphook applies to the lockstep variants (1, 2); variant 0 hooks per edge
template <int E, int VARIANT>
static void update_inst(const int* edges, int64_t k, int vec, int* parent, int n, DevState* ds,
                        int block, const cudaAccessPolicyWindow* window, int pdl, int minhook,
                        int warphook, BigArgs fb, cudaStream_t s) {
    if (VARIANT != 0 && warphook)
        update_inst2<E, VARIANT, VARIANT != 0>(edges, k, vec, parent, n, ds, block, window, pdl, minhook, fb, s);
    else
        update_inst2<E, VARIANT, false>(edges, k, vec, parent, n, ds, block, window, pdl, minhook, fb, s);
}

cudaError_t launch_update(int* parent, int n, const int* edges, int64_t k, DevState* ds,
                          Launch cfg, cudaStream_t s) {
    if (k <= 0) return cudaSuccess;
    const int vec = pair_vec(edges);
#define CC_UPD(E, V) update_inst<E, V>(edges, k, vec, parent, n, ds, cfg.block, cfg.window, cfg.pdl, cfg.minhook, cfg.warphook, BigArgs{cfg.big, cfg.alt}, s)
    switch (cfg.variant * 8 + cfg.ept) {
        case 1: CC_UPD(1, 0); break;
        case 2: CC_UPD(2, 0); break;
        case 4: CC_UPD(4, 0); break;
        case 9: CC_UPD(1, 1); break;
        case 10: CC_UPD(2, 1); break;
        case 12: CC_UPD(4, 1); break;
        case 17: CC_UPD(1, 2); break;
        case 18: CC_UPD(2, 2); break;
        case 20: CC_UPD(4, 2); break;
        case 25: update_deep_inst<1>(edges, k, vec, parent, n, ds, cfg.block, cfg.window, cfg.pdl, cfg.minhook, cfg.warphook, BigArgs{cfg.big, cfg.alt}, s); break;
        case 26: update_deep_inst<2>(edges, k, vec, parent, n, ds, cfg.block, cfg.window, cfg.pdl, cfg.minhook, cfg.warphook, BigArgs{cfg.big, cfg.alt}, s); break;
        case 28: update_deep_inst<4>(edges, k, vec, parent, n, ds, cfg.block, cfg.window, cfg.pdl, cfg.minhook, cfg.warphook, BigArgs{cfg.big, cfg.alt}, s); break;
        case 41: update_tiles_inst<1>(edges, k, vec, parent, n, ds, cfg.block, cfg.window, cfg.pdl, cfg.minhook, BigArgs{cfg.big, cfg.alt}, s); break;
        case 42: update_tiles_inst<2>(edges, k, vec, parent, n, ds, cfg.block, cfg.window, cfg.pdl, cfg.minhook, BigArgs{cfg.big, cfg.alt}, s); break;
        case 44: update_tiles_inst<4>(edges, k, vec, parent, n, ds, cfg.block, cfg.window, cfg.pdl, cfg.minhook, BigArgs{cfg.big, cfg.alt}, s); break;
        default: return cudaErrorInvalidValue;
    }
#undef CC_UPD
    return cudaGetLastError();
}

// ------------------------------------------------------------- Bulk-Query

template <int E>
__device__ __forceinline__ void store_answers(uint8_t* __restrict__ out, int64_t e0, int64_t k,
                                              bool ovec, const uint8_t (&a)[E]) {
    if (ovec && e0 + E <= k) {
        if (E == 4) {
            uchar4 w = make_uchar4(a[0], a[E > 1 ? 1 : 0], a[E > 2 ? 2 : 0], a[E > 3 ? 3 : 0]);
            __stcs(reinterpret_cast<uchar4*>(out + e0), w);
            return;
        }
        if (E == 2) {
            uchar2 w = make_uchar2(a[0], a[E > 1 ? 1 : 0]);
            __stcs(reinterpret_cast<uchar2*>(out + e0), w);
            return;
        }
    }
#pragma unroll
    for (int i = 0; i < E; i++)
        if (e0 + i < k) out[e0 + i] = a[i];
}

// One chunk of Algorithm 1: the E pairs (u, v) of this thread, answers in a.
// Returns whether a pair had an id outside [0, n). MODE as for k_query. With
// a largest-component bitmap, a pair whose endpoints are both marked is
// answered 1 from the bitmap alone: it reads no parent and walks nothing
// (its first parents are set equal, which every MODE below answers with 1).
template <int E, int MODE>
__device__ __forceinline__ bool query_chunk(int* __restrict__ parent, int n, int (&u)[E], int (&v)[E],
                                            int64_t e0, int64_t k, uint8_t (&a)[E],
                                            DevState* __restrict__ ds, const unsigned* bits) {
    bool ok[E];
    bool bad = false;
#pragma unroll
    for (int i = 0; i < E; i++) {
        ok[i] = e0 + i < k;
        if (ok[i] && !(in_range(u[i], n) && in_range(v[i], n))) {
            ok[i] = false;
            bad = true;
        }
        if (!ok[i]) { u[i] = 0; v[i] = 0; }
    }
    bool hit[E];
#pragma unroll
    for (int i = 0; i < E; i++) hit[i] = bits && ok[i] && big_member(bits, u[i]) && big_member(bits, v[i]);
    int pu[E], pv[E];
#pragma unroll
    for (int i = 0; i < E; i++) {
        if (hit[i]) {
            pu[i] = pv[i] = u[i];
        } else if (MODE == 1 || MODE == 3) {
            pu[i] = parent[u[i]];
            pv[i] = parent[v[i]];
        } else {
            pu[i] = __ldg(parent + u[i]);
            pv[i] = __ldg(parent + v[i]);
        }
    }
    if (MODE == 2) {
#pragma unroll
        for (int i = 0; i < E; i++) a[i] = (uint8_t)(ok[i] && pu[i] == pv[i]);
    } else if (MODE == 1) {
#pragma unroll
        for (int i = 0; i < E; i++) {
            if (!ok[i]) { a[i] = 0; continue; }
            if (pu[i] == pv[i]) { a[i] = 1; continue; }
            int ru = pu[i] == u[i] ? u[i] : find_from(parent, u[i], pu[i], ds);
            int rv = pv[i] == v[i] ? v[i] : find_from(parent, v[i], pv[i], ds);
            a[i] = (uint8_t)(ru == rv);
        }
    } else if (MODE == 3) {
        // all 2E walks in lockstep with path splitting (they write)
        int x[2 * E], p[2 * E];
#pragma unroll
        for (int i = 0; i < E; i++) {
            const bool live = ok[i] && pu[i] != pv[i];
            x[2 * i] = u[i];     p[2 * i] = live ? pu[i] : u[i];
            x[2 * i + 1] = v[i]; p[2 * i + 1] = live ? pv[i] : v[i];
        }
        walk_split<2 * E>(parent, x, p, ds);
#pragma unroll
        for (int i = 0; i < E; i++)
            a[i] = (uint8_t)(ok[i] && (pu[i] == pv[i] || x[2 * i] == x[2 * i + 1]));
    } else {
        // walk state: x = current node, p = its parent; done when p >= x
        int x[2 * E], p[2 * E];
#pragma unroll
        for (int i = 0; i < E; i++) {
            bool live = ok[i] && pu[i] != pv[i];
            x[2 * i] = u[i];     p[2 * i] = live ? pu[i] : u[i];
            x[2 * i + 1] = v[i]; p[2 * i + 1] = live ? pv[i] : v[i];
        }
        while (true) {
            bool any = false;
#pragma unroll
            for (int c = 0; c < 2 * E; c++) {
                if (p[c] < x[c]) {
                    x[c] = p[c];
                    p[c] = __ldg(parent + x[c]);
                    any = true;
                }
            }
            if (!any) break;
        }
#pragma unroll
        for (int i = 0; i < E; i++) {
            if (p[2 * i] > x[2 * i] || p[2 * i + 1] > x[2 * i + 1]) flag(ds, ST_CORRUPT);
            a[i] = (uint8_t)(ok[i] && (pu[i] == pv[i] || x[2 * i] == x[2 * i + 1]));
        }
    }
    return bad;
}

// Algorithm 1 over E pairs per thread. Lanes of a warp own consecutive pairs,
// so the pair loads (16 B per lane) and the answer stores (E bytes per lane)
// are coalesced across the warp.
//  MODE 0: read-only finds through the read-only data path; the 2E walks of a
//          thread advance in lockstep so their loads overlap.
//  MODE 1: finds with path halving, one pair after the other (they write, so
//          ordinary loads).
//  MODE 2: flat forest (every tree of height <= 1): parent equality decides.
//  MODE 3: the 2E walks in lockstep with path splitting (they write).
// PERSIST: a persistent grid that loads the next chunk's pairs before working
// on the current one, so those loads overlap the parent reads.
// early: as for k_update.
template <int E, int MODE, bool PERSIST>
__global__ void __launch_bounds__(1024)
k_query(int* __restrict__ parent, int n, const int* __restrict__ pairs, int64_t k, int vec,
        uint8_t* __restrict__ out, int ovec, DevState* __restrict__ ds, int early,
        const unsigned* __restrict__ big) {
    pdl_trigger();
    if (!early) pdl_wait();
    int64_t e0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * E;
    if (e0 >= k) return;
    bool bad = false;
    int u[E], v[E];
    uint8_t a[E];
    load_pairs<E>(pairs, e0, k, vec, u, v);
    if (early) pdl_wait();
    const unsigned* bits = big_active(big, ds);
    if (!PERSIST) {
        bad = query_chunk<E, MODE>(parent, n, u, v, e0, k, a, ds, bits);
        store_answers<E>(out, e0, k, ovec != 0, a);
    } else {
        const int64_t stride = (int64_t)gridDim.x * blockDim.x * E;
        while (e0 < k) {
            const int64_t nx = e0 + stride;
            int nu[E] = {}, nv[E] = {};
            if (nx < k) load_pairs<E>(pairs, nx, k, vec, nu, nv);
            bad |= query_chunk<E, MODE>(parent, n, u, v, e0, k, a, ds, bits);
            store_answers<E>(out, e0, k, ovec != 0, a);
#pragma unroll
            for (int i = 0; i < E; i++) {
                u[i] = nu[i];
                v[i] = nv[i];
            }
            e0 = nx;
        }
    }
    if (bad) flag(ds, ST_RANGE);
}

// Algorithm 1 with the warp as the unit of work. A warp takes chunks of
// 32 * CH consecutive pairs; each lane keeps S pairs in flight, and every
// round advances each unfinished walk one step (read-only, as MODE 0: all
// of a lane's loads of a round are independent). A finished pair writes its
// answer, and its slot takes the next pair of the chunk at once: a ballot
// over the finished slots gives each a distinct index, so the lanes whose
// walks are short keep working while another lane walks a long path, instead
// of idling until the warp's longest walk ends. A pair whose first parents
// are equal is answered after its first round.
template <int S, int CH>
__global__ void __launch_bounds__(1024)
k_query_warp(const int* __restrict__ parent, int n, const int* __restrict__ pairs, int64_t k, int vec,
             uint8_t* __restrict__ out, DevState* __restrict__ ds) {
    pdl_trigger();
    pdl_wait();
    const unsigned full = 0xffffffffu;
    const int lane = (int)(threadIdx.x & 31u);
    const unsigned lt = (1u << lane) - 1u;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    bool bad = false, corrupt = false;
    for (int64_t base = warp * 32 * CH; base < k; base += nwarps * 32 * CH) {
        const int64_t end = base + 32 * CH < k ? base + 32 * CH : k;
        int64_t next = base;  // warp-uniform: the next pair of the chunk not yet taken
        int64_t idx[S];
        int xu[S], pu[S], xv[S], pv[S];
        bool act[S], eq[S];
#pragma unroll
        for (int j = 0; j < S; j++) {
            act[j] = false;
            eq[j] = false;
            idx[j] = 0;
            xu[j] = pu[j] = xv[j] = pv[j] = 0;
        }
        bool take[S];
#pragma unroll
        for (int j = 0; j < S; j++) take[j] = true;
        while (true) {
            // hand the next pairs of the chunk to the slots that are free
#pragma unroll
            for (int j = 0; j < S; j++) {
                const unsigned want = __ballot_sync(full, take[j]);
                if (take[j]) {
                    idx[j] = next + __popc(want & lt);
                    act[j] = idx[j] < end;
                    if (act[j]) {
                        int u, v;
                        if (vec >= 1) {
                            const int2 q = __ldcs(reinterpret_cast<const int2*>(pairs) + idx[j]);
                            u = q.x;
                            v = q.y;
                        } else {
                            u = __ldcs(pairs + 2 * idx[j]);
                            v = __ldcs(pairs + 2 * idx[j] + 1);
                        }
                        if (!(in_range(u, n) && in_range(v, n))) {
                            bad = true;
                            out[idx[j]] = 0;
                            act[j] = false;
                        } else {
                            xu[j] = u;
                            xv[j] = v;
                            pu[j] = __ldg(parent + u);
                            pv[j] = __ldg(parent + v);
                            eq[j] = pu[j] == pv[j];
                        }
                    }
                    take[j] = false;
                }
                next += __popc(want);
            }
            bool any = false;
#pragma unroll
            for (int j = 0; j < S; j++) any |= act[j];
            if (!__any_sync(full, any) && next >= end) break;
            // one step of every unfinished walk; finished pairs answer and free their slot
#pragma unroll
            for (int j = 0; j < S; j++) {
                if (!act[j]) {
                    take[j] = next < end;  // an idle slot takes a pair while the chunk has any
                    continue;
                }
                if (!eq[j] && pu[j] < xu[j]) {
                    xu[j] = pu[j];
                    pu[j] = __ldg(parent + xu[j]);
                }
                if (!eq[j] && pv[j] < xv[j]) {
                    xv[j] = pv[j];
                    pv[j] = __ldg(parent + xv[j]);
                }
                if (eq[j] || (pu[j] >= xu[j] && pv[j] >= xv[j])) {
                    if (!eq[j] && (pu[j] > xu[j] || pv[j] > xv[j])) corrupt = true;
                    out[idx[j]] = (uint8_t)(eq[j] || xu[j] == xv[j]);
                    act[j] = false;
                    take[j] = true;
                }
            }
        }
    }
    if (bad) flag(ds, ST_RANGE);
    if (corrupt) flag(ds, ST_CORRUPT);
}

template <int E, int MODE, bool PERSIST>
static void query_one(unsigned g, int block, const cudaAccessPolicyWindow* window, int pdl, cudaStream_t s,
                      int* parent, int n, const int* pairs, int64_t k, int vec, uint8_t* out, int ovec,
                      DevState* ds, const unsigned* big) {
    if (PERSIST) {
        const int c = resident_grid<k_query<E, MODE, PERSIST>>(block);
        if (g > (unsigned)c) g = (unsigned)c;
    }
    launch_windowed(k_query<E, MODE, PERSIST>, g, block, s, window, pdl != 0, parent, n, pairs, k, vec, out, ovec,
                    ds, (int)(pdl == 2), big);
}

template <int MODE>
static void query_inst(unsigned g, Launch cfg, cudaStream_t s, int* parent, int n,
                       const int* pairs, int64_t k, int vec, uint8_t* out, int ovec, DevState* ds) {
#define CC_Q(E, P) query_one<E, MODE, P>(g, cfg.block, cfg.window, cfg.pdl, s, parent, n, pairs, k, vec, out, ovec, ds, cfg.big)
    const bool persist = cfg.query_variant == 1;
    switch (cfg.ept) {
        case 1: if (persist) CC_Q(1, true); else CC_Q(1, false); break;
        case 2: if (persist) CC_Q(2, true); else CC_Q(2, false); break;
        default: if (persist) CC_Q(4, true); else CC_Q(4, false); break;
    }
#undef CC_Q
}

cudaError_t launch_query(int* parent, int n, const int* pairs, int64_t k, uint8_t* out,
                         DevState* ds, int mode, Launch cfg, cudaStream_t s) {
    if (k <= 0) return cudaSuccess;
    if (cfg.query_variant == 2) {  // warp-cooperative, read-only walks whatever the mode
        constexpr int kS = 2, kCH = 16;
        const int64_t warps = (k + 32 * kCH - 1) / (32 * kCH);
        int64_t g = (warps * 32 + cfg.block - 1) / cfg.block;
        const int64_t cap = resident_grid<k_query_warp<kS, kCH>>(cfg.block);
        if (g > cap) g = cap;
        launch_windowed(k_query_warp<kS, kCH>, (unsigned)g, cfg.block, s, cfg.window, cfg.pdl != 0, (const int*)parent,
                        n, pairs, k, pair_vec(pairs), out, ds);
        return cudaGetLastError();
    }
    if (cfg.qept) cfg.ept = cfg.qept;
    const int vec = pair_vec(pairs);
    const int ovec = (reinterpret_cast<uintptr_t>(out) % cfg.ept) == 0;
    const unsigned g = blocks_for(k, (int64_t)cfg.ept * cfg.block);
    if (mode == 2) query_inst<2>(g, cfg, s, parent, n, pairs, k, vec, out, ovec, ds);
    else if (mode == 1) query_inst<1>(g, cfg, s, parent, n, pairs, k, vec, out, ovec, ds);
    else if (mode == 3) query_inst<3>(g, cfg, s, parent, n, pairs, k, vec, out, ovec, ds);
    else query_inst<0>(g, cfg, s, parent, n, pairs, k, vec, out, ovec, ds);
    return cudaGetLastError();
}

// ------------------------------------------------------------ compression

// Every vertex is pointed at its root (4 consecutive vertices per thread, one
// 16-byte read of their parents; the four walks advance in lockstep). Only
// entries that change are written. With OUT, the roots are also written to
// out[] -- the minimum-id labels, since the root is the smallest id of its
// tree. No hooks run concurrently, so the roots are fixed for the whole pass.
// With BIG, the pass also rewrites the largest-component bitmap: bit v = (the
// root of v is ds->big_root), one 32-bit word per 8 lanes (a warp covers 128
// consecutive vertices); every lane of a warp takes part, so threads past n
// do not leave early. (Counting the marked vertices here, one atomic per warp
// on one word, doubled the pass: launch_big_count does it on demand.)
template <bool OUT, bool BIG>
__global__ void __launch_bounds__(1024)
k_compress_all(int* __restrict__ parent, int64_t n, int* __restrict__ out,
               DevState* __restrict__ ds, unsigned* __restrict__ big) {
    const int64_t v0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (!BIG && v0 >= n) return;
    const bool full = v0 + 4 <= n;
    int p0[4], x[4], p[4];
    if (full) {
        int4 q = *reinterpret_cast<const int4*>(parent + v0);
        p0[0] = q.x; p0[1] = q.y; p0[2] = q.z; p0[3] = q.w;
    } else {
#pragma unroll
        for (int i = 0; i < 4; i++) p0[i] = v0 + i < n ? parent[v0 + i] : 0;
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
        x[i] = v0 + i < n ? (int)(v0 + i) : 0;  // past n: a walk of length 0
        p[i] = p0[i];
    }
    while (true) {
        bool any = false;
#pragma unroll
        for (int i = 0; i < 4; i++) {
            if (p[i] < x[i]) {
                x[i] = p[i];
                p[i] = parent[x[i]];
                any = true;
            }
        }
        if (!any) break;
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
        if (p[i] > x[i]) flag(ds, ST_CORRUPT);
        if (v0 + i < n && x[i] != p0[i]) parent[v0 + i] = x[i];
    }
    if (OUT) {
        if (full) {
            reinterpret_cast<int4*>(out)[v0 / 4] = make_int4(x[0], x[1], x[2], x[3]);
        } else {
#pragma unroll
            for (int i = 0; i < 4; i++)
                if (v0 + i < n) out[v0 + i] = x[i];
        }
    }
    if (BIG) {
        const int R = ds->big_root;  // the same for every thread
        if (R < 0) return;
        unsigned nib = 0;
#pragma unroll
        for (int i = 0; i < 4; i++)
            if (v0 + i < n && x[i] == R) nib |= 1u << i;
        const unsigned lane = threadIdx.x & 31u;
        unsigned w = nib << ((lane & 7u) * 4u);
        w |= __shfl_xor_sync(0xffffffffu, w, 1);
        w |= __shfl_xor_sync(0xffffffffu, w, 2);
        w |= __shfl_xor_sync(0xffffffffu, w, 4);
        if ((lane & 7u) == 0 && v0 < n) big[v0 >> 5] = w;  // word v0 / 32 holds vertices v0 .. v0 + 31
    }
}

// ds->big_members += the set bits of words[0, nwords): one atomic per CTA.
__global__ void __launch_bounds__(256)
k_big_count(const unsigned* __restrict__ words, int64_t nwords, DevState* __restrict__ ds) {
    __shared__ unsigned part[8];
    unsigned c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nwords; i += (int64_t)gridDim.x * blockDim.x)
        c += (unsigned)__popc(words[i]);
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += part[w];
        if (t) atomicAdd(&ds->big_members, t);
    }
}

cudaError_t launch_big_count(const unsigned* words, int64_t nwords, DevState* ds, cudaStream_t s) {
    if (nwords <= 0) return cudaSuccess;
    int64_t g = (nwords + 255) / 256;
    if (g > 1024) g = 1024;
    k_big_count<<<(unsigned)g, 256, 0, s>>>(words, nwords, ds);
    return cudaGetLastError();
}

// The root of the largest tree, estimated (the sampling step of Afforest's
// large-component skip): kBigSample vertices, spread over [0, n) by the
// golden-ratio sequence, are walked to their roots (read-only); the roots go
// into a shared-memory hash table with a count each, and the most frequent
// one (the smaller id on a tie) becomes ds->big_root if at least min_share of
// the sample reached it, else -1. One CTA of kBigSample threads.
__global__ void __launch_bounds__(kBigSample)
k_big_pick(const int* __restrict__ parent, int64_t n, int min_share, DevState* __restrict__ ds) {
    constexpr int kSlots = 2 * kBigSample;
    __shared__ int key[kSlots];
    __shared__ int cnt[kSlots];
    __shared__ unsigned long long best[kBigSample / 32];
    const int t = threadIdx.x;
    for (int i = t; i < kSlots; i += blockDim.x) {
        key[i] = -1;
        cnt[i] = 0;
    }
    // x = floor(frac((t + 1) * phi) * n), in [0, n)
    const uint64_t h = (uint64_t)(t + 1) * 0x9E3779B97F4A7C15ull;
    const int x = (int)(((h >> 32) * (uint64_t)n) >> 32);
    const int r = walk_root(parent, x, parent[x]);
    __syncthreads();
    unsigned slot = ((unsigned)r * 0x9E3779B1u) >> 21;  // 11 bits: kSlots slots
    for (int probe = 0; probe < kSlots; probe++) {       // at most kBigSample keys: a free slot exists
        const int prev = atomicCAS(&key[slot], -1, r);
        if (prev == -1 || prev == r) {
            atomicAdd(&cnt[slot], 1);
            break;
        }
        slot = (slot + 1) & (kSlots - 1);
    }
    __syncthreads();
    // (count, then the smaller id) as one 64-bit key; the maximum wins
    unsigned long long mine = 0;
    for (int i = t; i < kSlots; i += blockDim.x)
        if (cnt[i]) {
            const unsigned long long c = ((unsigned long long)cnt[i] << 32) | (unsigned)(0x7fffffff - key[i]);
            if (c > mine) mine = c;
        }
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, mine, d);
        if (o > mine) mine = o;
    }
    if ((t & 31) == 0) best[t >> 5] = mine;
    __syncthreads();
    if (t == 0) {
        unsigned long long b = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++)
            if (best[w] > b) b = best[w];
        const int count = (int)(b >> 32);
        const int root = 0x7fffffff - (int)(b & 0xffffffffu);
        ds->big_root = (b && count >= min_share) ? root : -1;
    }
}

cudaError_t launch_big_pick(const int* parent, int64_t n, int min_share, DevState* ds, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_big_pick<<<1, kBigSample, 0, s>>>(parent, n, min_share, ds);
    return cudaGetLastError();
}

cudaError_t launch_compress_all(int* parent, int64_t n, int* out, DevState* ds, int block,
                                cudaStream_t s, unsigned* big) {
    const unsigned g = blocks_for(n, 4LL * block);
    const bool aligned_out = out && reinterpret_cast<uintptr_t>(out) % 16 == 0;
    if (out && !aligned_out) {
        // labels into a buffer without 16-byte alignment: compress, then copy
        if (big) k_compress_all<false, true><<<g, block, 0, s>>>(parent, n, nullptr, ds, big);
        else k_compress_all<false, false><<<g, block, 0, s>>>(parent, n, nullptr, ds, nullptr);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        return cudaMemcpyAsync(out, parent, (size_t)n * sizeof(int), cudaMemcpyDeviceToDevice, s);
    }
    if (out) {
        if (big) k_compress_all<true, true><<<g, block, 0, s>>>(parent, n, out, ds, big);
        else k_compress_all<true, false><<<g, block, 0, s>>>(parent, n, out, ds, nullptr);
    } else {
        if (big) k_compress_all<false, true><<<g, block, 0, s>>>(parent, n, nullptr, ds, big);
        else k_compress_all<false, false><<<g, block, 0, s>>>(parent, n, nullptr, ds, nullptr);
    }
    return cudaGetLastError();
}

// Section 5.1's pragmatic compression for the endpoints of an edge array:
// find the root, then walk the path again pointing every node at it.
template <int E>
__global__ void __launch_bounds__(1024)
k_compress_touched(int* __restrict__ parent, int n, const int* __restrict__ edges, int64_t k,
                   int vec, DevState* __restrict__ ds) {
    const int64_t e0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * E;
    if (e0 >= k) return;
    int u[E], v[E];
    load_pairs<E>(edges, e0, k, vec, u, v);
#pragma unroll
    for (int j = 0; j < 2 * E; j++) {
        const int i = j >> 1;
        int x = (j & 1) ? v[i] : u[i];
        if (e0 + i >= k || !in_range(x, n)) continue;
        int p = parent[x];
        if (p >= x) continue;
        const int r = walk_root(parent, x, p);
        while (p != r && p < x) {
            parent[x] = r;
            x = p;
            p = parent[x];
        }
    }
}

cudaError_t launch_compress_touched(int* parent, int n, const int* edges, int64_t k,
                                    DevState* ds, Launch cfg, cudaStream_t s) {
    if (k <= 0) return cudaSuccess;
    const int vec = pair_vec(edges);
    const unsigned g = blocks_for(k, (int64_t)cfg.ept * cfg.block);
    switch (cfg.ept) {
        case 1: k_compress_touched<1><<<g, cfg.block, 0, s>>>(parent, n, edges, k, vec, ds); break;
        case 2: k_compress_touched<2><<<g, cfg.block, 0, s>>>(parent, n, edges, k, vec, ds); break;
        default: k_compress_touched<4><<<g, cfg.block, 0, s>>>(parent, n, edges, k, vec, ds); break;
    }
    return cudaGetLastError();
}

// ------------------------------------------------------- label validation

__global__ void __launch_bounds__(1024)
k_validate_labels(const int* __restrict__ lab, int64_t n, DevState* __restrict__ ds) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int root = 0;
    if (v < n) {
        const int l = lab[v];
        const bool good = l >= 0 && (int64_t)l <= v && lab[l] == l;
        if (!good) atomicOr(&ds->labels_bad, 1u);
        root = good && (int64_t)l == v;
    }
    root = __reduce_add_sync(0xffffffffu, root);
    if ((threadIdx.x & 31) == 0 && root) atomicAdd(&ds->roots, (unsigned long long)root);
}

__global__ void __launch_bounds__(1024)
k_validate_forest(const int* __restrict__ p, int64_t n, DevState* __restrict__ ds) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int root = 0;
    if (v < n) {
        const int x = p[v];
        if (x < 0 || (int64_t)x > v) atomicOr(&ds->labels_bad, 1u);
        root = (int64_t)x == v;
    }
    root = __reduce_add_sync(0xffffffffu, root);
    if ((threadIdx.x & 31) == 0 && root) atomicAdd(&ds->roots, (unsigned long long)root);
}

cudaError_t launch_validate_forest(const int* p, int64_t n, DevState* ds, int block, cudaStream_t s) {
    k_validate_forest<<<blocks_for(n, block), block, 0, s>>>(p, n, ds);
    return cudaGetLastError();
}

cudaError_t launch_validate_labels(const int* lab, int64_t n, DevState* ds, int block,
                                   cudaStream_t s) {
    k_validate_labels<<<blocks_for(n, block), block, 0, s>>>(lab, n, ds);
    return cudaGetLastError();
}

}  // namespace cc
