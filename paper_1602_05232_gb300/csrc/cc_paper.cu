// The paper's own Bulk-Update schedule (Algorithm 2), kept as an A/B option
// beside the fused CAS-hooking kernel:
//   1. relabel every edge (u, v) to (find(u), find(v)) and drop the pairs
//      whose roots agree (Algorithm 2's relabel and self-loop filter): the
//      survivors are compacted into A'';
//   2. connected components of A'' over the supernodes (Algorithm 2's CC
//      step), by an edge-list Shiloach-Vishkin pass: every round each edge
//      hooks the larger of its two component roots under the smaller
//      (atomicMin, only while that root is a root), then every endpoint
//      jumps to its root; rounds repeat until no edge hooks;
//   3. join each component of A'' in the forest (Algorithm 3's job): all its
//      roots are distinct roots of the forest, so each is pointed straight at
//      the component's smallest root -- one conflict-free write per root
//      instead of Parallel-Join's log-depth recursion.
// The forest keeps the invariant parent[v] <= v (every write points a root at
// a smaller root), so the plain path's query and label kernels apply as is.
#include <cstdint>

#include "cc_device.cuh"
#include "cc_internal.cuh"

namespace cc {

namespace {

// Append one pair per lane that has one, with one atomic per warp.
__device__ __forceinline__ void append_pair(bool has, int a, int b, int* __restrict__ out,
                                            unsigned* __restrict__ count) {
    const unsigned mask = __ballot_sync(0xffffffffu, has);
    if (!mask) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(count, (unsigned)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (has) {
        const unsigned slot = base + __popc(mask & ((1u << lane) - 1));
        out[2 * slot] = a;
        out[2 * slot + 1] = b;
    }
}

// Step 1: one edge per thread. Every thread of a warp reaches the ballot.
__global__ void __launch_bounds__(1024)
k_relabel(int* __restrict__ parent, int n, const int* __restrict__ edges, int64_t k, int vec,
          int* __restrict__ a2, unsigned* __restrict__ m2, int* __restrict__ comp,
          DevState* __restrict__ ds) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool has = false;
    int ru = 0, rv = 0;
    if (i < k) {
        int u[1], v[1];
        load_pairs<1>(edges, i, k, vec, u, v);
        if (in_range(u[0], n) && in_range(v[0], n)) {
            ru = find_halving(parent, u[0], ds);
            rv = find_halving(parent, v[0], ds);
            if (ru != rv) {
                has = true;
                comp[ru] = ru;  // every endpoint of A'' starts as its own component
                comp[rv] = rv;
            }
        } else {
            flag(ds, ST_RANGE);
        }
    }
    append_pair(has, ru, rv, a2, m2);
}

// Step 2a: hooking. The larger component root goes under the smaller one.
__global__ void __launch_bounds__(1024)
k_sv_hook(const int* __restrict__ a2, const unsigned* __restrict__ m2, int* __restrict__ comp,
          unsigned* __restrict__ hooked) {
    const unsigned m = *m2;
    bool any = false;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const int ca = comp[a2[2 * i]], cb = comp[a2[2 * i + 1]];
        if (ca == cb) continue;
        const int hi = ca > cb ? ca : cb, lo = ca > cb ? cb : ca;
        if (comp[hi] == hi) {
            atomicMin(comp + hi, lo);
            any = true;
        }
    }
    if (__any_sync(0xffffffffu, any) && (threadIdx.x & 31) == 0) *hooked = 1u;
}

// Step 2b: pointer jumping. Every endpoint of A'' points at its root.
__global__ void __launch_bounds__(1024)
k_sv_jump(const int* __restrict__ a2, const unsigned* __restrict__ m2, int* __restrict__ comp) {
    const unsigned m2x2 = 2u * *m2;
    for (unsigned j = blockIdx.x * blockDim.x + threadIdx.x; j < m2x2; j += gridDim.x * blockDim.x) {
        const int x = a2[j];
        int r = comp[x];
        while (comp[r] < r) r = comp[r];  // component labels only decrease
        comp[x] = r;
    }
}

// Step 3: join. Every root x of A'' is pointed at its component's smallest
// root; the compare-and-swap lets exactly one of x's copies count the link.
__global__ void __launch_bounds__(1024)
k_join(const int* __restrict__ a2, const unsigned* __restrict__ m2, const int* __restrict__ comp,
       int* __restrict__ parent, DevState* __restrict__ ds) {
    const unsigned m2x2 = 2u * *m2;
    int made = 0;
    for (unsigned j = blockIdx.x * blockDim.x + threadIdx.x; j < m2x2; j += gridDim.x * blockDim.x) {
        const int x = a2[j];
        const int r = comp[x];
        if (r != x && atomicCAS(parent + x, x, r) == x) made++;
    }
    made = __reduce_add_sync(0xffffffffu, made);
    if ((threadIdx.x & 31) == 0 && made) atomicAdd(&ds->unions, (unsigned long long)made);
}

}  // namespace

cudaError_t launch_relabel(int* parent, int n, const int* edges, int64_t k, int* a2, unsigned* m2,
                           int* comp, DevState* ds, int block, cudaStream_t s) {
    if (k <= 0) return cudaSuccess;
    const unsigned g = (unsigned)((k + block - 1) / block);
    k_relabel<<<g, block, 0, s>>>(parent, n, edges, k, pair_vec(edges), a2, m2, comp, ds);
    return cudaGetLastError();
}

cudaError_t launch_sv_round(const int* a2, const unsigned* m2, int* comp, unsigned* hooked,
                            int grid, int block, cudaStream_t s) {
    k_sv_hook<<<grid, block, 0, s>>>(a2, m2, comp, hooked);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sv_jump<<<grid, block, 0, s>>>(a2, m2, comp);
    return cudaGetLastError();
}

cudaError_t launch_join(const int* a2, const unsigned* m2, const int* comp, int* parent,
                        DevState* ds, int grid, int block, cudaStream_t s) {
    k_join<<<grid, block, 0, s>>>(a2, m2, comp, parent, ds);
    return cudaGetLastError();
}

}  // namespace cc
