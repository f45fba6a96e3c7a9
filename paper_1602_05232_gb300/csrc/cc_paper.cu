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

#include "cc_append.cuh"
#include "cc_device.cuh"
#include "cc_internal.cuh"

namespace cc {

namespace {

// Step 1: one edge per thread. Every thread of the block reaches the append.
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
            // both first parent reads in flight together; a parent read before
            // the other walk's halving writes is still an ancestor of v
            const int pu = parent[u[0]], pv = parent[v[0]];
            ru = pu == u[0] ? u[0] : find_from(parent, u[0], pu, ds);
            rv = pv == v[0] ? v[0] : find_from(parent, v[0], pv, ds);
            if (ru != rv) {
                has = true;
                comp[ru] = ru;  // every endpoint of A'' starts as its own component
                comp[rv] = rv;
            }
        } else {
            flag(ds, ST_RANGE);
        }
    }
    append2_block(has, ru, rv, a2, m2);
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
// A root that ends many A'' edges (a hub's) has many copies: within a warp
// only one copy per distinct root tries, and a plain read that already shows
// the root linked skips the compare-and-swap, so the copies do not queue on
// its parent word. The loop is warp-uniform for the warp-wide steps.
__global__ void __launch_bounds__(1024)
k_join(const int* __restrict__ a2, const unsigned* __restrict__ m2, const int* __restrict__ comp,
       int* __restrict__ parent, DevState* __restrict__ ds) {
    const unsigned m2x2 = 2u * *m2;
    const unsigned lane = threadIdx.x & 31u;
    int made = 0;
    for (unsigned j0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); j0 < m2x2; j0 += gridDim.x * blockDim.x) {
        const unsigned j = j0 + lane;
        int x = -1, r = -1;
        if (j < m2x2) {
            x = a2[j];
            r = comp[x];
        }
        const bool live = j < m2x2 && r != x;
        const unsigned act = __ballot_sync(0xffffffffu, live);
        if (!live) continue;
        const unsigned g = __match_any_sync(act, x);
        if ((unsigned)(__ffs(g) - 1) == lane && *(volatile const int*)(parent + x) == x &&
            atomicCAS(parent + x, x, r) == x)
            made++;
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

// --- the hooking rounds as one CUDA graph with a device-side loop ----------
//
// pc[0] = |A''| (written by the relabel step), pc[1] = the hooked flag of the
// round just run, pc[2] = rounds run so far. The graph is
//   k_sv_start -> while (condition) { pc[1] = 0; k_sv_hook; k_sv_jump; k_sv_continue }
// so the rounds repeat on the device until one hooks nothing, with no host
// round trip between them.

namespace {

__global__ void k_sv_start(unsigned* __restrict__ pc, cudaGraphConditionalHandle h) {
    pc[2] = 0u;
    cudaGraphSetConditional(h, pc[0] > 0u ? 1u : 0u);  // an empty A'' needs no round
}

// Another round while the last one hooked. Each round that hooks removes at
// least one component root, so more than 2|A''| + 1 rounds means a broken
// forest: it is reported and the loop stops (the host loop's bound).
__global__ void k_sv_continue(unsigned* __restrict__ pc, cudaGraphConditionalHandle h,
                              DevState* __restrict__ ds) {
    const unsigned r = ++pc[2];
    unsigned go = pc[1] != 0u ? 1u : 0u;
    if (go && r >= 2u * pc[0] + 1u) {
        flag(ds, ST_CORRUPT);
        go = 0u;
    }
    cudaGraphSetConditional(h, go);
}

}  // namespace

cudaError_t build_sv_loop(const int* a2, unsigned* pc, int* comp, DevState* ds, int grid, int block,
                          cudaGraphExec_t* out) {
    *out = nullptr;
    cudaGraph_t g = nullptr;
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    cudaGraphConditionalHandle h = 0;
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, g, 0, 0);
    cudaGraphNode_t start = nullptr, loop = nullptr;
    if (e == cudaSuccess) {
        void* args[] = {&pc, &h};
        cudaKernelNodeParams kp = {};
        kp.func = reinterpret_cast<void*>(k_sv_start);
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(1);
        kp.kernelParams = args;
        e = cudaGraphAddKernelNode(&start, g, nullptr, 0, &kp);
    }
    cudaGraphNodeParams cp = {};
    if (e == cudaSuccess) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&loop, g, &start, nullptr, 1, &cp);
    }
    // the loop body, recorded by capturing the round's launches into it
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaStreamBeginCaptureToGraph(cs, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t e1 = cudaMemsetAsync(pc + 1, 0, sizeof(unsigned), cs);
        if (e1 == cudaSuccess) e1 = launch_sv_round(a2, pc, comp, pc + 1, grid, block, cs);
        if (e1 == cudaSuccess) {
            k_sv_continue<<<1, 1, 0, cs>>>(pc, h, ds);
            e1 = cudaGetLastError();
        }
        cudaGraph_t body = nullptr;
        e = cudaStreamEndCapture(cs, &body);
        if (e == cudaSuccess) e = e1;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    if (cs) cudaStreamDestroy(cs);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) *out = nullptr;
    return e;
}

}  // namespace cc

// ---------------------------------------------------------------------------
// Union by size (Section 3: the tree with fewer vertices goes under the one
// with more, which keeps every tree O(log n) high, Lemma 1). Only the paper's
// schedule can link this way without locks: within one minibatch each root
// of A'' is linked at most once, under its component's winner, which is not
// itself linked. Forests built this way no longer satisfy parent[v] <= v, so
// they are walked with the generic loops below (p != x), each capped at n
// steps: a longer walk can only mean a cycle, which is reported, not followed.
// ---------------------------------------------------------------------------

namespace cc {

namespace {

__device__ __forceinline__ int gfind(int* parent, int x, int n, DevState* ds) {
    int p = parent[x];
    for (int steps = 0; p != x; steps++) {
        if (steps > n) {
            flag(ds, ST_CORRUPT);
            return x;
        }
        const int gp = parent[p];
        if (gp == p) return p;
        parent[x] = gp;  // halving
        x = gp;
        p = parent[x];
    }
    return x;
}

__device__ __forceinline__ int groot(const int* parent, int x, int n, DevState* ds) {
    int p = parent[x];
    for (int steps = 0; p != x; steps++) {
        if (steps > n) {
            flag(ds, ST_CORRUPT);
            return x;
        }
        x = p;
        p = parent[x];
    }
    return x;
}

__global__ void __launch_bounds__(1024)
k_relabel_generic(int* __restrict__ parent, int n, const int* __restrict__ edges, int64_t k, int vec,
                  int* __restrict__ a2, unsigned* __restrict__ m2, int* __restrict__ comp,
                  unsigned long long* __restrict__ best, DevState* __restrict__ ds) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool has = false;
    int ru = 0, rv = 0;
    if (i < k) {
        int u[1], v[1];
        load_pairs<1>(edges, i, k, vec, u, v);
        if (in_range(u[0], n) && in_range(v[0], n)) {
            ru = gfind(parent, u[0], n, ds);
            rv = gfind(parent, v[0], n, ds);
            if (ru != rv) {
                has = true;
                comp[ru] = ru;
                comp[rv] = rv;
                best[ru] = 0ull;
                best[rv] = 0ull;
            }
        } else {
            flag(ds, ST_RANGE);
        }
    }
    append2_block(has, ru, rv, a2, m2);
}

// The vote key orders roots by size, then by smaller id.
__device__ __forceinline__ unsigned long long vote_key(int size, int x) {
    return ((unsigned long long)(unsigned)size << 32) | (unsigned long long)(0xffffffffu - (unsigned)x);
}

__global__ void __launch_bounds__(1024)
k_size_vote(const int* __restrict__ a2, const unsigned* __restrict__ m2, const int* __restrict__ comp,
            const int* __restrict__ size, unsigned long long* __restrict__ best) {
    // Most endpoints of A'' vote in the same few components (small trees
    // joining a giant one), so the votes are first reduced per component
    // within the warp: one atomicMax per distinct component per warp instead
    // of one per endpoint on the same word. The loop is warp-uniform so that
    // every lane takes part in the warp-wide steps.
    const unsigned m2x2 = 2u * *m2;
    const unsigned lane = threadIdx.x & 31u;
    for (unsigned j0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); j0 < m2x2; j0 += gridDim.x * blockDim.x) {
        const unsigned j = j0 + lane;
        const bool live = j < m2x2;
        int t = 0;
        unsigned long long key = 0ull;
        if (live) {
            const int x = a2[j];
            t = comp[x];
            key = vote_key(size[x], x);
        }
        const unsigned active = __ballot_sync(0xffffffffu, live);
        if (!live) continue;
        const unsigned g = __match_any_sync(active, t);
        unsigned long long m = key;
        for (unsigned rest = g; rest; rest &= rest - 1) {
            const unsigned long long o = __shfl_sync(g, key, __ffs(rest) - 1);
            m = o > m ? o : m;
        }
        if ((unsigned)(__ffs(g) - 1) == lane) atomicMax(best + t, m);
    }
}

__global__ void __launch_bounds__(1024)
k_size_join(const int* __restrict__ a2, const unsigned* __restrict__ m2, const int* __restrict__ comp,
            const unsigned long long* __restrict__ best, int* __restrict__ parent,
            int* __restrict__ size, DevState* __restrict__ ds) {
    // The sizes of the roots linked under one winner are summed within the
    // warp first (one atomicAdd per winner per warp), for the same reason.
    const unsigned m2x2 = 2u * *m2;
    const unsigned lane = threadIdx.x & 31u;
    int made = 0;
    for (unsigned j0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); j0 < m2x2; j0 += gridDim.x * blockDim.x) {
        const unsigned j = j0 + lane;
        bool linked = false;
        int w = 0, sx = 0;
        if (j < m2x2) {
            const int x = a2[j];
            w = (int)(0xffffffffu - (unsigned)(best[comp[x]] & 0xffffffffull));
            if (w != x && atomicCAS(parent + x, x, w) == x) {
                linked = true;
                sx = size[x];  // x is no longer a root: its size is final
                made++;
            }
        }
        const unsigned act = __ballot_sync(0xffffffffu, linked);
        if (!linked) continue;
        const unsigned g = __match_any_sync(act, w);
        const int sum = __reduce_add_sync(g, sx);
        if ((unsigned)(__ffs(g) - 1) == lane) atomicAdd(size + w, sum);
    }
    made = __reduce_add_sync(0xffffffffu, made);
    if ((threadIdx.x & 31) == 0 && made) atomicAdd(&ds->unions, (unsigned long long)made);
}

__global__ void __launch_bounds__(1024) k_fill(int* __restrict__ a, int64_t n, int value) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) a[v] = value;
}

// Sizes of a forest loaded from labels: every vertex adds one to its root.
__global__ void __launch_bounds__(1024)
k_size_count(const int* __restrict__ parent, int64_t n, int* __restrict__ size, DevState* ds) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) atomicAdd(size + groot(parent, (int)v, (int)n, ds), 1);
}

// Bulk-Query on any acyclic forest. FLAT: every tree has height <= 1.
template <bool FLAT>
__global__ void __launch_bounds__(1024)
k_query_generic(int* __restrict__ parent, int n, const int* __restrict__ pairs, int64_t k, int vec,
                uint8_t* __restrict__ out, DevState* __restrict__ ds) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k) return;
    int u[1], v[1];
    load_pairs<1>(pairs, i, k, vec, u, v);
    uint8_t a = 0;
    if (in_range(u[0], n) && in_range(v[0], n)) {
        if (FLAT) a = (uint8_t)(parent[u[0]] == parent[v[0]]);
        else a = (uint8_t)(gfind(parent, u[0], n, ds) == gfind(parent, v[0], n, ds));
    } else {
        flag(ds, ST_RANGE);
    }
    out[i] = a;
}

// Full compression on any acyclic forest; with MINID also the min-id reduce.
template <bool MINID>
__global__ void __launch_bounds__(1024)
k_compress_generic(int* __restrict__ parent, int64_t n, int* __restrict__ minid, DevState* ds) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int r = groot(parent, (int)v, (int)n, ds);
    if (parent[v] != r) parent[v] = r;
    if (MINID) atomicMin(minid + r, (int)v);
}

__global__ void __launch_bounds__(1024)
k_labels_generic(const int* __restrict__ parent, int64_t n, const int* __restrict__ minid,
                 int* __restrict__ out) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) out[v] = minid[parent[v]];  // parent[v] is v's root after the compression
}

__global__ void __launch_bounds__(1024)
k_depth(const int* __restrict__ parent, int64_t n, unsigned* __restrict__ max_depth,
        unsigned long long* __restrict__ sum_depth, DevState* ds) {
    const int64_t v0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned d = 0;
    if (v0 < n) {
        int x = (int)v0, p = parent[x];
        while (p != x && d <= (unsigned)n) {
            x = p;
            p = parent[x];
            d++;
        }
        if (d > (unsigned)n) flag(ds, ST_CORRUPT);
    }
    const unsigned mx = __reduce_max_sync(0xffffffffu, d);
    const unsigned sm = __reduce_add_sync(0xffffffffu, d);
    if ((threadIdx.x & 31) == 0) {
        if (mx) atomicMax(max_depth, mx);
        if (sm) atomicAdd(sum_depth, (unsigned long long)sm);
    }
}

}  // namespace

static inline unsigned grid1(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

cudaError_t launch_relabel_generic(int* parent, int n, const int* edges, int64_t k, int* a2,
                                   unsigned* m2, int* comp, unsigned long long* best, DevState* ds,
                                   int block, cudaStream_t s) {
    if (k <= 0) return cudaSuccess;
    k_relabel_generic<<<grid1(k, block), block, 0, s>>>(parent, n, edges, k, pair_vec(edges), a2, m2,
                                                        comp, best, ds);
    return cudaGetLastError();
}

cudaError_t launch_size_join(const int* a2, const unsigned* m2, const int* comp, int* parent,
                             int* size, unsigned long long* best, DevState* ds, int grid, int block,
                             cudaStream_t s) {
    k_size_vote<<<grid, block, 0, s>>>(a2, m2, comp, size, best);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_size_join<<<grid, block, 0, s>>>(a2, m2, comp, best, parent, size, ds);
    return cudaGetLastError();
}

cudaError_t launch_fill(int* a, int64_t n, int value, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_fill<<<grid1(n, 256), 256, 0, s>>>(a, n, value);
    return cudaGetLastError();
}

cudaError_t launch_size_count(const int* parent, int64_t n, int* size, DevState* ds, cudaStream_t s) {
    cudaError_t e = launch_fill(size, n, 0, s);
    if (e != cudaSuccess) return e;
    k_size_count<<<grid1(n, 256), 256, 0, s>>>(parent, n, size, ds);
    return cudaGetLastError();
}

cudaError_t launch_query_generic(int* parent, int n, const int* pairs, int64_t k, uint8_t* out,
                                 DevState* ds, bool flat, int block, cudaStream_t s) {
    if (k <= 0) return cudaSuccess;
    if (flat) k_query_generic<true><<<grid1(k, block), block, 0, s>>>(parent, n, pairs, k, pair_vec(pairs), out, ds);
    else k_query_generic<false><<<grid1(k, block), block, 0, s>>>(parent, n, pairs, k, pair_vec(pairs), out, ds);
    return cudaGetLastError();
}

cudaError_t launch_compress_generic(int* parent, int64_t n, int* labels_out, int* minid_scratch,
                                    DevState* ds, int block, cudaStream_t s) {
    if (!labels_out) {
        k_compress_generic<false><<<grid1(n, block), block, 0, s>>>(parent, n, nullptr, ds);
        return cudaGetLastError();
    }
    cudaError_t e = launch_fill(minid_scratch, n, 0x7fffffff, s);
    if (e != cudaSuccess) return e;
    k_compress_generic<true><<<grid1(n, block), block, 0, s>>>(parent, n, minid_scratch, ds);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_labels_generic<<<grid1(n, block), block, 0, s>>>(parent, n, minid_scratch, labels_out);
    return cudaGetLastError();
}

namespace {
__global__ void __launch_bounds__(1024)
k_filter_roots(const int* __restrict__ res, int64_t k, int* __restrict__ a2, unsigned* __restrict__ m2,
               int* __restrict__ comp, unsigned long long* __restrict__ best) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool has = false;
    int ru = 0, rv = 0;
    if (i < k) {
        ru = res[2 * i];
        rv = res[2 * i + 1];
        if (ru >= 0 && rv >= 0 && ru != rv) {
            has = true;
            comp[ru] = ru;
            comp[rv] = rv;
            if (best) {
                best[ru] = 0ull;
                best[rv] = 0ull;
            }
        }
    }
    append2_block(has, ru, rv, a2, m2);
}
}  // namespace

cudaError_t launch_filter_roots(const int* res, int64_t k, int* a2, unsigned* m2, int* comp,
                                unsigned long long* best, int block, cudaStream_t s) {
    if (k <= 0) return cudaSuccess;
    k_filter_roots<<<grid1(k, block), block, 0, s>>>(res, k, a2, m2, comp, best);
    return cudaGetLastError();
}

cudaError_t launch_depth(const int* parent, int64_t n, unsigned* max_depth,
                         unsigned long long* sum_depth, DevState* ds, cudaStream_t s) {
    k_depth<<<grid1(n, 256), 256, 0, s>>>(parent, n, max_depth, sum_depth, ds);
    return cudaGetLastError();
}

}  // namespace cc
