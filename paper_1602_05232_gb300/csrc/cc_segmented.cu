// Batched form: many independent graphs, each with its own ordered list of
// Bulk-Update / Bulk-Query minibatches of any size (Section 1: minibatches
// need not be equal), all executed by ONE persistent kernel.
//
// Every graph g owns the slice parent[seg_off[g] .. seg_off[g+1]) of one
// forest, with its own local ids. A CTA claims a whole graph from a work
// queue (largest work first) and runs that graph's operations in list order,
// separated by __syncthreads(), so each bulk operation completes before the
// next one starts. A graph of at most `smem_cap` vertices is worked on in
// shared memory: its slice is loaded as 16-bit local ids (up to 65,536
// vertices = 128 KiB), finds and hooks use shared-memory atomics, and the
// slice is written back flattened (every vertex pointing at its root). Larger
// graphs are worked on in place in global memory with the plain path's
// find/hook. The work queue counter is the only scratch and is reset before
// every launch.
#include <cstdint>

#include "cc_device.cuh"
#include "cc_internal.cuh"

namespace cc {

namespace {

// --- shared-memory forest primitives (same invariant: sp[x] <= x) ---------

__device__ __forceinline__ int sfind(volatile unsigned short* sp, int x) {
    int p = sp[x];
    while (p != x) {
        int gp = sp[p];
        if (gp == p) return p;
        sp[x] = (unsigned short)gp;  // halving
        x = gp;
        p = sp[x];
    }
    return x;
}

__device__ __forceinline__ int sroot(const volatile unsigned short* sp, int x) {
    int p = sp[x];
    while (p < x) {
        x = p;
        p = sp[x];
    }
    return x;
}

// Roots of a and b, walked in lockstep with path splitting (every visited
// node is repointed at its grandparent): the two chains of dependent
// shared-memory loads are in flight together instead of one after the other.
__device__ __forceinline__ void sfind_pair(volatile unsigned short* sp, int& a, int& b) {
    int pa = sp[a], pb = sp[b];
    while (pa != a || pb != b) {
        const int ga = sp[pa], gb = sp[pb];  // both loads issued before either is used
        if (pa != a) {
            if (ga != pa) sp[a] = (unsigned short)ga;
            a = pa;
            pa = ga;
        }
        if (pb != b) {
            if (gb != pb) sp[b] = (unsigned short)gb;
            b = pb;
            pb = gb;
        }
    }
}

// Whether a and b have the same root, in a forest that does not change
// meanwhile (a Bulk-Query between barriers): both walks in lockstep, stopping
// early when they meet.
__device__ __forceinline__ bool ssame(const unsigned short* sp, int a, int b) {
    int pa = sp[a], pb = sp[b];
    while (a != b && (pa < a || pb < b)) {
        a = pa;
        b = pb;
        pa = sp[a];
        pb = sp[b];
    }
    return a == b;
}

__device__ __forceinline__ int shook(unsigned short* sp, int ru, int rv) {
    while (ru != rv) {
        const int hi = ru > rv ? ru : rv;
        const int lo = ru > rv ? rv : ru;
        const unsigned short old = atomicCAS(sp + hi, (unsigned short)hi, (unsigned short)lo);
        if (old == hi) return 1;
        const int r = sfind(sp, old);
        if (hi == ru) ru = r; else rv = r;
    }
    return 0;
}

// The operations [ob, oe) of one graph in shared memory, software-pipelined:
// an operation is cut into chunks of blockDim * E pairs, and while a chunk is
// being worked on, every thread already has the loads of its pairs of the
// NEXT chunk in flight -- the next chunk of the same operation, or the first
// one of the graph's next operation (its data does not depend on this one's
// result). A barrier separates consecutive operations only. Returns the
// number of links made.
template <int E>
__device__ __forceinline__ int seg_run_smem(unsigned short* sp, int ng, const SegOp* __restrict__ ops,
                                            int ob, int oe, DevState* ds) {
    const int64_t chunk = (int64_t)blockDim.x * E;
    const int64_t mine = (int64_t)threadIdx.x * E;
    int made = 0;
    bool bad = false;
    int o = ob;
    int64_t off = 0;
    // the current operation, field by field
    const int* data = nullptr;
    uint8_t* out = nullptr;
    int64_t k = 0;
    int kind = 0;
    int u[E] = {}, v[E] = {};
    if (o < oe) {
        data = ops[o].data; out = ops[o].out; k = ops[o].k; kind = ops[o].kind;
        if (mine < k) load_pairs<E>(data, mine, k, pair_vec_dev(data), u, v);
    }
    while (o < oe) {
        // where the next chunk is, and its loads
        int o2 = o;
        int64_t off2 = off + chunk;
        const int* data2 = data;
        uint8_t* out2 = out;
        int64_t k2 = k;
        int kind2 = kind;
        if (off2 >= k) {
            o2 = o + 1;
            off2 = 0;
            if (o2 < oe) {
                data2 = ops[o2].data; out2 = ops[o2].out; k2 = ops[o2].k; kind2 = ops[o2].kind;
            }
        }
        int nu[E] = {}, nv[E] = {};
        if (o2 < oe && off2 + mine < k2) load_pairs<E>(data2, off2 + mine, k2, pair_vec_dev(data2), nu, nv);
        // this chunk
        const int64_t i0 = off + mine;
        if (kind == CC_OP_UPDATE) {
#pragma unroll
            for (int j = 0; j < E; j++) {
                if (i0 + j >= k) break;
                if (!(in_range(u[j], ng) && in_range(v[j], ng))) {
                    bad = true;
                    continue;
                }
                int ru = u[j], rv = v[j];
                sfind_pair(sp, ru, rv);
                made += shook(sp, ru, rv);
            }
        } else {
#pragma unroll
            for (int j = 0; j < E; j++) {
                if (i0 + j >= k) break;
                uint8_t a = 0;
                if (in_range(u[j], ng) && in_range(v[j], ng))
                    a = (uint8_t)ssame(sp, u[j], v[j]);
                else
                    bad = true;
                out[i0 + j] = a;
            }
        }
        if (o2 != o) __syncthreads();  // the operation is complete before the next starts
#pragma unroll
        for (int j = 0; j < E; j++) {
            u[j] = nu[j];
            v[j] = nv[j];
        }
        o = o2; off = off2; data = data2; out = out2; k = k2; kind = kind2;
    }
    if (bad) flag(ds, ST_RANGE);
    return made;
}

// --- the same operations in place on the global forest (large graphs) ----

template <int E>
__device__ __forceinline__ int seg_update_global(int* parent, int64_t base, int ng,
                                                 const SegOp& op, DevState* ds) {
    const int vec = pair_vec_dev(op.data);
    int made = 0;
    bool bad = false;
    for (int64_t i = (int64_t)threadIdx.x * E; i < op.k; i += (int64_t)blockDim.x * E) {
        int u[E], v[E];
        load_pairs<E>(op.data, i, op.k, vec, u, v);
#pragma unroll
        for (int j = 0; j < E; j++) {
            if (i + j >= op.k) break;
            if (!(in_range(u[j], ng) && in_range(v[j], ng))) {
                bad = true;
                continue;
            }
            const int gu = (int)(base + u[j]), gv = (int)(base + v[j]);
            made += hook(parent, find_halving(parent, gu, ds), find_halving(parent, gv, ds), ds);
        }
    }
    if (bad) flag(ds, ST_RANGE);
    return made;
}

template <int E>
__device__ __forceinline__ void seg_query_global(int* parent, int64_t base, int ng,
                                                 const SegOp& op, DevState* ds) {
    const int vec = pair_vec_dev(op.data);
    bool bad = false;
    for (int64_t i = (int64_t)threadIdx.x * E; i < op.k; i += (int64_t)blockDim.x * E) {
        int u[E], v[E];
        load_pairs<E>(op.data, i, op.k, vec, u, v);
#pragma unroll
        for (int j = 0; j < E; j++) {
            if (i + j >= op.k) break;
            uint8_t a = 0;
            if (in_range(u[j], ng) && in_range(v[j], ng)) {
                const int gu = (int)(base + u[j]), gv = (int)(base + v[j]);
                a = (uint8_t)(walk_root(parent, gu, parent[gu]) == walk_root(parent, gv, parent[gv]));
            } else {
                bad = true;
            }
            op.out[i + j] = a;
        }
    }
    if (bad) flag(ds, ST_RANGE);
}

}  // namespace

template <int E>
__global__ void __launch_bounds__(1024, 1)
k_segmented(int* __restrict__ parent, const int64_t* __restrict__ seg_off, SegTables t,
            unsigned* __restrict__ queue, DevState* __restrict__ ds, int smem_cap) {
    extern __shared__ unsigned short sp[];
    __shared__ int s_idx;
    int made = 0;
    const int nactive = *t.nactive;
    for (;;) {
        if (threadIdx.x == 0) s_idx = (int)atomicAdd(queue, 1u);
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();  // all have read s_idx before thread 0 may overwrite it
        if (idx >= nactive) break;
        const int g = t.order[idx];
        const int64_t base = seg_off[g];
        const int ng = (int)(seg_off[g + 1] - base);
        const int ob = t.op_begin[g], oe = t.op_begin[g + 1];
        if (ng <= smem_cap) {
            // four loads in flight per thread, then the tail one at a time
            int v = threadIdx.x;
            for (; v + 3 * (int)blockDim.x < ng; v += 4 * blockDim.x) {
                int pv[4];
#pragma unroll
                for (int j = 0; j < 4; j++) pv[j] = __ldcs(parent + base + v + j * blockDim.x);
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const int w = v + j * blockDim.x;
                    int64_t l = (int64_t)pv[j] - base;
                    if (l < 0 || l > w) {  // not a forest of this slice: keep w alone
                        flag(ds, ST_CORRUPT);
                        l = w;
                    }
                    sp[w] = (unsigned short)l;
                }
            }
            for (; v < ng; v += blockDim.x) {
                const int64_t pv = (int64_t)parent[base + v] - base;
                if (pv < 0 || pv > v) {  // not a forest of this slice: keep v alone
                    flag(ds, ST_CORRUPT);
                    sp[v] = (unsigned short)v;
                } else {
                    sp[v] = (unsigned short)pv;
                }
            }
            __syncthreads();
            made += seg_run_smem<E>(sp, ng, t.ops, ob, oe, ds);
            for (int v = threadIdx.x; v < ng; v += blockDim.x)
                parent[base + v] = (int)(base + sroot(sp, v));
            __syncthreads();  // the slice is out before the buffer is reused
        } else {
            for (int o = ob; o < oe; o++) {
                const SegOp op = t.ops[o];
                if (op.kind == CC_OP_UPDATE) made += seg_update_global<E>(parent, base, ng, op, ds);
                else seg_query_global<E>(parent, base, ng, op, ds);
                __syncthreads();
            }
        }
    }
    made = __reduce_add_sync(0xffffffffu, made);
    if ((threadIdx.x & 31) == 0 && made) atomicAdd(&ds->unions, (unsigned long long)made);
}

template <int E>
static cudaError_t seg_prepare(SegLaunch& cfg) {
    const size_t smem = (size_t)cfg.smem_cap * sizeof(unsigned short);
    cudaError_t e = cudaFuncSetAttribute(k_segmented<E>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_segmented<E>, cfg.block, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    cfg.grid = per_sm * sms;
    if (cfg.max_ctas > 0 && cfg.grid > cfg.max_ctas) cfg.grid = cfg.max_ctas;
    return cudaSuccess;
}

cudaError_t prepare_segmented(SegLaunch& cfg) {
    switch (cfg.ept) {
        case 1: return seg_prepare<1>(cfg);
        case 2: return seg_prepare<2>(cfg);
        default: return seg_prepare<4>(cfg);
    }
}

cudaError_t launch_segmented(int* parent, const int64_t* seg_off, const SegTables& t,
                             unsigned* queue, DevState* ds, const SegLaunch& cfg, cudaStream_t s) {
    if (cfg.grid < 1) return cudaErrorInvalidConfiguration;
    const size_t smem = (size_t)cfg.smem_cap * sizeof(unsigned short);
    switch (cfg.ept) {
        case 1: k_segmented<1><<<cfg.grid, cfg.block, smem, s>>>(parent, seg_off, t, queue, ds, cfg.smem_cap); break;
        case 2: k_segmented<2><<<cfg.grid, cfg.block, smem, s>>>(parent, seg_off, t, queue, ds, cfg.smem_cap); break;
        default: k_segmented<4><<<cfg.grid, cfg.block, smem, s>>>(parent, seg_off, t, queue, ds, cfg.smem_cap); break;
    }
    return cudaGetLastError();
}

}  // namespace cc
