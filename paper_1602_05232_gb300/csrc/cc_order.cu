// Locality order for a Bulk-Update: the minibatch's edges are bucketed by
// the smaller of their two endpoints before the update kernel runs.
//
// Bulk-Update treats a minibatch as a set (Section 1, "Model"), so the order
// in which its edges are folded in does not change the result. It does change
// the cost on a GPU. The update's first step reads parent[u] and parent[v]
// for every edge (the relabel step of Algorithm 2); in a minibatch given in
// random order those are random 4-byte reads spread over the whole forest,
// and once the forest is larger than L2 each costs a DRAM burst of its own.
// Where the graph has locality in its vertex ids (a mesh numbered row by row:
// every edge joins ids at most one row apart), edges bucketed by their smaller
// endpoint make the warps in flight at any moment read one narrow band of the
// forest, which L2 then serves: the forest is swept roughly in address order,
// each line fetched about once per minibatch, and the roots of neighbouring
// vertices (often the same root) are hot as well.
//
// A counting sort into 2^b buckets (bucket = min(u, v) >> shift, shift chosen
// so that every id in [0, n) maps below 2^b), in two kernels:
//   1. k_order_count: every CTA counts its tiles' edges per bucket in shared
//      memory and adds the counts to totals[bucket];
//   2. k_order_scatter: every CTA turns totals into bucket starts (an
//      exclusive scan in shared memory), then for each of its tiles of
//      kTile edges sorts the tile by bucket in shared memory, reserves one
//      output range per bucket present with an atomic on fill[bucket], and
//      writes the tile out in runs of consecutive slots. The last CTA to
//      finish clears totals and fill for the next call.
// Edges with an endpoint outside [0, n) go to bucket 0 unchanged; the update
// kernel skips and reports them as it does for unordered input. The order
// within a bucket is arbitrary.
#include <cstdint>

#include "cc_device.cuh"
#include "cc_internal.cuh"

namespace cc {

namespace {

constexpr int kOrderBlock = 512;
constexpr int kOrderEpt = 8;                          // edges per thread per tile
constexpr int kTile = kOrderBlock * kOrderEpt;        // 4096 edges
constexpr int kMaxBuckets = 1 << 9;  // shared memory of the scatter kernel stays below 48 KiB

__device__ __forceinline__ void pdl_trigger_o() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_wait_o() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

__device__ __forceinline__ int order_key(int u, int v, int n, int shift) {
    if (!(in_range(u, n) && in_range(v, n))) return 0;
    return (u < v ? u : v) >> shift;
}

// In-place exclusive scan of a[0, nb) (nb <= 2 * blockDim.x, blockDim.x = kOrderBlock)
// in shared memory; `warp_sums` holds kOrderBlock / 32 ints. Returns the total.
__device__ __forceinline__ int block_exclusive_scan(int* a, int nb, int* warp_sums) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int i0 = 2 * t, i1 = 2 * t + 1;
    const int x0 = i0 < nb ? a[i0] : 0, x1 = i1 < nb ? a[i1] : 0;
    int s = x0 + x1, inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int w = lane < kOrderBlock / 32 ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kOrderBlock / 32) warp_sums[lane] = w;
    }
    __syncthreads();
    const int before = inc - s + (warp ? warp_sums[warp - 1] : 0);
    const int total = warp_sums[kOrderBlock / 32 - 1];
    __syncthreads();  // every thread has read warp_sums
    if (i0 < nb) a[i0] = before;
    if (i1 < nb) a[i1] = before + x0;
    __syncthreads();
    return total;
}

// early (programmatic dependent launch): read and count the edges before
// waiting for the kernel launched before this one, else wait first. Either
// way the wait comes before this kernel can complete, so the kernels after
// it still see everything before it complete.
__global__ void __launch_bounds__(kOrderBlock)
k_order_count(const int* __restrict__ edges, int64_t k, int vec, int n, int shift, int nb,
              int* __restrict__ totals, int early, const unsigned* big, const DevState* ds) {
    __shared__ int hist[kMaxBuckets];
    pdl_trigger_o();
    if (big && ds->big_root >= 0) {  // the update reads the caller's order (BigArgs)
        pdl_wait_o();                // still complete only after the kernel before
        return;
    }
    if (!early) pdl_wait_o();
    for (int b = threadIdx.x; b < nb; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    const int64_t tiles = (k + kTile - 1) / kTile;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t e0 = t * kTile + (int64_t)threadIdx.x * kOrderEpt;
        if (e0 >= k) continue;
        int u[kOrderEpt], v[kOrderEpt];
        load_pairs<kOrderEpt>(edges, e0, k, vec, u, v);
#pragma unroll
        for (int i = 0; i < kOrderEpt; i++)
            if (e0 + i < k) atomicAdd(&hist[order_key(u[i], v[i], n, shift)], 1);
    }
    if (early) pdl_wait_o();
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        if (hist[b]) atomicAdd(&totals[b], hist[b]);
}

__global__ void __launch_bounds__(kOrderBlock)
k_order_scatter(const int* __restrict__ edges, int64_t k, int vec, int n, int shift, int nb,
                int* __restrict__ totals, int* __restrict__ fill, unsigned* __restrict__ done,
                int2* __restrict__ out, const unsigned* big, const DevState* ds) {
    __shared__ int start[kMaxBuckets];   // global first slot of each bucket
    __shared__ int cnt[kMaxBuckets];     // this tile: edges per bucket, then their local starts
    __shared__ int gbase[kMaxBuckets];   // this tile: global slot of its first edge of each bucket
    __shared__ int2 stage[kTile];        // this tile, sorted by bucket
    __shared__ unsigned short skey[kTile];
    __shared__ int warp_sums[kOrderBlock / 32];
    __shared__ bool last;
    pdl_trigger_o();
    pdl_wait_o();  // totals are complete
    if (big && ds->big_root >= 0) return;  // as in k_order_count: nothing was counted
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        start[b] = totals[b];
        cnt[b] = 0;
    }
    __syncthreads();
    block_exclusive_scan(start, nb, warp_sums);
    const int64_t tiles = (k + kTile - 1) / kTile;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t t0 = t * kTile;
        const int count = k - t0 < kTile ? (int)(k - t0) : kTile;
        const int64_t e0 = t0 + (int64_t)threadIdx.x * kOrderEpt;
        int u[kOrderEpt], v[kOrderEpt], key[kOrderEpt], rank[kOrderEpt];
        if (e0 < k) load_pairs<kOrderEpt>(edges, e0, k, vec, u, v);
#pragma unroll
        for (int i = 0; i < kOrderEpt; i++) {
            key[i] = 0;
            rank[i] = 0;
            if (e0 + i < k) {
                key[i] = order_key(u[i], v[i], n, shift);
                rank[i] = atomicAdd(&cnt[key[i]], 1);
            }
        }
        __syncthreads();
        // reserve this tile's range in every bucket it has edges in
        for (int b = threadIdx.x; b < nb; b += blockDim.x)
            if (cnt[b]) gbase[b] = start[b] + atomicAdd(&fill[b], cnt[b]);
        __syncthreads();
        block_exclusive_scan(cnt, nb, warp_sums);  // cnt = local starts
#pragma unroll
        for (int i = 0; i < kOrderEpt; i++)
            if (e0 + i < k) {
                const int p = cnt[key[i]] + rank[i];
                stage[p] = make_int2(u[i], v[i]);
                skey[p] = (unsigned short)key[i];
            }
        __syncthreads();
        // slot p of the sorted tile: bucket b, at position p - (local start of b)
        for (int p = threadIdx.x; p < count; p += blockDim.x) {
            const int b = skey[p];
            out[gbase[b] + (p - cnt[b])] = stage[p];
        }
        __syncthreads();
        for (int b = threadIdx.x; b < nb; b += blockDim.x) cnt[b] = 0;
        __syncthreads();
    }
    // the last CTA to finish clears the counters for the next call
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
            totals[b] = 0;
            fill[b] = 0;
        }
        if (threadIdx.x == 0) *done = 0u;
    }
}

template <typename K, typename... Args>
cudaError_t launch_pdl(K kernel, unsigned grid, cudaStream_t s, bool pdl, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kOrderBlock);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

int order_grid(int64_t k) {
    static thread_local int cache[16] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    int* slot = (dev >= 0 && dev < 16) ? &cache[dev] : nullptr;
    int sms = slot && *slot ? *slot : 0;
    if (!sms) {
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
        if (slot) *slot = sms;
    }
    // up to two CTAs per SM (the scatter kernel's shared memory allows two),
    // but no more CTAs than tiles
    const int64_t tiles = (k + kTile - 1) / kTile;
    const int64_t g = 2LL * sms;
    return (int)(tiles < g ? (tiles > 0 ? tiles : 1) : g);
}

}  // namespace

int order_shift(int64_t n, int log_buckets) {
    int bits = 0;
    while (bits < 31 && ((int64_t)1 << bits) < n) bits++;  // ids < 2^bits
    return bits > log_buckets ? bits - log_buckets : 0;
}

int64_t order_counter_ints(int log_buckets) { return 2 * ((int64_t)1 << log_buckets) + 1; }

cudaError_t launch_order_edges(const int* edges, int64_t k, int n, int log_buckets, int* counters,
                               int* out, int pdl, cudaStream_t s, int* kernels, const unsigned* big,
                               const DevState* ds) {
    *kernels = 0;
    if (k <= 0) return cudaSuccess;
    if (log_buckets < 0 || (1 << log_buckets) > kMaxBuckets) return cudaErrorInvalidValue;
    const int nb = 1 << log_buckets;
    const int shift = order_shift(n, log_buckets);
    const int G = order_grid(k);
    const int vec = pair_vec(edges);
    int* totals = counters;
    int* fill = counters + nb;
    unsigned* done = reinterpret_cast<unsigned*>(counters + 2 * nb);
    // The count kernel becomes a dependent launch only when it reads its
    // edges before the wait (pdl 2): launched early just to wait, its CTAs
    // would hold SM slots that the previous kernel's remaining CTAs need.
    cudaError_t e = launch_pdl(k_order_count, (unsigned)G, s, pdl == 2, edges, k, vec, n, shift, nb, totals,
                               (int)(pdl == 2), big, ds);
    if (e != cudaSuccess) return e;
    e = launch_pdl(k_order_scatter, (unsigned)G, s, pdl != 0, edges, k, vec, n, shift, nb, totals, fill, done,
                   reinterpret_cast<int2*>(out), big, ds);
    *kernels = 2;
    return e;
}

}  // namespace cc
