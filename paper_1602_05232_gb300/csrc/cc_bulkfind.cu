// Bulk-Find (Algorithm 4; Section 4): the roots of a set S of vertices with
// path compression shared across the whole set.
//
// Phase I walks up from all of S at once, one level per kernel: the frontier
// F_i starts deduplicated (removeDup), every frontier node v that is not a
// root records the pair (parent[v], v) into R_u and sends its parent on to
// F_{i+1} -- unless the parent was already visited or another flow got there
// first in this level (both are one atomic exchange on an epoch-stamped mark
// array, so "visited" never has to be cleared). Roots are collected.
//
// The Response Distributor (Section 4.1) indexes R_u by `from`: a
// multiply-shift hash into rho = 3|R_u| buckets, a counting sort of the pairs
// by bucket (histogram, exclusive scan, scatter) and the bucket offsets.
// allFrom(f) scans bucket h(f) for pairs whose `from` is f.
//
// Phase II walks back down from the roots, one level per kernel: every (v, r)
// in D_i sets parent[v] = r and expands to (u, r) for each u in allFrom(v).
// Afterwards every traversed node points at its root and res[i] =
// parent[S[i]]. Every level's frontier holds at most |S| entries (each
// traversed node is on some query's path, and a path has one node per level).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "cc_append.cuh"
#include "cc_device.cuh"
#include "cc_internal.cuh"

namespace cc {

namespace {

// Multiply-shift hash of a vertex id into [0, rho).
__device__ __forceinline__ unsigned rd_hash(int f, unsigned rho) {
    const unsigned h = (unsigned)f * 0x9E3779B1u;
    return (unsigned)(((unsigned long long)h * rho) >> 32);
}

// F_0 = removeDup(S): the first lane to stamp a vertex with this epoch keeps it.
__global__ void __launch_bounds__(1024)
k_bf_seed(const int* __restrict__ S, int64_t k, int n, int* __restrict__ mark, int epoch,
          int* __restrict__ front, unsigned* __restrict__ count, DevState* __restrict__ ds) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool has = false, ok = false;
    int s = 0;
    if (i < k) {
        s = S[i];
        ok = in_range(s, n);
        if (!ok) flag(ds, ST_RANGE);
    }
    // Query sets repeat popular vertices: one lane per distinct vertex per
    // warp stamps it, after a read that does not already show this call's stamp.
    const unsigned act = __ballot_sync(0xffffffffu, ok);
    if (ok) {
        const unsigned g = __match_any_sync(act, s);
        if ((unsigned)(__ffs(g) - 1) == (threadIdx.x & 31u))
            has = *(volatile const int*)(mark + s) != epoch && atomicExch(mark + s, epoch) != epoch;
    }
    append1_block(has, s, front, count);
}

// One Phase I level.
__global__ void __launch_bounds__(1024)
k_bf_up(const int* __restrict__ front, unsigned c, const int* __restrict__ parent,
        int* __restrict__ mark, int epoch, int* __restrict__ next, unsigned* __restrict__ next_count,
        int* __restrict__ roots, unsigned* __restrict__ roots_count, int* __restrict__ R,
        unsigned* __restrict__ R_count) {
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    int v = 0, p = 0;
    bool live = i < c;
    if (live) {
        v = front[i];
        p = parent[v];
    }
    const bool is_root = live && p == v;
    const bool edge = live && p != v;
    append1_block(is_root, v, roots, roots_count);
    append2_block(edge, p, v, R, R_count);
    // Only the first to stamp p carries the flow on. Many frontier nodes share
    // a parent (a big tree's root): within a warp one lane per distinct parent
    // stamps it, and a read that already shows this call's stamp skips the
    // exchange, so the nodes do not queue on that one mark word.
    const unsigned act = __ballot_sync(0xffffffffu, edge);
    bool go_on = false;
    if (edge) {
        const unsigned g = __match_any_sync(act, p);
        if ((unsigned)(__ffs(g) - 1) == (threadIdx.x & 31u))
            go_on = *(volatile const int*)(mark + p) != epoch && atomicExch(mark + p, epoch) != epoch;
    }
    append1_block(go_on, p, next, next_count);
}

// atomicAdd(counter + key, 1) for every live lane, one atomic per distinct
// key in the warp (many pairs share a `from`, e.g. a big tree's root); returns
// the value each lane would have got from its own atomic.
__device__ __forceinline__ int add_one_grouped(bool live, unsigned key, int* __restrict__ counter) {
    const unsigned live_mask = __ballot_sync(0xffffffffu, live);
    const unsigned peers = __match_any_sync(0xffffffffu, live ? key : 0xffffffffu) & live_mask;
    int base = 0;
    if (live) {
        const int lane = threadIdx.x & 31;
        const int leader = __ffs(peers) - 1;
        if (lane == leader) base = atomicAdd(counter + key, __popc(peers));
        base = __shfl_sync(peers, base, leader);
        base += __popc(peers & ((1u << lane) - 1));
    }
    return base;
}

// Response Distributor: histogram of the pairs' buckets.
__global__ void __launch_bounds__(1024)
k_rd_hist(const int* __restrict__ R, unsigned lambda, unsigned rho, int* __restrict__ bucket) {
    const unsigned j = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = j < lambda;
    add_one_grouped(live, live ? rd_hash(R[2 * j], rho) : 0u, bucket);
}

// Response Distributor: scatter the pairs to their bucket's range.
__global__ void __launch_bounds__(1024)
k_rd_scatter(const int* __restrict__ R, unsigned lambda, unsigned rho, int* __restrict__ cursor,
             int* __restrict__ sorted) {
    const unsigned j = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = j < lambda;
    const int f = live ? R[2 * j] : 0;
    const int pos = add_one_grouped(live, live ? rd_hash(f, rho) : 0u, cursor);
    if (live) {
        sorted[2 * pos] = f;
        sorted[2 * pos + 1] = R[2 * j + 1];
    }
}

__global__ void __launch_bounds__(1024)
k_bf_roots_to_d(const int* __restrict__ roots, unsigned c, int* __restrict__ D) {
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < c) {
        D[2 * i] = roots[i];
        D[2 * i + 1] = roots[i];
    }
}

// One Phase II level, first half: point v at r and size the bucket that
// allFrom(v) has to scan (work[i]; work[c] = 0 so the scan yields the total).
__global__ void __launch_bounds__(1024)
k_bf_down_point(const int* __restrict__ D, unsigned c, int* __restrict__ parent,
                const int* __restrict__ offset, unsigned rho, int* __restrict__ work) {
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < c) {
        const int v = D[2 * i], r = D[2 * i + 1];
        if (v != r) parent[v] = r;
        const unsigned b = rd_hash(v, rho);
        work[i] = offset[b + 1] - offset[b];
    } else if (i == c) {
        work[c] = 0;
    }
}

// Second half: allFrom(v) for every v of D_i at once, one thread per bucket
// slot to scan (the slots of all buckets are laid end to end by the exclusive
// scan of the sizes, and each thread finds its D entry by binary search), so
// a bucket as large as a big tree's fan-in is scanned in parallel.
__global__ void __launch_bounds__(1024)
k_bf_down_expand(const int* __restrict__ D, unsigned c, const int* __restrict__ work_off,
                 unsigned total, const int* __restrict__ sorted, const int* __restrict__ offset,
                 unsigned rho, int* __restrict__ next, unsigned* __restrict__ next_count) {
    const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
    bool has = false;
    int u = 0, r = 0;
    if (t < total) {
        unsigned lo = 0, hi = c;  // last i with work_off[i] <= t
        while (hi - lo > 1) {
            const unsigned mid = (lo + hi) >> 1;
            if ((unsigned)work_off[mid] <= t) lo = mid; else hi = mid;
        }
        const int v = D[2 * lo];
        const int j = offset[rd_hash(v, rho)] + (int)(t - (unsigned)work_off[lo]);
        if (sorted[2 * j] == v) {
            has = true;
            u = sorted[2 * j + 1];
            r = D[2 * lo + 1];
        }
    }
    append2_block(has, u, r, next, next_count);
}

__global__ void __launch_bounds__(1024)
k_bf_gather(const int* __restrict__ S, int64_t k, int n, const int* __restrict__ parent,
            int* __restrict__ res) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k) {
        const int s = S[i];
        res[i] = in_range(s, n) ? parent[s] : -1;
    }
}

__global__ void __launch_bounds__(1024)
k_bf_answers(const int* __restrict__ res, int64_t k, uint8_t* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k) {
        const int a = res[2 * i], b = res[2 * i + 1];
        out[i] = (uint8_t)(a >= 0 && a == b);
    }
}

// ---- exclusive scan (in place), used by the Response Distributor's sort ----

constexpr int kScanBlock = 1024, kScanItems = 4, kScanTile = kScanBlock * kScanItems;

__global__ void __launch_bounds__(kScanBlock)
k_scan_tiles(int* __restrict__ a, int64_t len, int* __restrict__ tile_sums) {
    __shared__ int warp_sums[kScanBlock / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int v[kScanItems];
    int sum = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        v[j] = base + j < len ? a[base + j] : 0;
        sum += v[j];
    }
    // inclusive scan of the per-thread sums across the block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = warp_sums[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_sums[lane] = w;
    }
    __syncthreads();
    int run = x - sum + (warp ? warp_sums[warp - 1] : 0);  // exclusive prefix of this thread
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        if (base + j < len) a[base + j] = run;
        run += v[j];
    }
    if (threadIdx.x == kScanBlock - 1 && tile_sums) tile_sums[blockIdx.x] = run;
}

__global__ void __launch_bounds__(kScanBlock)
k_scan_add(int* __restrict__ a, int64_t len, const int* __restrict__ tile_offsets) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    const int add = tile_offsets[blockIdx.x];
#pragma unroll
    for (int j = 0; j < kScanItems; j++)
        if (base + j < len) a[base + j] += add;
}

}  // namespace

int64_t scan_scratch_ints(int64_t len) {
    int64_t total = 0;
    while (len > kScanTile) {
        len = (len + kScanTile - 1) / kScanTile;
        total += len;
    }
    return total + 1;
}

cudaError_t exclusive_scan(int* a, int64_t len, int* scratch, cudaStream_t s) {
    if (len <= 0) return cudaSuccess;
    const int64_t tiles = (len + kScanTile - 1) / kScanTile;
    if (tiles == 1) {
        k_scan_tiles<<<1, kScanBlock, 0, s>>>(a, len, nullptr);
        return cudaGetLastError();
    }
    k_scan_tiles<<<(unsigned)tiles, kScanBlock, 0, s>>>(a, len, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = exclusive_scan(scratch, tiles, scratch + tiles, s);
    if (e != cudaSuccess) return e;
    k_scan_add<<<(unsigned)tiles, kScanBlock, 0, s>>>(a, len, scratch);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- driver

static unsigned blocks(int64_t work, int block = 256) { return (unsigned)((work + block - 1) / block); }

static cudaError_t grow(int** p, int64_t* cap, int64_t need, int64_t ints_per) {
    if (need <= *cap) return cudaSuccess;
    int64_t c = *cap ? *cap : 1024;
    while (c < need) c *= 2;
    int* q = nullptr;
    cudaError_t e = cudaMalloc(&q, sizeof(int) * (size_t)(c * ints_per));
    if (e != cudaSuccess) return e;
    cudaFree(*p);
    *p = q;
    *cap = c;
    return cudaSuccess;
}

void bulk_find_free(BulkFindState& b) {
    cudaFree(b.mark);
    cudaFree(b.front[0]);
    cudaFree(b.front[1]);
    cudaFree(b.roots);
    cudaFree(b.R);
    cudaFree(b.sorted);
    cudaFree(b.bucket);
    cudaFree(b.cursor);
    cudaFree(b.scan);
    cudaFree(b.D[0]);
    cudaFree(b.D[1]);
    cudaFree(b.work);
    cudaFree(b.res);
    cudaFree(b.count);
    b = BulkFindState{};
}

static cudaError_t read_count(const unsigned* d, unsigned* h, cudaStream_t s) {
    cudaError_t e = cudaMemcpyAsync(h, d, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
}

cudaError_t bulk_find(BulkFindState& b, int* parent, int n, const int* S, int64_t k, int* res,
                      DevState* ds, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    if (!b.mark) {
        e = cudaMalloc(&b.mark, sizeof(int) * (size_t)n);
        if (e == cudaSuccess) e = cudaMemsetAsync(b.mark, 0, sizeof(int) * (size_t)n, s);
        if (e == cudaSuccess) e = cudaMalloc(&b.count, 4 * sizeof(unsigned));
        if (e != cudaSuccess) return e;
        b.epoch = 0;
    }
    if (b.epoch >= 0x7ffffff0) {  // stamps would wrap: start over
        e = cudaMemsetAsync(b.mark, 0, sizeof(int) * (size_t)n, s);
        if (e != cudaSuccess) return e;
        b.epoch = 0;
    }
    const int epoch = ++b.epoch;
    int64_t cap_s = b.cap_front;
    if (k > cap_s) {
        int64_t c0 = b.cap_front, c1 = b.cap_front, c2 = b.cap_front, c3 = b.cap_front, c4 = b.cap_front;
        e = grow(&b.front[0], &c0, k, 1);
        if (e == cudaSuccess) e = grow(&b.front[1], &c1, k, 1);
        if (e == cudaSuccess) e = grow(&b.roots, &c2, k, 1);
        if (e == cudaSuccess) e = grow(&b.D[0], &c3, k, 2);
        if (e == cudaSuccess) e = grow(&b.D[1], &c4, k, 2);
        if (e != cudaSuccess) return e;
        b.cap_front = c0;
    }
    b.traversed = 0;
    b.levels_up = b.levels_down = 0;
    // counters: [0] frontier, [1] roots, [2] R_u, [3] spare
    e = cudaMemsetAsync(b.count, 0, 4 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    k_bf_seed<<<blocks(k), 256, 0, s>>>(S, k, n, b.mark, epoch, b.front[0], b.count, ds);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    b.launches += 1;
    unsigned c = 0;
    if ((e = read_count(b.count, &c, s)) != cudaSuccess) return e;
    // ---- Phase I
    int cur = 0;
    int64_t R_total = 0;
    while (c > 0) {
        if (R_total + c > b.cap_R) {  // keep what R_u holds so far
            int64_t cap = b.cap_R ? b.cap_R : 1024;
            while (cap < R_total + c) cap *= 2;
            int* q = nullptr;
            if ((e = cudaMalloc(&q, sizeof(int) * 2 * (size_t)cap)) != cudaSuccess) return e;
            if (R_total)
                e = cudaMemcpyAsync(q, b.R, sizeof(int) * 2 * (size_t)R_total, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) {
                cudaFree(q);
                return e;
            }
            cudaFree(b.R);
            b.R = q;
            b.cap_R = cap;
        }
        e = cudaMemsetAsync(b.count, 0, sizeof(unsigned), s);
        if (e != cudaSuccess) return e;
        k_bf_up<<<blocks(c), 256, 0, s>>>(b.front[cur], c, parent, b.mark, epoch, b.front[cur ^ 1],
                                          b.count, b.roots, b.count + 1, b.R, b.count + 2);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        b.launches += 1;
        b.levels_up++;
        unsigned h[3];
        e = cudaMemcpyAsync(h, b.count, 3 * sizeof(unsigned), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
        c = h[0];
        R_total = h[2];
        cur ^= 1;
    }
    b.traversed = R_total;
    unsigned n_roots = 0;
    if ((e = read_count(b.count + 1, &n_roots, s)) != cudaSuccess) return e;
    // ---- Response Distributor over R_u
    const unsigned lambda = (unsigned)R_total;
    // rho = 3 lambda buckets (Section 4.1), kept inside 31 bits
    const unsigned rho = lambda ? (unsigned)std::min<uint64_t>(3ull * lambda, 0x7fffffffull) : 1u;
    if (lambda > 0) {
        int64_t cs = b.cap_R2;
        if ((e = grow(&b.sorted, &cs, lambda, 2)) != cudaSuccess) return e;
        b.cap_R2 = cs;
        int64_t cb = b.cap_bucket, cc2 = b.cap_bucket;
        if ((e = grow(&b.bucket, &cb, (int64_t)rho + 1, 1)) != cudaSuccess) return e;
        if ((e = grow(&b.cursor, &cc2, (int64_t)rho + 1, 1)) != cudaSuccess) return e;
        b.cap_bucket = cb;
        int64_t csc = b.cap_scan;
        if ((e = grow(&b.scan, &csc, scan_scratch_ints((int64_t)rho + 1), 1)) != cudaSuccess) return e;
        b.cap_scan = csc;
        e = cudaMemsetAsync(b.bucket, 0, sizeof(int) * ((size_t)rho + 1), s);
        if (e != cudaSuccess) return e;
        k_rd_hist<<<blocks(lambda), 256, 0, s>>>(b.R, lambda, rho, b.bucket);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = exclusive_scan(b.bucket, (int64_t)rho + 1, b.scan, s)) != cudaSuccess) return e;
        e = cudaMemcpyAsync(b.cursor, b.bucket, sizeof(int) * (size_t)rho, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
        k_rd_scatter<<<blocks(lambda), 256, 0, s>>>(b.R, lambda, rho, b.cursor, b.sorted);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        b.launches += 3;
    }
    // ---- Phase II (nothing to do when every query node was a root)
    if (lambda > 0) {
        int64_t cw = b.cap_work;
        if ((e = grow(&b.work, &cw, b.cap_front + 1, 1)) != cudaSuccess) return e;
        b.cap_work = cw;
        int64_t csc = b.cap_scan;
        if ((e = grow(&b.scan, &csc, scan_scratch_ints(b.cap_front + 1), 1)) != cudaSuccess) return e;
        b.cap_scan = csc;
        k_bf_roots_to_d<<<blocks(n_roots), 256, 0, s>>>(b.roots, n_roots, b.D[0]);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        c = n_roots;
        cur = 0;
        while (c > 0) {
            k_bf_down_point<<<blocks((int64_t)c + 1), 256, 0, s>>>(b.D[cur], c, parent, b.bucket, rho, b.work);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            if ((e = exclusive_scan(b.work, (int64_t)c + 1, b.scan, s)) != cudaSuccess) return e;
            unsigned total = 0;
            if ((e = read_count(reinterpret_cast<const unsigned*>(b.work + c), &total, s)) != cudaSuccess) return e;
            e = cudaMemsetAsync(b.count + 3, 0, sizeof(unsigned), s);
            if (e != cudaSuccess) return e;
            if (total > 0) {
                k_bf_down_expand<<<blocks(total), 256, 0, s>>>(b.D[cur], c, b.work, total, b.sorted, b.bucket,
                                                                rho, b.D[cur ^ 1], b.count + 3);
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
            }
            b.launches += 3;
            b.levels_down++;
            if ((e = read_count(b.count + 3, &c, s)) != cudaSuccess) return e;
            cur ^= 1;
        }
    }
    if (res) {
        k_bf_gather<<<blocks(k), 256, 0, s>>>(S, k, n, parent, res);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        b.launches += 1;
    }
    return cudaSuccess;
}

cudaError_t bulk_find_query(BulkFindState& b, int* parent, int n, const int* pairs, int64_t k,
                            uint8_t* out, DevState* ds, cudaStream_t s) {
    int64_t cres = b.cap_res;
    cudaError_t e = grow(&b.res, &cres, 2 * k, 1);
    if (e != cudaSuccess) return e;
    b.cap_res = cres;
    e = bulk_find(b, parent, n, pairs, 2 * k, b.res, ds, s);
    if (e != cudaSuccess) return e;
    k_bf_answers<<<blocks(k), 256, 0, s>>>(b.res, k, out);
    b.launches += 1;
    return cudaGetLastError();
}

}  // namespace cc
