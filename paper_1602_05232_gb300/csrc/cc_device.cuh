// Device primitives of the union-find forest: find and hook.
//
// Forest invariant: parent[x] <= x for every x, with equality exactly at the
// roots. Hooks link the larger root under the smaller, and path halving and
// compression only repoint a node at one of its ancestors, so every write
// keeps the invariant. Consequences used throughout:
//  * every walk strictly decreases the id, so it ends within n steps (no
//    iteration limit is needed, and none can livelock);
//  * once a node stops being a root it never becomes one again, so only roots
//    are ever compare-and-swapped and only non-roots ever get plain stores;
//  * a value read late or early is still an ancestor: two endpoints that reach
//    the same node are connected, whatever else is happening.
#pragma once

#include <cstdint>

#include "cc_internal.cuh"

namespace cc {

__device__ __forceinline__ void flag(DevState* ds, unsigned bit) { atomicOr(&ds->status, bit); }

__device__ __forceinline__ bool in_range(int x, int n) { return (unsigned)x < (unsigned)n; }

// Alignment class of a pair array: 2 = 16-byte, 1 = 8-byte, 0 = 4-byte.
__device__ __forceinline__ int pair_vec_dev(const void* p) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    return (a % 16 == 0) ? 2 : (a % 8 == 0) ? 1 : 0;
}

// Root of x's tree, given p = parent[x] already read and p != x. Walks with
// path halving: each visited node is repointed at its grandparent, which
// roughly halves the path for later walks (the Section 5.1 idea of making
// later finds cheaper, done on the way up rather than in a second pass).
__device__ __forceinline__ int find_from(int* parent, int x, int p, DevState* ds) {
    while (true) {
        if (p > x) {  // broken invariant: stop rather than loop
            flag(ds, ST_CORRUPT);
            return x;
        }
        int gp = parent[p];
        if (gp == p) return p;
        parent[x] = gp;
        x = gp;
        p = parent[x];
        if (p == x) return x;
    }
}

__device__ __forceinline__ int find_halving(int* parent, int x, DevState* ds) {
    int p = parent[x];
    return p == x ? x : find_from(parent, x, p, ds);
}

// Join the trees of roots-or-former-roots ru and rv: the larger root becomes a
// child of the smaller one with a compare-and-swap that succeeds only while it
// is still a root. If another thread linked it first, continue from its new
// root. Each failed round strictly lowers max(ru, rv), so it ends. Returns 1
// if this call made the link, 0 if the two were already joined.
__device__ __forceinline__ int hook(int* parent, int ru, int rv, DevState* ds) {
    while (ru != rv) {
        int hi = ru > rv ? ru : rv;
        int lo = ru > rv ? rv : ru;
        int old = atomicCAS(parent + hi, hi, lo);
        if (old == hi) return 1;
        if (old > hi) {
            flag(ds, ST_CORRUPT);
            return 0;
        }
        int r = find_halving(parent, old, ds);
        if (hi == ru) ru = r; else rv = r;
    }
    return 0;
}

// The same join with atomicMin instead of a compare-and-swap: parent[hi] is
// lowered to lo (hi = the larger id). If hi was still a root, that is the
// link. If not, its parent `old` comes back. When old > lo this call has just
// moved hi's subtree from old's tree into lo's, and when old < lo it changed
// nothing; either way the loop goes on joining old and lo, from their current
// roots, which are both below hi -- so it ends, and old's tree is joined to
// lo's, which keeps every earlier connection. Pointers only ever decrease, so
// no cycle can form. A hook counts only a write at a root, so the number of
// trees drops by exactly the links it returns. Under contention (many edges
// of a minibatch on one hub root) every caller issues one atomic on the hub
// and repairs elsewhere, where the CAS version fails, walks and retries in
// rounds.
static __device__ __noinline__ int hook_min(int* parent, int ru, int rv, DevState* ds) {
    while (ru != rv) {
        const int hi = ru > rv ? ru : rv;
        const int lo = ru > rv ? rv : ru;
        const int old = atomicMin(parent + hi, lo);
        if (old == hi) return 1;
        if (old > hi) {
            flag(ds, ST_CORRUPT);
            return 0;
        }
        if (old == lo) return 0;
        ru = find_halving(parent, old, ds);
        rv = find_halving(parent, lo, ds);
    }
    return 0;
}

// hook or hook_min, chosen per launch.
__device__ __forceinline__ int hook_as(int* parent, int ru, int rv, DevState* ds, int minhook) {
    return minhook ? hook_min(parent, ru, rv, ds) : hook(parent, ru, rv, ds);
}

// The hooks of a whole warp, grouped by target. Must be called by all 32
// lanes together. Lane l joins roots-or-former-roots a[i], b[i] for every i
// with want[i]. In each round the lanes whose larger root `hi` is the same
// form a group (__match_any_sync): only one lane of the group -- the one
// with the smallest `lo` -- writes parent[hi], with a compare-and-swap
// (hook) or an atomicMin (hook_min), instead of every lane of the group
// contending for that word. Then:
//  - the write linked hi under lo_min: the leader is done, and every other
//    member joins its own lo with lo_min (hi is now in lo_min's tree);
//  - compare-and-swap failed (hi is no longer a root): the leader finds the
//    root r of hi's new parent once, and every member continues with
//    (r, its lo);
//  - atomicMin found hi under old < hi: the leader continues joining old
//    and lo_min (as hook_min does), every other member joins its lo with
//    lo_min.
// Every continuing pair has both ids below hi, so each lane's larger id
// strictly decreases from round to round and the loop ends. Returns the
// links this lane made (a write at a root counts once).
template <int E>
__device__ __forceinline__ int hook_warp(int* parent, const bool (&want0)[E], const int (&a0)[E],
                                         const int (&b0)[E], DevState* ds, int minhook) {
    const unsigned full = 0xffffffffu;
    const int lane = (int)(threadIdx.x & 31u);
    int made = 0;
#pragma unroll
    for (int i = 0; i < E; i++) {
        bool want = want0[i];
        int a = a0[i], b = b0[i];
        while (__any_sync(full, want)) {
            int hi = a > b ? a : b, lo = a > b ? b : a;
            if (want && hi == lo) want = false;
            const unsigned m = __match_any_sync(full, want ? hi : -1 - lane);
            if (!want) continue;
            const int lo_min = __reduce_min_sync(m, lo);
            const int leader = __ffs(__ballot_sync(m, lo == lo_min)) - 1;
            int old = 0;
            if (lane == leader)
                old = minhook ? atomicMin(parent + hi, lo_min) : atomicCAS(parent + hi, hi, lo_min);
            old = __shfl_sync(m, old, leader);
            if (old > hi) {  // broken invariant: stop rather than loop
                if (lane == leader) flag(ds, ST_CORRUPT);
                want = false;
            } else if (old == hi) {  // linked hi under lo_min
                if (lane == leader) {
                    made++;
                    want = false;
                } else {
                    a = lo;
                    b = lo_min;
                }
            } else if (minhook) {  // hi was already under old
                if (lane == leader) {
                    if (old == lo_min) {
                        want = false;
                    } else {
                        a = find_halving(parent, old, ds);
                        b = find_halving(parent, lo_min, ds);
                    }
                } else {
                    a = lo;
                    b = lo_min;
                }
            } else {  // compare-and-swap failed: hi is no longer a root
                int r = 0;
                if (lane == leader) r = find_halving(parent, old, ds);
                a = __shfl_sync(m, r, leader);
                b = lo;
            }
        }
    }
    return made;
}

// Walk W chains to their roots in lockstep with path splitting. Chain c is at
// node x[c] whose parent p[c] has been read; it is finished when p[c] >= x[c]
// (p == x: x is the root). Each round reads the grandparent of every
// unfinished chain -- independent loads, all in flight together -- then
// repoints the node at its grandparent and moves up one level. On exit x[c]
// is the root of chain c (or, with a broken invariant, where it stopped).
template <int W>
__device__ __forceinline__ void walk_split(int* parent, int (&x)[W], int (&p)[W], DevState* ds) {
    while (true) {
        int gp[W];
        bool any = false;
#pragma unroll
        for (int c = 0; c < W; c++) {
            gp[c] = p[c];
            if (p[c] < x[c]) {
                gp[c] = parent[p[c]];
                any = true;
            }
        }
        if (!any) break;
#pragma unroll
        for (int c = 0; c < W; c++) {
            if (p[c] < x[c]) {
                if (gp[c] == p[c]) {
                    x[c] = p[c];          // p is the root
                } else if (gp[c] > p[c]) {
                    flag(ds, ST_CORRUPT);
                    x[c] = p[c];
                    p[c] = x[c];
                } else {
                    parent[x[c]] = gp[c];  // splitting: skip a level
                    x[c] = p[c];
                    p[c] = gp[c];
                }
            }
        }
    }
}

// Largest-component filter (the large-component skip of Afforest: Sutton,
// Ben-Nun and Barak, IPDPS 2018). Bit x of `big` says that x was in the tree
// of one root R when the bitmap was last written (a full compression pass).
// Trees only ever merge, so two vertices whose bits are set stay connected
// whatever is linked afterwards: a query on them answers 1 and an edge
// between them joins nothing, without a read of the forest. The bitmap is
// n bits (8 MiB for 2^26 vertices), so it stays in L2 while the forest
// lines come and go.
__device__ __forceinline__ bool big_member(const unsigned* __restrict__ big, int x) {
    return (__ldg(big + (x >> 5)) >> (x & 31)) & 1u;
}

// The bitmap a kernel may use: `big` when the handle has one and it marks a
// tree (big_root >= 0), else none. Read after the kernel's wait for the one
// before it (the compression pass that wrote the bitmap).
__device__ __forceinline__ const unsigned* big_active(const unsigned* big, const DevState* ds) {
    return (big && ds->big_root >= 0) ? big : nullptr;
}

// Read-only walk to the root from x with p = parent[x] already read.
__device__ __forceinline__ int walk_root(const int* parent, int x, int p) {
    while (p < x) {
        x = p;
        p = parent[x];
    }
    return x;
}

// Load E pairs starting at pair index e0 of a flat u0 v0 u1 v1 ... array.
// vec: 2 = the array is 16-byte aligned, 1 = 8-byte, 0 = 4-byte. Pairs past k
// are left as (0, 0) and must be ignored by the caller. Streaming loads: each
// pair is read once, so it should not displace the forest from L2.
template <int E>
__device__ __forceinline__ void load_pairs(const int* __restrict__ a, int64_t e0, int64_t k,
                                           int vec, int (&u)[E], int (&v)[E]) {
    if (e0 + E <= k) {
        if (E % 2 == 0 && vec == 2) {
#pragma unroll
            for (int i = 0; i < E / 2; i++) {
                int4 q = __ldcs(reinterpret_cast<const int4*>(a + 2 * e0) + i);
                u[2 * i] = q.x; v[2 * i] = q.y; u[2 * i + 1] = q.z; v[2 * i + 1] = q.w;
            }
            return;
        }
        if (vec >= 1) {
#pragma unroll
            for (int i = 0; i < E; i++) {
                int2 q = __ldcs(reinterpret_cast<const int2*>(a + 2 * e0) + i);
                u[i] = q.x; v[i] = q.y;
            }
            return;
        }
    }
#pragma unroll
    for (int i = 0; i < E; i++) {
        if (e0 + i < k) {
            u[i] = __ldcs(a + 2 * (e0 + i));
            v[i] = __ldcs(a + 2 * (e0 + i) + 1);
        } else {
            u[i] = 0; v[i] = 0;
        }
    }
}

}  // namespace cc
