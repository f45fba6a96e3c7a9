// Appending to a device list whose length lives in one counter, from every
// thread of a block at once (stream compaction without a separate scan).
#pragma once

#include <cstdint>

namespace cc {

// The slot of this thread's item among the block's items, reserved with ONE
// atomicAdd per block on `count` (rather than one per warp): a list that
// grows by a million items per launch through a single counter otherwise
// queues tens of thousands of atomics on that one word. The warps' counts are
// scanned in shared memory by one thread, which takes the block's range.
// Every thread of the block must call it (it contains barriers); threads with
// has == false get a slot they must not use. A warp reads and writes only its
// own count, the next call's write coming after that call's warp-wide ballot
// (which all lanes reach only after their reads), and the scan and the base
// are rewritten only after the next call's first barrier, so consecutive
// calls need no barrier between them.
__device__ __forceinline__ unsigned block_slot(bool has, unsigned* __restrict__ count) {
    __shared__ unsigned warp_base[32];
    __shared__ unsigned block_base;
    const unsigned mask = __ballot_sync(0xffffffffu, has);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) warp_base[w] = __popc(mask);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned total = 0;
        const int warps = (blockDim.x + 31) >> 5;
        for (int j = 0; j < warps; j++) {
            const unsigned c = warp_base[j];
            warp_base[j] = total;
            total += c;
        }
        block_base = total ? atomicAdd(count, total) : 0u;
    }
    __syncthreads();
    return block_base + warp_base[w] + __popc(mask & ((1u << lane) - 1));
}

__device__ __forceinline__ void append1_block(bool has, int v, int* __restrict__ out,
                                              unsigned* __restrict__ count) {
    const unsigned slot = block_slot(has, count);
    if (has) out[slot] = v;
}

__device__ __forceinline__ void append2_block(bool has, int a, int b, int* __restrict__ out,
                                              unsigned* __restrict__ count) {
    const unsigned slot = block_slot(has, count);
    if (has) {
        out[2 * (size_t)slot] = a;
        out[2 * (size_t)slot + 1] = b;
    }
}

}  // namespace cc
