// Bounded grid-wide barrier for cooperative launches (all blocks resident).
//
// bar[0] is a 64-bit arrival counter that only grows: each block adds one per
// barrier (after a fence that publishes its writes), and barrier j of a launch
// is passed when the counter reaches base + j * gridDim.x, where base = bar[1]
// is the counter's value when the launch starts.  Once every block has read
// bar[1] (after the launch's first barrier), block 0 advances it by the
// launch's total arrivals, so the next launch on the same stream starts from
// there.  A wait gives up after `limit` ns of device time (2 s unless the owner
// sets another bound), records kErrTimeout in *err and reports failure; the
// owner then resets both words before reuse.
#pragma once

#include "ms_internal.h"

namespace msgb {

__device__ __forceinline__ unsigned long long gs_now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Returns false (for every thread of the block) when the wait ran out.
__device__ __forceinline__ bool grid_wait(unsigned long long *cnt, unsigned long long target, int *err,
                                          unsigned long long limit) {
    __shared__ int s_fail;
    __syncthreads();
    if (threadIdx.x == 0) {
        s_fail = 0;
        __threadfence();
        atomicAdd(cnt, 1ull);
        volatile unsigned long long *c = cnt;
        unsigned long long t0 = 0;
        int spins = 0;
        while (*c < target) {
            if ((++spins & 63) == 0) {
                const unsigned long long now = gs_now_ns();
                if (t0 == 0) t0 = now;
                else if (now - t0 > limit) {
                    atomicOr(err, kErrTimeout);
                    s_fail = 1;
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return s_fail == 0;
}

// Barrier j (1-based) of a launch that passes `total` barriers in all.
struct GridSync {
    unsigned long long *bar;
    unsigned long long base;
    int *err;
    unsigned long long limit;
    int passed;

    __device__ __forceinline__ void begin(unsigned long long *b, int *e, unsigned long long lim = kDefaultWaitNs) {
        bar = b;
        err = e;
        limit = lim;
        base = __ldcg(&b[1]);
        passed = 0;
    }
    __device__ __forceinline__ bool sync(int total) {
        ++passed;
        if (!grid_wait(bar, base + (unsigned long long)passed * gridDim.x, err, limit)) return false;
        if (passed == 1 && blockIdx.x == 0 && threadIdx.x == 0)   // every block has read bar[1]
            bar[1] = base + (unsigned long long)total * gridDim.x;
        return true;
    }
};

}  // namespace msgb
