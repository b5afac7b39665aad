// Grid-wide barrier for cooperative launches, with bounded waits.
//
// A generation counter: thread 0 of every block makes its block's writes
// visible (fence), arrives on a global counter, and the last arriver resets the
// counter and publishes the next generation; the others wait for it.  The
// reset comes before the publication, so no block can arrive at the next
// barrier before the counter is back to zero.  Every wait gives up after
// `limit` polls and reports it, so a launch always ends.
#pragma once

namespace fdlbm {
namespace {

struct GridBarrier {
    unsigned count, gen;
    unsigned work[2];  // tile counters of even and odd steps (dynamic tile fetch)
};

__device__ __forceinline__ unsigned load_volatile(const unsigned *p)
{
    return *reinterpret_cast<const volatile unsigned *>(p);
}

// Block-uniform result: false when this block gave up waiting, after `limit`
// polls (the last block to arrive never waits).
__device__ bool grid_barrier(GridBarrier *bar, unsigned &gen, unsigned limit)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        int ok = 1;
        const unsigned target = gen + 1u;
        __threadfence();
        if (atomicAdd(&bar->count, 1u) + 1u == gridDim.x) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicExch(&bar->gen, target);
        } else {
            for (unsigned k = 0; load_volatile(&bar->gen) != target; ++k) {
                if (k >= limit) {
                    ok = 0;
                    break;
                }
                if (k > 32) __nanosleep(64);
            }
        }
        __threadfence();
        gen = target;
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

}  // namespace
}  // namespace fdlbm
