// Persistent staged T2S2-FDLBM stepping (the batched mode's opt-in persistent
// mode): one cooperative launch advances any number of independent cases
// (uneven sizes, walls or not, force or not, both schemes) by any number of
// steps.  One kernel holds every stage, so its register allocation is that of
// the largest stage and every stage runs at that stage's occupancy; on the
// 64-case sweep the per-stage launches of step_batched.cu are faster, and
// they are the default.
//
// The stages of a step are those of the staged path (staged_nodes.cuh):
//   prepare (all nodes) | [Eq. 3.10 on P, scheme 2] | star (interior) |
//   Eq. 3.10 on S | update (interior) | Eq. 3.10 on the new state
// Each stage loops over the node tiles of every case (tile b belongs to case
// blk_case[b], tiles row-major within a case; each block takes a contiguous
// range) or, grid-stride, over the wall nodes of every case (prefix sums in
// wall_start), and consecutive stages are separated by a grid-wide barrier.  The blocks of a
// cooperative launch are all resident, so they can wait on one another.
//
// The grid barrier is a generation counter: thread 0 of every block makes its
// block's writes visible (fence), arrives on a global counter, and the last
// arriver resets the counter and publishes the next generation; the others
// wait for it.  Every wait is bounded: a block that waits longer than its poll
// limit (by default 2^24 polls, well over a second with the sleeps) records the
// error flag of every case and leaves, and the blocks still running then time
// out at their next barrier, so the launch always ends.  A limit of 0 makes
// every block but the last to arrive give up at the first barrier: a way to
// exercise this path without a fault (fdlbm_batch_set_spin_limit).
#include <algorithm>

#include <cuda_runtime.h>

#include "grid_barrier.cuh"
#include "staged_nodes.cuh"

namespace fdlbm {
namespace {

struct PersistArgs {
    BatchTables t;
    GridBarrier *bar;
    int parity0;  // ping-pong parity of the first step
    int nsteps;
    unsigned spin_limit;  // polls before a block gives up at a grid barrier
};

// Copy one case's arguments into shared memory with all threads.
template <class R>
__device__ __forceinline__ void load_case(StepArgs<R> &dst, const StepArgs<R> *src)
{
    static_assert(sizeof(StepArgs<R>) % 4 == 0, "argument block is copied as 32-bit words");
    const int *s = reinterpret_cast<const int *>(src);
    int *d = reinterpret_cast<int *>(&dst);
    constexpr int nw = (int)(sizeof(StepArgs<R>) / 4);
    __syncthreads();  // the previous tile's readers are done with dst
    for (int k = threadIdx.y * blockDim.x + threadIdx.x; k < nw; k += blockDim.x * blockDim.y)
        d[k] = s[k];
    __syncthreads();
}

// Last case whose prefix value is <= k.
__device__ __forceinline__ int find_case(const int *start, int ncases, int k)
{
    int lo = 0, hi = ncases - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (start[mid] <= k) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Block b takes the contiguous tiles [b T / G, (b + 1) T / G) of the T tiles of
// all cases (G blocks), so that consecutive tiles mostly share a case and the
// case's arguments are copied only when it changes.
template <class R, int STAGE>
__device__ void node_stage(const BatchTables &t, const StepArgs<R> *cases, StepArgs<R> &a)
{
    const long long T = t.total_blocks;
    const int b0 = (int)(T * blockIdx.x / gridDim.x), b1 = (int)(T * (blockIdx.x + 1) / gridDim.x);
    int loaded = -1;
    for (int b = b0; b < b1; ++b) {
        const int c = t.blk_case[b];
        if (c != loaded) {  // uniform over the block
            load_case(a, cases + c);
            loaded = c;
        }
        const int lb = b - t.blk_start[c], tx = t.tiles_x[c];
        const int x = (lb % tx) * blockDim.x + threadIdx.x;
        const int y = (lb / tx) * blockDim.y + threadIdx.y;
        if (x < a.nx && y < a.ny) {
            if (STAGE == 0) prepare_node<R, true>(a, x, y);
            else if (STAGE == 1) star_node<R, true>(a, x, y);
            else update_node<R>(a, x, y);
        }
    }
}

// WHICH: 0 = f* (S, shift 0), 1 = new state (shift dt/2), 2 = physical f^n
// (P, shift 0; T2S2-FDLBM2 cases only).
template <class R, int WHICH>
__device__ void wall_stage(const BatchTables &t, const StepArgs<R> *cases)
{
    const int nthr = blockDim.x * blockDim.y;
    const int stride = gridDim.x * nthr;
    for (int k = blockIdx.x * nthr + threadIdx.y * blockDim.x + threadIdx.x; k < t.total_wall;
         k += stride) {
        const int c = find_case(t.wall_start, t.ncases, k);
        const StepArgs<R> &a = cases[c];
        if (WHICH == 2 && a.scheme != FDLBM_SCHEME_T2S2_2) continue;
        R *fld = WHICH == 0 ? a.S : (WHICH == 1 ? a.gout : a.P);
        const R shift = WHICH == 1 ? a.c.half_dt : R(0);
        wall_node<R, WHICH == 1>(a, fld, shift, k - t.wall_start[c]);
    }
}

template <class R>
__global__ void k_persist(const PersistArgs p)
{
    __shared__ __align__(16) unsigned char buf[sizeof(StepArgs<R>)];
    StepArgs<R> &a = *reinterpret_cast<StepArgs<R> *>(buf);
    const BatchTables &t = p.t;
    unsigned gen = 0;
    for (int k = 0; k < p.nsteps; ++k) {
        const StepArgs<R> *cases = static_cast<const StepArgs<R> *>(t.args[(p.parity0 + k) & 1]);
        node_stage<R, 0>(t, cases, a);
        if (!grid_barrier(p.bar, gen, p.spin_limit)) goto timeout;
        if (t.total_wall > 0 && t.any_scheme2) {
            wall_stage<R, 2>(t, cases);
            if (!grid_barrier(p.bar, gen, p.spin_limit)) goto timeout;
        }
        node_stage<R, 1>(t, cases, a);
        if (!grid_barrier(p.bar, gen, p.spin_limit)) goto timeout;
        if (t.total_wall > 0) {
            wall_stage<R, 0>(t, cases);
            if (!grid_barrier(p.bar, gen, p.spin_limit)) goto timeout;
        }
        node_stage<R, 2>(t, cases, a);
        if (!grid_barrier(p.bar, gen, p.spin_limit)) goto timeout;
        if (t.total_wall > 0) {
            wall_stage<R, 1>(t, cases);
            if (!grid_barrier(p.bar, gen, p.spin_limit)) goto timeout;
        }
    }
    return;
timeout:
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const StepArgs<R> *cases = static_cast<const StepArgs<R> *>(t.args[0]);
        for (int c = 0; c < t.ncases; ++c) atomicOr(cases[c].err, 2);
    }
}

}  // namespace

template <class R>
int persistent_blocks_per_sm(dim3 blk)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_persist<R>, (int)(blk.x * blk.y * blk.z),
                                                      0) != cudaSuccess)
        return 0;
    return n;
}

// Zero the barrier, then one cooperative launch of nsteps steps.  `bar` is two
// unsigned words of device memory owned by the caller; spin_limit bounds every
// wait at a grid barrier (in polls).
template <class R>
cudaError_t launch_persistent(const BatchTables &t, void *bar, int parity0, int nsteps, dim3 blk,
                              cudaStream_t s, unsigned spin_limit)
{
    if (nsteps <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int per_sm = persistent_blocks_per_sm<R>(blk);
    if (per_sm <= 0) return cudaErrorInvalidConfiguration;
    const int grid = std::max(1, std::min(t.total_blocks, per_sm * sms));
    e = cudaMemsetAsync(bar, 0, sizeof(GridBarrier), s);
    if (e != cudaSuccess) return e;
    PersistArgs p{t, static_cast<GridBarrier *>(bar), parity0, nsteps, spin_limit};
    void *params[] = {&p};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(k_persist<R>), dim3(grid), blk,
                                       params, 0, s);
}

size_t persistent_barrier_bytes() { return sizeof(GridBarrier); }

template int persistent_blocks_per_sm<float>(dim3);
template int persistent_blocks_per_sm<double>(dim3);
template cudaError_t launch_persistent<float>(const BatchTables &, void *, int, int, dim3, cudaStream_t,
                                              unsigned);
template cudaError_t launch_persistent<double>(const BatchTables &, void *, int, int, dim3,
                                               cudaStream_t, unsigned);

}  // namespace fdlbm
