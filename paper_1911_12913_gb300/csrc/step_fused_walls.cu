// Fused T2S2-FDLBM1 step with walls, one launch per step: the sweep of
// walls_sweep.cuh in blocks of 128 columns (120 outputs), for single grids,
// batches and the persistent batch.
#include <cstdint>

#include <algorithm>

#include "grid_barrier.cuh"
#include "internal.h"
#include "walls_sweep.cuh"

namespace fdlbm {
namespace {

using walls_sweep::kHalo;
constexpr int NT = 128;
template <class R>
using Smem = walls_sweep::Smem<R, NT>;

// Offset of the argument block after the rings in the persistent batch kernel's
// dynamic shared memory, and that memory's size.
template <class R>
constexpr size_t kArgOffset = (sizeof(Smem<R>) + 15) / 16 * 16;
template <class R>
constexpr size_t kPersistSmem = kArgOffset<R> + sizeof(StepArgs<R>);

// PF (metric and force a row ahead): the single-grid and batched FP32 sweeps,
// whose registers allow it.
template <class R, bool FORCE, bool PF = sizeof(R) == 4, bool TAIL = false>
__device__ __forceinline__ void sweep_tile(const StepArgs<R> &a, Smem<R> &sm, int x0, int y0)
{
    walls_sweep::sweep_tile<R, FORCE, NT, PF, TAIL>(a, sm, x0, a.nx, y0, min(y0 + a.rows, a.ny));
}

template <class R, bool FORCE>
__global__ void __launch_bounds__(NT, sizeof(R) == 4 ? 3 : 2) k_step_fused_walls(const StepArgs<R> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<R> &sm = *reinterpret_cast<Smem<R> *>(smem_raw);
    const int y0 = blockIdx.y * a.rows;
    if (y0 >= a.ny) return;  // uniform over the block
    sweep_tile<R, FORCE>(a, sm, blockIdx.x * (NT - 2 * kHalo), y0);
}

// Batched: block b is tile (b - blk_start[c]) of case c = blk_case[b], with
// strips[c] strips per row of tiles; the case's arguments (its own tile height
// in .rows) are copied into shared memory first.
template <class R>
__global__ void __launch_bounds__(NT, sizeof(R) == 4 ? 3 : 2)
    kb_step_fused_walls(const StepArgs<R> *cases, const int *blk_case, const int *blk_start,
                        const int *strips, int blk_off)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<R> &sm = *reinterpret_cast<Smem<R> *>(smem_raw);
    __shared__ __align__(16) unsigned char abuf[sizeof(StepArgs<R>)];
    static_assert(sizeof(StepArgs<R>) % 4 == 0, "argument block is copied as 32-bit words");
    const int bid = blk_off + blockIdx.x;
    const int c = blk_case[bid];
    {
        const int *src = reinterpret_cast<const int *>(cases + c);
        int *dst = reinterpret_cast<int *>(abuf);
        for (int k = threadIdx.x; k < (int)(sizeof(StepArgs<R>) / 4); k += blockDim.x) dst[k] = src[k];
    }
    __syncthreads();
    const StepArgs<R> &a = *reinterpret_cast<const StepArgs<R> *>(abuf);
    const int lb = bid - blk_start[c], ns = strips[c];
    const int y0 = (lb / ns) * a.rows;
    if (y0 >= a.ny) return;  // uniform over the block
    sweep_tile<R, true>(a, sm, (lb % ns) * (NT - 2 * kHalo), y0);
}

// Persistent batched: all tiles of all cases for nsteps steps in one
// cooperative launch (all blocks resident).  Within a step the blocks fetch
// tiles from a global counter, as the hardware would hand out the blocks of
// one launch; one grid barrier separates consecutive steps, since a step reads
// the state the previous one wrote around its tile.  Steps alternate between
// two counters: block 0 clears the next step's counter at the start of a step,
// when every block has passed the barrier after that counter's last use.  A
// barrier that times out sets every case's error flag and the block leaves;
// the others then time out at their next barrier.
template <class R>
__global__ void __launch_bounds__(NT, sizeof(R) == 4 ? 3 : 2)
    kp_step_fused_walls(const BatchTables t, GridBarrier *bar, int parity0, int nsteps,
                        unsigned spin_limit)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<R> &sm = *reinterpret_cast<Smem<R> *>(smem_raw);
    unsigned char *abuf = smem_raw + kArgOffset<R>;
    static_assert(sizeof(StepArgs<R>) % 4 == 0, "argument block is copied as 32-bit words");
    __shared__ int tile_s;
    unsigned gen = 0;
    for (int k = 0; k < nsteps; ++k) {
        const StepArgs<R> *cases = static_cast<const StepArgs<R> *>(t.args[(parity0 + k) & 1]);
        unsigned *work = &bar->work[k & 1];
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(&bar->work[(k + 1) & 1], 0u);
        for (;;) {
            __syncthreads();  // the previous tile is done with the argument block and tile_s
            if (threadIdx.x == 0) tile_s = (int)atomicAdd(work, 1u);
            __syncthreads();
            const int b = tile_s;
            if (b >= t.total_blocks) break;  // uniform over the block
            const int c = t.blk_case[b];
            {
                const int *src = reinterpret_cast<const int *>(cases + c);
                int *dst = reinterpret_cast<int *>(abuf);
                for (int q = threadIdx.x; q < (int)(sizeof(StepArgs<R>) / 4); q += blockDim.x)
                    dst[q] = src[q];
            }
            __syncthreads();
            const StepArgs<R> &a = *reinterpret_cast<const StepArgs<R> *>(abuf);
            const int lb = b - t.blk_start[c], ns = t.tiles_x[c];
            const int y0 = (lb / ns) * a.rows;
            if (y0 < a.ny)  // uniform over the block
                sweep_tile<R, true, false, true>(a, sm, (lb % ns) * (NT - 2 * kHalo), y0);
        }
        if (!grid_barrier(bar, gen, spin_limit)) {
            if (threadIdx.x == 0) {
                const StepArgs<R> *c0 = static_cast<const StepArgs<R> *>(t.args[0]);
                for (int c = 0; c < t.ncases; ++c) atomicOr(c0[c].err, 2);
            }
            return;
        }
    }
}

template <class R, bool FORCE>
cudaError_t launch_t(const StepArgs<R> &a, cudaStream_t s)
{
    constexpr int W = NT - 2 * kHalo;
    constexpr size_t smem = sizeof(Smem<R>);
    cudaError_t e = cudaFuncSetAttribute(k_step_fused_walls<R, FORCE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((a.nx + W - 1) / W, (a.ny + a.rows - 1) / a.rows);
    k_step_fused_walls<R, FORCE><<<grid, NT, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

template <class R>
cudaError_t launch_fused_walls(const StepArgs<R> &a, cudaStream_t s)
{
    return a.force ? launch_t<R, true>(a, s) : launch_t<R, false>(a, s);
}

template <class R>
int fused_walls_blocks_per_sm()
{
    int n = 0;
    constexpr size_t smem = sizeof(Smem<R>);
    cudaFuncSetAttribute(k_step_fused_walls<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_fused_walls<R, false>, NT, smem) !=
        cudaSuccess)
        return 0;
    return n;
}

// One step of T2S2-FDLBM1 cases of a batch on the walls sweep (tiles
// [blk_off, blk_off + nblocks) of its tables): one launch.
template <class R>
cudaError_t launch_batched_fused(const BatchTables &t, int parity, int blk_off, int nblocks,
                                 cudaStream_t s)
{
    if (nblocks <= 0) return cudaSuccess;
    constexpr size_t smem = sizeof(Smem<R>);
    cudaError_t e = cudaFuncSetAttribute(kb_step_fused_walls<R>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kb_step_fused_walls<R><<<nblocks, NT, smem, s>>>(
        static_cast<const StepArgs<R> *>(t.args[parity]), t.blk_case, t.blk_start, t.tiles_x, blk_off);
    return cudaGetLastError();
}

int fused_tile_width_walls() { return NT - 2 * kHalo; }

template <class R>
int persistent_fused_blocks_per_sm()
{
    int n = 0;
    constexpr size_t smem = kPersistSmem<R>;
    cudaFuncSetAttribute(kp_step_fused_walls<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kp_step_fused_walls<R>, NT, smem) !=
        cudaSuccess)
        return 0;
    return n;
}

// Zero the barrier, then one cooperative launch of nsteps steps of every case
// (the tables of the fused batch).  `bar` is device memory of
// persistent_barrier_bytes() bytes owned by the caller.
template <class R>
cudaError_t launch_persistent_fused(const BatchTables &t, void *bar, int parity0, int nsteps,
                                    cudaStream_t s, unsigned spin_limit)
{
    if (nsteps <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    constexpr size_t smem = kPersistSmem<R>;
    e = cudaFuncSetAttribute(kp_step_fused_walls<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    const int per_sm = persistent_fused_blocks_per_sm<R>();
    if (per_sm <= 0) return cudaErrorInvalidConfiguration;
    const int grid = std::max(1, std::min(t.total_blocks, per_sm * sms));
    e = cudaMemsetAsync(bar, 0, sizeof(GridBarrier), s);
    if (e != cudaSuccess) return e;
    BatchTables tt = t;
    GridBarrier *gb = static_cast<GridBarrier *>(bar);
    void *params[] = {&tt, &gb, &parity0, &nsteps, &spin_limit};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(kp_step_fused_walls<R>),
                                       dim3(grid), dim3(NT), params, smem, s);
}

template int persistent_fused_blocks_per_sm<float>();
template int persistent_fused_blocks_per_sm<double>();
template cudaError_t launch_persistent_fused<float>(const BatchTables &, void *, int, int,
                                                    cudaStream_t, unsigned);
template cudaError_t launch_persistent_fused<double>(const BatchTables &, void *, int, int,
                                                     cudaStream_t, unsigned);

template cudaError_t launch_batched_fused<float>(const BatchTables &, int, int, int, cudaStream_t);
template cudaError_t launch_batched_fused<double>(const BatchTables &, int, int, int, cudaStream_t);
template cudaError_t launch_fused_walls<float>(const StepArgs<float> &, cudaStream_t);
template cudaError_t launch_fused_walls<double>(const StepArgs<double> &, cudaStream_t);
template int fused_walls_blocks_per_sm<float>();
template int fused_walls_blocks_per_sm<double>();

}  // namespace fdlbm
