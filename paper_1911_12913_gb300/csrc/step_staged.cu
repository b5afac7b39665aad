// Staged T2S2-FDLBM step for any boundary combination (periodic or walled
// axes, Eq. 3.10 walls): the stages of Sec. 2D run as separate kernels through
// three scratch fields P, Q, S, one thread per node (stage bodies in
// staged_nodes.cuh).  This path serves the wall-bounded cases (channel,
// cavity), T2S2-FDLBM2 and grids too small for the fused kernel's halo.
//
// Launch order per step: prepare (all nodes), [scheme 2 with walls: Eq. 3.10
// on P], star (interior), Eq. 3.10 on S, update (interior), Eq. 3.10 on the
// new state.
#include "staged_nodes.cuh"

namespace fdlbm {
namespace {

template <class R, bool FORCE>
__global__ void k_prepare(const StepArgs<R> a)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x < a.nx && y < a.ny) prepare_node<R, FORCE>(a, x, y);
}

template <class R, bool FORCE>
__global__ void k_star(const StepArgs<R> a)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x < a.nx && y < a.ny) star_node<R, FORCE>(a, x, y);
}

template <class R>
__global__ void k_update(const StepArgs<R> a)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x < a.nx && y < a.ny) update_node<R>(a, x, y);
}

template <class R, bool FORCE>
__global__ void k_wall_nee(const StepArgs<R> a, R *fld, R shift)
{
    wall_node<R, FORCE>(a, fld, shift, blockIdx.x * blockDim.x + threadIdx.x);
}

template <class R, bool FORCE>
cudaError_t run(const StepArgs<R> &a, cudaStream_t s)
{
    const dim3 blk(32, 8);
    const dim3 grd((a.nx + 31) / 32, (a.ny + 7) / 8);
    const int nwall = wall_count(a);
    const bool walls = nwall > 0;
    k_prepare<R, FORCE><<<grd, blk, 0, s>>>(a);
    if (walls && a.scheme == FDLBM_SCHEME_T2S2_2)
        k_wall_nee<R, false><<<(nwall + 127) / 128, 128, 0, s>>>(a, a.P, R(0));
    k_star<R, FORCE><<<grd, blk, 0, s>>>(a);
    if (walls) k_wall_nee<R, false><<<(nwall + 127) / 128, 128, 0, s>>>(a, a.S, R(0));
    k_update<R><<<grd, blk, 0, s>>>(a);
    if (walls) k_wall_nee<R, FORCE><<<(nwall + 127) / 128, 128, 0, s>>>(a, a.gout, a.c.half_dt);
    return cudaGetLastError();
}

}  // namespace

template <class R>
cudaError_t launch_staged(const StepArgs<R> &a, cudaStream_t s)
{
    return a.force ? run<R, true>(a, s) : run<R, false>(a, s);
}

template cudaError_t launch_staged<float>(const StepArgs<float> &, cudaStream_t);
template cudaError_t launch_staged<double>(const StepArgs<double> &, cudaStream_t);

}  // namespace fdlbm
