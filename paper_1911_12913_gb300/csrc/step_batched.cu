// Batched staged step: many independent cases (uneven sizes, walls or not,
// force or not) advanced by one launch per stage for all cases together.
//
// Node kernels use a flat 1-D grid over the tiles of every case: block b
// belongs to case blk_case[b] and is tile (b - blk_start[c]) of that case, in
// row-major tile order with tiles_x[c] tiles per row.  The block shape is a
// launch parameter (chosen by the autotuner).  Wall kernels use a flat index
// over the wall nodes of every case (prefix sums in wall_start).  The stage
// bodies are those of the single-case staged path (staged_nodes.cuh).
#include "staged_nodes.cuh"

namespace fdlbm {
namespace {

// Copy one case's arguments into shared memory with all threads.
template <class R>
__device__ __forceinline__ void load_case(StepArgs<R> &dst, const StepArgs<R> *src)
{
    static_assert(sizeof(StepArgs<R>) % 4 == 0, "argument block is copied as 32-bit words");
    const int *s = reinterpret_cast<const int *>(src);
    int *d = reinterpret_cast<int *>(&dst);
    constexpr int nw = (int)(sizeof(StepArgs<R>) / 4);
    for (int k = threadIdx.y * blockDim.x + threadIdx.x; k < nw; k += blockDim.x * blockDim.y)
        d[k] = s[k];
    __syncthreads();
}

template <class R, int STAGE>
__global__ void kb_nodes(const StepArgs<R> *cases, const int *blk_case, const int *blk_start,
                         const int *tiles_x)
{
    __shared__ __align__(16) unsigned char buf[sizeof(StepArgs<R>)];
    StepArgs<R> &a = *reinterpret_cast<StepArgs<R> *>(buf);
    const int c = blk_case[blockIdx.x];
    load_case(a, cases + c);
    const int lb = blockIdx.x - blk_start[c], tx = tiles_x[c];
    const int x = (lb % tx) * blockDim.x + threadIdx.x;
    const int y = (lb / tx) * blockDim.y + threadIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    if (STAGE == 0) prepare_node<R, true>(a, x, y);
    else if (STAGE == 1) star_node<R, true>(a, x, y);
    else update_node<R>(a, x, y);
}

// WHICH: 0 = f* (S, shift 0), 1 = new state (shift dt/2), 2 = physical f^n
// (P, shift 0; T2S2-FDLBM2 cases only).
template <class R, int WHICH>
__global__ void kb_walls(const StepArgs<R> *cases, const int *wall_start, int ncases, int total)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= total) return;
    int lo = 0, hi = ncases - 1;  // last case whose first wall node is <= k
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (wall_start[mid] <= k) lo = mid;
        else hi = mid - 1;
    }
    const StepArgs<R> &a = cases[lo];
    if (WHICH == 2 && a.scheme != FDLBM_SCHEME_T2S2_2) return;
    R *fld = WHICH == 0 ? a.S : (WHICH == 1 ? a.gout : a.P);
    const R shift = WHICH == 1 ? a.c.half_dt : R(0);
    wall_node<R, WHICH == 1>(a, fld, shift, k - wall_start[lo]);
}

}  // namespace

template <class R>
cudaError_t launch_batched(const BatchTables &t, int parity, dim3 blk, cudaStream_t s)
{
    const StepArgs<R> *cases = static_cast<const StepArgs<R> *>(t.args[parity]);
    const int nwb = (t.total_wall + 127) / 128;
    kb_nodes<R, 0><<<t.total_blocks, blk, 0, s>>>(cases, t.blk_case, t.blk_start, t.tiles_x);
    if (t.total_wall > 0 && t.any_scheme2)
        kb_walls<R, 2><<<nwb, 128, 0, s>>>(cases, t.wall_start, t.ncases, t.total_wall);
    kb_nodes<R, 1><<<t.total_blocks, blk, 0, s>>>(cases, t.blk_case, t.blk_start, t.tiles_x);
    if (t.total_wall > 0) kb_walls<R, 0><<<nwb, 128, 0, s>>>(cases, t.wall_start, t.ncases, t.total_wall);
    kb_nodes<R, 2><<<t.total_blocks, blk, 0, s>>>(cases, t.blk_case, t.blk_start, t.tiles_x);
    if (t.total_wall > 0) kb_walls<R, 1><<<nwb, 128, 0, s>>>(cases, t.wall_start, t.ncases, t.total_wall);
    return cudaGetLastError();
}

template cudaError_t launch_batched<float>(const BatchTables &, int, dim3, cudaStream_t);
template cudaError_t launch_batched<double>(const BatchTables &, int, dim3, cudaStream_t);

}  // namespace fdlbm
