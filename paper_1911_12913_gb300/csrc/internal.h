// Host-side state of a handle and the launchers each translation unit provides.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <string>
#include <vector>

#include "fdlbm.h"
#include "lattice.cuh"

namespace fdlbm {

// Everything a step kernel needs, passed by value.
template <class R>
struct StepArgs {
    const R *gin;        // [9][ny][pitch] deviations at t_n
    R *gout;             // [9][ny][pitch] deviations at t_{n+1}
    const R *mx, *my;    // metrics d zeta/dx (nx), d mu/dy (ny)
    const R *force;      // [2][ny][pitch] or nullptr
    int nx, ny, pitch;
    size_t plane;        // ny * pitch
    int bc_x, bc_y;      // FDLBM_PERIODIC / FDLBM_WALL
    R wall_u[4][2];
    Coeffs<R> c;
    Stencil<R> st;       // mixed weights
    Stencil<R> stc;      // central-only weights (next to walls)
    int rows;            // fused kernel: rows per CTA
    int *err;            // kernel-side failure flag (bounded waits that gave up)
    int scheme;          // FDLBM_SCHEME_T2S2_1 / _2 (the second only on the staged path)
    // staged path scratch, [9][ny][pitch] each
    R *P, *Q, *S;
};

// Device tables of a batch (step_batched.cu, step_persist.cu).
struct BatchTables {
    const void *args[2];   // StepArgs<R>[ncases] for even / odd steps (ping-pong)
    const int *blk_case;   // [total_blocks] case of each node tile
    const int *blk_start;  // [ncases] first node tile of each case
    const int *tiles_x;    // [ncases]
    const int *wall_start; // [ncases]
    int ncases, total_blocks, total_wall;
    bool any_scheme2;
    int blocks_s1;         // fused tables: tiles of T2S2-FDLBM1 cases, which come first
};

// Tensor maps (CUtensorMap, 128 bytes each) of the warp-tile kernel: the
// ping-pong state buffers with boxes of 64 and 4 columns, and the force field.
struct WarpMaps {
    alignas(64) unsigned char state[2][128];
    alignas(64) unsigned char side[2][128];
    alignas(64) unsigned char force[128];
    alignas(64) unsigned char force_side[128];
    bool has_force = false;
};

struct Layout {
    size_t state[2], mx, my, mxd, myd, force, P, Q, S, uprev, partials, red, err, staging;
    size_t staging_elems, total;
    int nblocks_red;
};

}  // namespace fdlbm

struct fdlbm_ctx {
    int nx = 0, ny = 0, pitch = 0;
    size_t plane = 0;
    int bc_x = 0, bc_y = 0;
    double wall_u[4][2] = {};
    int precision = FDLBM_FP64;
    int scheme = FDLBM_SCHEME_T2S2_1;
    int incomp = 0;                      // FDLBM_EQ_INCOMPRESSIBLE
    double nu = 0, tau = 0, dt = 0, cfl = 0, beta = 0, A = 0.5, rho0 = 1;
    int has_force = 0;
    int path = FDLBM_PATH_FUSED;
    int variant = FDLBM_VARIANT_SCALAR;  // fused kernel actually used
    bool in_batch = false;               // owned by a batch: stepped by fdlbm_batch_step
    bool adjoint = false;                // scratch for the adjoint step reserved
    int graph_steps = 0;                 // steps per replayed CUDA graph (even), 0 = none
    fdlbm::WarpMaps wmaps{};             // tensor maps of the warp-tile kernel
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int rows = 64;
    cudaStream_t stream = nullptr;
    char *ws = nullptr;
    size_t ws_bytes = 0;
    bool owns_ws = false;
    int device = 0;
    fdlbm::Layout lay{};
    int cur = 0;
    bool have_uprev = false;
    long long steps = 0;
    std::string err;
    std::string desc;
};

namespace fdlbm {

size_t real_size(int precision);
fdlbm_status handle_prepare(const fdlbm_grid *g, const fdlbm_metrics *metrics, double nu,
                            double cfl, double blend, const fdlbm_opts &o, bool force_staged,
                            fdlbm_ctx **out, std::vector<double> &mx, std::vector<double> &my);
fdlbm_status handle_upload(fdlbm_ctx *h, const std::vector<double> &mx,
                           const std::vector<double> &my);
template <class R>
StepArgs<R> handle_step_args(fdlbm_ctx *h);
Layout make_layout(int nx, int ny, int pitch, int precision, int has_force, bool staged);

// step_fused.cu
template <class R>
cudaError_t launch_fused(const StepArgs<R> &a, cudaStream_t s);
int fused_tile_width();
template <class R>
int fused_blocks_per_sm();
// step_fused_s2.cu (T2S2-FDLBM2, periodic grids)
template <class R>
cudaError_t launch_fused_s2(const StepArgs<R> &a, cudaStream_t s);
template <class R>
int fused_s2_blocks_per_sm();
template <class R>
cudaError_t launch_batched_fused_s2(const BatchTables &t, int parity, int blk_off, int nblocks,
                                    cudaStream_t s);
// step_fused_warp.cu (FP32, one independent warp per tile, packed f32x2)
bool fused_warp_ok(int nx, int ny, bool wall_x);
cudaError_t fused_warp_encode(WarpMaps *m, const float *state0, const float *state1,
                              const float *force, int nx, int ny, int pitch, size_t plane);
cudaError_t launch_fused_warp(const StepArgs<float> &a, const WarpMaps &maps, int cur,
                              cudaStream_t s);
// Frame geometry of a walled grid split between the warp-tile kernel (the
// interior rectangle [xoff, xend) x [yoff, yend)) and a walls sweep in blocks
// of one warp (nframe tiles, erows rows beside the interior rows).
struct FrameGeom {
    int nx, ny, wx, wy;
    int xoff, xend, yoff, yend, erows, nframe;
};
// step_fused_s2.cu: the frame of a walled T2S2-FDLBM2 grid (FP32).
cudaError_t launch_frame_s2(const FrameGeom &g, const StepArgs<float> &a, cudaStream_t s);
int frame_s2_blocks_per_sm();

// The instance of the warp-tile kernel a grid needs.
struct WarpKind {
    bool inc = false, grid = false, force = false, s2 = false;  // s2: T2S2-FDLBM2
    bool operator==(const WarpKind &o) const
    {
        return inc == o.inc && grid == o.grid && force == o.force && s2 == o.s2;
    }
};
WarpKind warp_kind(const StepArgs<float> &s);
// Batches: the per-case argument blocks (tensor maps and scalars) in a device
// table, and one launch over tiles of cases of one kind.
size_t fused_warp_args_bytes();
cudaError_t fused_warp_args(void *dst, const StepArgs<float> &s, const WarpMaps &maps, int cur);
cudaError_t launch_batched_warp(const void *args, const int *blk_case, const int *blk_start,
                                int blk_off, int nblocks, WarpKind k, cudaStream_t s);
// The frames of walled cases (the walls sweep in blocks of one warp): frame
// tile b - frame_start[c] of case c = blk_case[b].
cudaError_t launch_batched_frame(const void *args, const void *sargs, const int *blk_case,
                                 const int *frame_start, int blk_off, int nblocks, bool force,
                                 cudaStream_t s);
// Interior tiles (warp-tile launch) and frame tiles (walls-sweep launch, 0 on
// a periodic grid) of one grid at its tile height.
void fused_warp_tiles(const StepArgs<float> &s, int *interior, int *frame);
// The same tiles as a list (5 ints each: kind 0 interior / 1 frame, x0, end of
// the stored columns, y0, y1); host only.  Returns the count (entries past cap
// are not written).
int warp_tile_plan(int nx, int ny, bool wx, bool wy, int rows, bool s2, int *out, int cap);
int fused_warp_tile_width();
int fused_warp_blocks_per_sm();
// step_fused_walls.cu (scalar sweep with walled axes and Eq. 3.10 inside)
template <class R>
cudaError_t launch_fused_walls(const StepArgs<R> &a, cudaStream_t s);
template <class R>
int fused_walls_blocks_per_sm();
template <class R>
cudaError_t launch_batched_fused(const BatchTables &t, int parity, int blk_off, int nblocks,
                                 cudaStream_t s);
int fused_tile_width_walls();
// step_staged.cu
template <class R>
cudaError_t launch_staged(const StepArgs<R> &a, cudaStream_t s);
// step_batched.cu (one launch per stage for all cases of a batch)
template <class R>
cudaError_t launch_batched(const BatchTables &t, int parity, dim3 blk, cudaStream_t s);
// step_persist.cu (one cooperative launch for many steps of all cases)
template <class R>
cudaError_t launch_persistent(const BatchTables &t, void *bar, int parity0, int nsteps, dim3 blk,
                              cudaStream_t s, unsigned spin_limit);
template <class R>
int persistent_blocks_per_sm(dim3 blk);
// step_fused_walls.cu: the fused batch sweep as one cooperative launch
template <class R>
cudaError_t launch_persistent_fused(const BatchTables &t, void *bar, int parity0, int nsteps,
                                    cudaStream_t s, unsigned spin_limit);
template <class R>
int persistent_fused_blocks_per_sm();
size_t persistent_barrier_bytes();
// adjoint.cu
template <class R>
cudaError_t launch_adjoint(const StepArgs<R> &a, const R *lam_next, R *lam_prev, R *P, R *lgs,
                           double *fB, double *dforce, cudaStream_t s);
template <class R>
cudaError_t launch_init_vjp(const StepArgs<R> &a, const double *rho, const double *ux,
                            const double *uy, const R *lam, double dt, double *drho, double *dux,
                            double *duy, double *dforce, cudaStream_t s);
template <class R>
cudaError_t launch_moments_vjp(const StepArgs<R> &a, const double *du, R *lam, double *dforce,
                               cudaStream_t s);
// fields.cu
template <class T>
cudaError_t launch_init_fields(fdlbm_ctx *h, const T *rho, const T *ux, const T *uy, const T *grad,
                               int row0, int nrows, size_t src_pitch_rows);
cudaError_t launch_convert_in(fdlbm_ctx *h, const double *f, int row0, int nrows,
                              size_t src_plane);
cudaError_t launch_convert_out(fdlbm_ctx *h, double *f, int row0, int nrows, size_t dst_plane);
cudaError_t launch_set_force(fdlbm_ctx *h, const double *force, int row0, int nrows,
                             size_t src_plane);
template <class T>
cudaError_t launch_moments(fdlbm_ctx *h, T *rho, T *ux, T *uy, int row0, int nrows,
                           size_t dst_plane);
cudaError_t launch_reduce(fdlbm_ctx *h, int use_prev);

}  // namespace fdlbm
