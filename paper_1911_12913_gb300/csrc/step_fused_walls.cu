// Fused T2S2-FDLBM1 step with walls: the rolling sweep of step_fused.cu (stages
// A, B, C of Sec. 2D at rows r, r-2, r-4; one column per thread; y-differences
// from register windows, x-differences from shared-memory rings) on grids with
// one or two walled axes, with the non-equilibrium extrapolation of Eq. 3.10 done
// inside the sweep.  One launch per step, one read and one write of f~ per node.
//
// Walls (the same conventions as the staged kernels, staged_nodes.cuh):
//   - wall nodes take no part in stages B and C; their f* and new f~ come from
//     Eq. 3.10 at the nearest interior node x_j along the inward normal
//     (diagonal at corners, where the W/E walls own the wall velocity);
//   - an interior node whose second-order upwind difference would reach outside
//     the domain uses the central difference alone.
// Eq. 3.10 is evaluated by the thread that owns x_j, right after it has x_j's
// values:
//   f* of a W/E wall node    stage B at x_j, written into the shared ring (the
//                            x-differences of stage C read it there);
//   f* of the S wall row     stage B at row 1, written into the register
//                            window slot of row 0 (read by stage C at row 1);
//   f* of the N wall row     stage B at row ny-1, from the window row ny-2;
//   new f~ of wall nodes     stage C at x_j, stored with x_j's own output.
// f* of corner nodes is never read (the differences are one-dimensional).
//
// On a walled axis, loads outside the domain read the nearest row or column and
// stages B and C are not evaluated there; slots that a central difference
// weights by zero always hold finite values (stage B writes zeros for rows and
// columns it does not evaluate), so the zero weights never meet a NaN.
#include <cstdint>

#include <algorithm>

#include "grid_barrier.cuh"
#include "internal.h"
#include "walls_nodes.cuh"

namespace fdlbm {
namespace {

constexpr int kHalo = 4;
constexpr int kRing = 5;
constexpr int NT = 128;

template <class R>
struct Smem {
    R P[kRing][6][NT];   // fbar^{+,h} of the x-moving populations
    R S[kRing][6][NT];   // f* of the x-moving populations
    R Q[kRing][9][NT];   // f~+ (read back by the same thread only)
};

// Offset of the argument block after the rings in the persistent batch kernel's
// dynamic shared memory, and that memory's size.
template <class R>
constexpr size_t kArgOffset = (sizeof(Smem<R>) + 15) / 16 * 16;
template <class R>
constexpr size_t kPersistSmem = kArgOffset<R> + sizeof(StepArgs<R>);

template <class R, bool FORCE>
struct SweepW {
    const StepArgs<R> a;
    Smem<R> &sm;
    const int t, xc, gx;
    const bool wx, wy;       // walled axes
    const bool colB, colC;   // this column evaluates stage B / stage C
    const R mxc;
    const Coeffs<R> c;
    Stencil<R> sxp, sxn;     // x-differences at this column for sign + / -
    R Pw[9][kRing];
    R Sw[9][kRing];
    R cur[9], nxt[9];
    int rA;                  // logical row of cur (may lie outside [0, ny))
    int y1;                  // end of the segment's output rows

    __device__ int mem_row(int r) const
    {
        return wy ? min(max(r, 0), a.ny - 1) : wrap_index(r, a.ny);
    }

    __device__ void load(R *dst, int r) const
    {
        const size_t off = (size_t)mem_row(r) * a.pitch + gx;
#pragma unroll
        for (int i = 0; i < 9; ++i) dst[i] = __ldg(a.gin + i * a.plane + off);
    }

    __device__ void force_at(int r, R &Fx, R &Fy) const
    {
        Fx = Fy = R(0);
        if (FORCE && a.force) {
            const size_t fo = (size_t)mem_row(r) * a.pitch + gx;
            Fx = __ldg(a.force + fo);
            Fy = __ldg(a.force + a.plane + fo);
        }
    }

    // wall velocity (component k) of the W or E wall (west = true) and of the S
    // or N wall (south = true); constant indices only, so that the argument
    // block is never indexed at run time
    __device__ R uwx_side(bool west, int k) const
    {
        return west ? (k ? a.wall_u[FDLBM_WALL_W][1] : a.wall_u[FDLBM_WALL_W][0])
                    : (k ? a.wall_u[FDLBM_WALL_E][1] : a.wall_u[FDLBM_WALL_E][0]);
    }
    __device__ R uwy_side(bool south, int k) const
    {
        return south ? (k ? a.wall_u[FDLBM_WALL_S][1] : a.wall_u[FDLBM_WALL_S][0])
                     : (k ? a.wall_u[FDLBM_WALL_N][1] : a.wall_u[FDLBM_WALL_N][0]);
    }

    template <int PH>
    __device__ void row(bool load_next, bool doB, bool doC)
    {
        constexpr int p0 = PH;
        constexpr int p1 = (PH + 4) % kRing;
        constexpr int p2 = (PH + 3) % kRing;
        constexpr int p3 = (PH + 2) % kRing;
        constexpr int p4 = (PH + 1) % kRing;
        const int r = rA;
        if (load_next) load(nxt, r + 1);
        // ------------------------------------------------------------ A (row r)
        {
            R Fx, Fy;
            force_at(r, Fx, Fy);
            R drho, rho, ux, uy, geq[9], F[9];
            node_eq<R, FORCE>(c, cur, Fx, Fy, c.half_dt, drho, rho, ux, uy, geq);
            if (FORCE) force_terms(c.rho0, geq, ux, uy, Fx, Fy, F, force_dshift(c, drho));
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const R neq = geq[i] - cur[i];
                R gb = cur[i] + c.b_bar * neq;
                R gt = cur[i] + c.b_til * neq;
                if (FORCE) {
                    gb += c.c_bar * F[i];
                    gt += c.c_til * F[i];
                }
                Pw[i][p0] = gb;
                if (xslot(i) >= 0) sm.P[p0][xslot(i)][t] = gb;
                sm.Q[p0][i][t] = gt;
            }
        }
        __syncthreads();
        // ------------------------------------------------------------ B (row r-2)
        if (doB) {
            const int rb = r - 2;
            const bool rowin = !wy || (rb >= 1 && rb <= a.ny - 2);
            if (colB && rowin) {
                const R hx = c.h * mxc, hy = c.h * a.my[mem_row(rb)];
                const Stencil<R> syp = (wy && rb == 1) ? a.stc : a.st;
                const Stencil<R> syn = (wy && rb == a.ny - 2) ? a.stc : a.st;
                R gs[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const R v0 = Pw[i][p2];
                    R acc = v0;
                    if (cx(i) != 0) {
                        const R *rw = sm.P[p2][xslot(i)];
                        acc -= hx * apply_stencil(cx(i) > 0 ? sxp : sxn, cx(i), rw[t - 2], rw[t - 1],
                                                  v0, rw[t + 1], rw[t + 2]);
                    }
                    if (cy(i) != 0)
                        acc -= hy * apply_stencil(cy(i) > 0 ? syp : syn, cy(i), Pw[i][p4], Pw[i][p3],
                                                  v0, Pw[i][p1], Pw[i][p0]);
                    gs[i] = acc;
                }
                R Fx, Fy;
                force_at(rb, Fx, Fy);
                R drho, rho, ux, uy, geq[9], F[9];
                node_eq<R, FORCE>(c, gs, Fx, Fy, c.half_h, drho, rho, ux, uy, geq);
                if (FORCE) force_terms(c.rho0, geq, ux, uy, Fx, Fy, F, force_dshift(c, drho));
                R st[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    R v = gs[i] + c.b_star * (geq[i] - gs[i]);
                    if (FORCE) v += c.c_star * F[i];
                    st[i] = v;
                    Sw[i][p0] = v;
                    if (xslot(i) >= 0) sm.S[p0][xslot(i)][t] = v;
                }
                // Eq. 3.10 for f* (no force shift) of the wall nodes next to x_j
                if (wx && (xc == 1 || xc == a.nx - 2)) {
                    R wv[9];
                    nee<R, false>(c, st, R(0), R(0), R(0), uwx_side(xc == 1, 0), uwx_side(xc == 1, 1), wv);
                    const int tw = xc == 1 ? t - 1 : t + 1;
#pragma unroll
                    for (int i = 0; i < 9; ++i)
                        if (xslot(i) >= 0) sm.S[p0][xslot(i)][tw] = wv[i];
                }
                if (wy && rb == 1) {  // the S wall row, into the window slot of row 0
                    R wv[9];
                    nee<R, false>(c, st, R(0), R(0), R(0), uwy_side(true, 0), uwy_side(true, 1), wv);
#pragma unroll
                    for (int i = 0; i < 9; ++i) Sw[i][p1] = wv[i];
                }
            } else if (colB && wy && rb == a.ny - 1) {
                // the N wall row, from the window row ny-2
                R sj[9], wv[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) sj[i] = Sw[i][p1];
                nee<R, false>(c, sj, R(0), R(0), R(0), uwy_side(false, 0), uwy_side(false, 1), wv);
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    Sw[i][p0] = wv[i];
                    if (xslot(i) >= 0) sm.S[p0][xslot(i)][t] = wv[i];
                }
            } else {
                // not evaluated here: finite zeros (wall columns keep the value
                // their interior neighbour writes into the ring)
                const bool wallcol = wx && (xc == 0 || xc == a.nx - 1);
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    Sw[i][p0] = R(0);
                    if (xslot(i) >= 0 && !wallcol) sm.S[p0][xslot(i)][t] = R(0);
                }
            }
        }
        __syncthreads();
        // ------------------------------------------------------------ C (row r-4)
        if (doC) {
            const int rc = r - 4;
            const bool rowin = !wy || (rc >= 1 && rc <= a.ny - 2);
            if (colC && rowin && rc < y1) {
                const R dx = c.dt * mxc, dy = c.dt * a.my[mem_row(rc)];
                const Stencil<R> syp = (wy && rc == 1) ? a.stc : a.st;
                const Stencil<R> syn = (wy && rc == a.ny - 2) ? a.stc : a.st;
                R out[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const R v0 = Sw[i][p2];
                    R acc = sm.Q[p4][i][t];
                    if (cx(i) != 0) {
                        const R *rw = sm.S[p2][xslot(i)];
                        acc -= dx * apply_stencil(cx(i) > 0 ? sxp : sxn, cx(i), rw[t - 2], rw[t - 1],
                                                  v0, rw[t + 1], rw[t + 2]);
                    }
                    if (cy(i) != 0)
                        acc -= dy * apply_stencil(cy(i) > 0 ? syp : syn, cy(i), Sw[i][p4], Sw[i][p3],
                                                  v0, Sw[i][p1], Sw[i][p0]);
                    out[i] = acc;
                }
                const int my_row = mem_row(rc);
                auto put = [&](int x, int y, const R *v) {
                    const size_t o = (size_t)y * a.pitch + x;
#pragma unroll
                    for (int i = 0; i < 9; ++i) a.gout[i * a.plane + o] = v[i];
                };
                put(gx, my_row, out);
                // Eq. 3.10 on the new f~ (force shift dt/2) of the wall nodes
                // whose x_j is this node
                const bool bw = wy && rc == 1, tw = wy && rc == a.ny - 2;
                const bool lw = wx && xc == 1, rw = wx && xc == a.nx - 2;
                if (bw || tw || lw || rw) {
                    R Fx, Fy;
                    force_at(rc, Fx, Fy);
                    R wv[9];
                    if (bw) {
                        nee<R, FORCE>(c, out, Fx, Fy, c.half_dt, uwy_side(true, 0), uwy_side(true, 1), wv);
                        put(gx, 0, wv);
                    }
                    if (tw) {
                        nee<R, FORCE>(c, out, Fx, Fy, c.half_dt, uwy_side(false, 0), uwy_side(false, 1), wv);
                        put(gx, a.ny - 1, wv);
                    }
                    if (lw || rw) {
                        const int xw = lw ? 0 : a.nx - 1;
                        nee<R, FORCE>(c, out, Fx, Fy, c.half_dt, uwx_side(lw, 0), uwx_side(lw, 1), wv);
                        put(xw, my_row, wv);
                        if (bw) put(xw, 0, wv);           // corner, diagonal x_j
                        if (tw) put(xw, a.ny - 1, wv);
                    }
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) cur[i] = nxt[i];
        ++rA;
    }
};

// One tile: output columns x0 .. x0 + W - 1 and rows y0 .. y0 + a.rows - 1.
template <class R, bool FORCE>
__device__ __forceinline__ void sweep_tile(const StepArgs<R> &a, Smem<R> &sm, int x0, int y0)
{
    const int t = threadIdx.x;
    const int xc = x0 - kHalo + t;
    const int y1 = min(y0 + a.rows, a.ny);
    const bool wx = a.bc_x == FDLBM_WALL, wy = a.bc_y == FDLBM_WALL;
    const bool inside = !wx || (xc >= 0 && xc < a.nx);
    const int gx = wx ? min(max(xc, 0), a.nx - 1) : wrap_index(xc, a.nx);
    const bool colint = !wx || (xc >= 1 && xc <= a.nx - 2);
    const bool colB = (t >= 2) && (t < NT - 2) && inside && colint;
    const bool colC = (t >= kHalo) && (t < NT - kHalo) && xc < a.nx && inside && colint;
    SweepW<R, FORCE> sw{a,
                        sm,
                        t,
                        xc,
                        gx,
                        wx,
                        wy,
                        colB,
                        colC,
                        a.mx[gx],
                        a.c,
                        (wx && xc == 1) ? a.stc : a.st,
                        (wx && xc == a.nx - 2) ? a.stc : a.st};
    sw.y1 = y1;
    sw.rA = y0 - kHalo;
    sw.load(sw.cur, sw.rA);
    const int iters = (y1 - y0) + 2 * kHalo;
    int k = 0;
    for (; k + kRing <= iters; k += kRing) {
        sw.template row<0>(k + 1 < iters, k >= 4, k >= 8);
        sw.template row<1>(k + 2 < iters, k + 1 >= 4, k + 1 >= 8);
        sw.template row<2>(k + 3 < iters, k + 2 >= 4, k + 2 >= 8);
        sw.template row<3>(k + 4 < iters, k + 3 >= 4, k + 3 >= 8);
        sw.template row<4>(k + 5 < iters, k + 4 >= 4, k + 4 >= 8);
    }
    if (k < iters) sw.template row<0>(k + 1 < iters, true, k >= 8);
    if (k + 1 < iters) sw.template row<1>(k + 2 < iters, true, k + 1 >= 8);
    if (k + 2 < iters) sw.template row<2>(k + 3 < iters, true, k + 2 >= 8);
    if (k + 3 < iters) sw.template row<3>(k + 4 < iters, true, k + 3 >= 8);
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
// Persistent batched: all tiles of all cases for nsteps steps in one
// cooperative launch (all blocks resident).  Within a step the blocks fetch
// tiles from a global counter, as the hardware would hand out the blocks of
// one launch; one grid barrier separates consecutive steps, since a step reads
// the state the previous one wrote around its tile.  Steps alternate between
// two counters: block 0 clears the next step's counter at the start of a step,
// when every block has passed the barrier after that counter's last use.  A
// barrier that times out sets every case's error flag and the block leaves;
// the others then time out at their next barrier.
// One tile of the persistent batch, out of line: the tile sweep then gets the
// registers of the batched kernel, and the step loop of the caller keeps only
// a few values live across the call.  The case's argument block goes to
// dynamic shared memory after the sweep's rings.
template <class R>
__device__ __noinline__ void persistent_tile(const StepArgs<R> *cases, const int *blk_case,
                                             const int *blk_start, const int *tiles_x, int b)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<R> &sm = *reinterpret_cast<Smem<R> *>(smem_raw);
    unsigned char *abuf = smem_raw + kArgOffset<R>;
    static_assert(sizeof(StepArgs<R>) % 4 == 0, "argument block is copied as 32-bit words");
    const int c = blk_case[b];
    {
        const int *src = reinterpret_cast<const int *>(cases + c);
        int *dst = reinterpret_cast<int *>(abuf);
        for (int q = threadIdx.x; q < (int)(sizeof(StepArgs<R>) / 4); q += blockDim.x) dst[q] = src[q];
    }
    __syncthreads();
    const StepArgs<R> &a = *reinterpret_cast<const StepArgs<R> *>(abuf);
    const int lb = b - blk_start[c], ns = tiles_x[c];
    const int y0 = (lb / ns) * a.rows;
    if (y0 < a.ny)  // uniform over the block
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
                sweep_tile<R, true>(a, sm, (lb % ns) * (NT - 2 * kHalo), y0);
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
