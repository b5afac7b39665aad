// The fused T2S2-FDLBM1 sweep with walls: the rolling sweep of step_fused.cu (stages
// A, B, C of Sec. 2D at rows r, r-2, r-4; one column per thread; y-differences
// from register windows, x-differences from shared-memory rings) on grids with
// one or two walled axes, with the non-equilibrium extrapolation of Eq. 3.10 done
// inside the sweep.  One read and one write of f~ per node.  Blocks of NT
// threads, one column each: 128 for the walls sweep of step_fused_walls.cu,
// one warp for the frame of a walled grid around the warp-tile kernel's
// interior (step_fused_warp.cu).
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
#pragma once

#include <cstdint>

#include <algorithm>

#include "internal.h"
#include "walls_nodes.cuh"

namespace fdlbm {
namespace walls_sweep {

constexpr int kHalo = 4;
constexpr int kRing = 5;

template <class R, int NT>
struct Smem {
    R P[kRing][6][NT];   // fbar^{+,h} of the x-moving populations
    R S[kRing][6][NT];   // f* of the x-moving populations
    R Q[kRing][9][NT];   // f~+ (read back by the same thread only)
};

// PF: the y metric and the force arrive a row ahead, as f~ does, instead of
// at the row that uses them (a dependent load in every row of the sweep);
// for kernels whose registers allow it.
template <class R, bool FORCE, int NT, bool PF>
struct SweepW {
    const StepArgs<R> a;
    Smem<R, NT> &sm;
    const int t, xc, gx;
    const bool wx, wy;       // walled axes
    const bool colB, colC;   // this column evaluates stage B / stage C
    const R mxc;
    const Coeffs<R> c;
    Stencil<R> sxp, sxn;     // x-differences at this column for sign + / -
    R Pw[9][kRing];
    R Sw[9][kRing];
    R cur[9], nxt[9];
    // PF: the y metric of stage B's rows r-2, r-3, r-4 (stage C's row) and of
    // r-1, and the force of rows r+1 (nF) .. r-2
    R myB[PF ? 4 : 1];
    R F0[2], F1[2], F2[2], nF[2];
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
        if (load_next) {
            load(nxt, r + 1);
            if (PF && FORCE) force_at(r + 1, nF[0], nF[1]);
        }
        if constexpr (PF) myB[3] = a.my[mem_row(r - 1)];  // stage B of the next row
        // ------------------------------------------------------------ A (row r)
        {
            R Fx = F0[0], Fy = F0[1];
            if (!PF) force_at(r, Fx, Fy);
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
                const R hx = c.h * mxc, hy = c.h * (PF ? myB[0] : a.my[mem_row(rb)]);
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
                R Fx = F2[0], Fy = F2[1];
                if (!PF) force_at(rb, Fx, Fy);
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
                R myc;
                if constexpr (PF) myc = myB[2];
                else myc = a.my[mem_row(rc)];
                const R dx = c.dt * mxc, dy = c.dt * myc;
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
        if constexpr (PF) {
            myB[2] = myB[1];
            myB[1] = myB[0];
            myB[0] = myB[3];
        }
        if (PF && FORCE) {
            F2[0] = F1[0];
            F2[1] = F1[1];
            F1[0] = F0[0];
            F1[1] = F0[1];
            F0[0] = nF[0];
            F0[1] = nF[1];
        }
        ++rA;
    }
};

// One tile: output columns x0 .. x0 + NT - 9 below xhi and rows y0 .. y1 - 1.
// TAIL: the rows past the last full group of five in a separate copy of the
// row phases (twice the code: faster only where instruction fetch does not
// limit, the persistent batch kernel).
template <class R, bool FORCE, int NT, bool PF = false, bool TAIL = false>
__device__ __forceinline__ void sweep_tile(const StepArgs<R> &a, Smem<R, NT> &sm, int x0, int xhi,
                                           int y0, int y1)
{
    const int t = threadIdx.x;
    const int xc = x0 - kHalo + t;
    const bool wx = a.bc_x == FDLBM_WALL, wy = a.bc_y == FDLBM_WALL;
    const bool inside = !wx || (xc >= 0 && xc < a.nx);
    const int gx = wx ? min(max(xc, 0), a.nx - 1) : wrap_index(xc, a.nx);
    const bool colint = !wx || (xc >= 1 && xc <= a.nx - 2);
    const bool colB = (t >= 2) && (t < NT - 2) && inside && colint;
    const bool colC = (t >= kHalo) && (t < NT - kHalo) && xc < min(a.nx, xhi) && inside && colint;
    SweepW<R, FORCE, NT, PF> sw{a,
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
    sw.F0[0] = sw.F0[1] = sw.F1[0] = sw.F1[1] = sw.F2[0] = sw.F2[1] = sw.nF[0] = sw.nF[1] = R(0);
    if constexpr (PF) {
        // (rows before the segment's first: their stage B and C results are discarded)
        sw.myB[0] = sw.myB[1] = sw.myB[2] = sw.myB[3] = a.my[sw.mem_row(sw.rA - 2)];
        sw.force_at(sw.rA, sw.F0[0], sw.F0[1]);
    }
    const int iters = (y1 - y0) + 2 * kHalo;
    if constexpr (TAIL) {
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
    } else {
        // one copy of each phase of the unrolled row (the rows past the
        // segment's end skipped by uniform guards): half the code of a separate
        // tail, which matters to the instruction cache
        for (int k = 0; k < iters; k += kRing) {
            sw.template row<0>(k + 1 < iters, k >= 4, k >= 8);
            if (k + 1 < iters) sw.template row<1>(k + 2 < iters, k + 1 >= 4, k + 1 >= 8);
            if (k + 2 < iters) sw.template row<2>(k + 3 < iters, k + 2 >= 4, k + 2 >= 8);
            if (k + 3 < iters) sw.template row<3>(k + 4 < iters, k + 3 >= 4, k + 3 >= 8);
            if (k + 4 < iters) sw.template row<4>(k + 5 < iters, k + 4 >= 4, k + 4 >= 8);
        }
    }
}

}  // namespace walls_sweep
}  // namespace fdlbm
