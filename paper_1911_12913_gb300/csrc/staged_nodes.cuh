// Per-node stages of the staged T2S2-FDLBM step (any boundary combination),
// shared by the single-case kernels (step_staged.cu), the batched kernels
// (step_batched.cu) and the persistent batched kernel (step_persist.cu).
//
//   prepare_node  all nodes        P = fbar^{+,h} (Eqs. 2.19, 2.34), Q = f~+ (Eq. 2.20)
//                                  (scheme 2: P = physical f^n, Eq. 2.32 with h = dt)
//   star_node     interior nodes   S = f* from fbar* = src - h xi.grad src (Eqs. 2.32-2.35),
//                                  src = P (scheme 1) or Q (scheme 2: fbar^{+,h} = f~+ for h = dt)
//   update_node   interior nodes   out = Q - dt xi.grad S (Eq. 2.23)
//                                  (scheme 2: out = Q - dt/2 xi.grad (P + S), Eq. 5.23)
//   wall_node     wall nodes       Eq. 3.10 from the nearest interior node
//
// Next to a wall, where the second-order upwind difference would need a node
// outside the domain, the central difference is used alone.  A null force
// pointer means no body force even when FORCE is set (the batched kernels mix
// cases with and without a force field).
#pragma once

#include "internal.h"

namespace fdlbm {

template <class R>
__device__ __forceinline__ bool is_wall_node(const StepArgs<R> &a, int x, int y)
{
    return (a.bc_x == FDLBM_WALL && (x == 0 || x == a.nx - 1)) ||
           (a.bc_y == FDLBM_WALL && (y == 0 || y == a.ny - 1));
}

// m_x sgn(c_x) D_x + m_y sgn(c_y) D_y of population i of `fld` ([ny][pitch]
// plane) at interior node (x, y): xi_i . grad f_i in physical coordinates.
template <class R>
__device__ R xi_grad(const StepArgs<R> &a, const R *__restrict__ fld, int i, int x, int y)
{
    R out = R(0);
    if (cx(i) != 0) {
        const int s = cx(i);
        const bool per = a.bc_x == FDLBM_PERIODIC;
        const bool up = per || (s > 0 ? x >= 2 : x <= a.nx - 3);
        const R *row = fld + (size_t)y * a.pitch;
        auto at = [&](int d) {
            int xx = x + d;
            if (per) xx = wrap_index(xx, a.nx);
            return row[xx];
        };
        // read only the taps the stencil of this sign uses (the far tap on the
        // other side may lie outside a walled domain)
        R v;
        if (up)
            v = s > 0 ? apply_stencil(a.st, s, at(-2), at(-1), at(0), at(1), R(0))
                      : apply_stencil(a.st, s, R(0), at(-1), at(0), at(1), at(2));
        else
            v = apply_stencil(a.stc, s, R(0), at(-1), R(0), at(1), R(0));
        out += a.mx[x] * v;
    }
    if (cy(i) != 0) {
        const int s = cy(i);
        const bool per = a.bc_y == FDLBM_PERIODIC;
        const bool up = per || (s > 0 ? y >= 2 : y <= a.ny - 3);
        auto at = [&](int d) {
            int yy = y + d;
            if (per) yy = wrap_index(yy, a.ny);
            return fld[(size_t)yy * a.pitch + x];
        };
        R v;
        if (up)
            v = s > 0 ? apply_stencil(a.st, s, at(-2), at(-1), at(0), at(1), R(0))
                      : apply_stencil(a.st, s, R(0), at(-1), at(0), at(1), at(2));
        else
            v = apply_stencil(a.stc, s, R(0), at(-1), R(0), at(1), R(0));
        out += a.my[y] * v;
    }
    return out;
}

// Eq. 3.3 for a distribution whose first moment lacks `shift rho F`.
template <class R, bool FORCE>
__device__ __forceinline__ void node_macro(const StepArgs<R> &a, const R g[9], R shift, size_t fo,
                                           R &drho, R &rho, R &ux, R &uy, R &Fx, R &Fy)
{
    R jx, jy;
    moments_dev(g, drho, jx, jy);
    rho = macro_density(a.c, drho);
    Fx = R(0);
    Fy = R(0);
    if (FORCE && a.force) {
        Fx = a.force[fo];
        Fy = a.force[a.plane + fo];
        jx += shift * rho * Fx;
        jy += shift * rho * Fy;
    }
    const R inv = R(1) / rho;
    ux = jx * inv;
    uy = jy * inv;
}

template <class R, bool FORCE>
__device__ void prepare_node(const StepArgs<R> &a, int x, int y)
{
    const size_t o = (size_t)y * a.pitch + x;
    R g[9], geq[9], F[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) g[i] = a.gin[i * a.plane + o];
    R drho, rho, ux, uy, Fx, Fy;
    node_macro<R, FORCE>(a, g, a.c.half_dt, o, drho, rho, ux, uy, Fx, Fy);
    equilibrium_dev(drho, rho, ux, uy, geq);
    if (FORCE) force_terms(a.c.rho0, geq, ux, uy, Fx, Fy, F, force_dshift(a.c, drho));
    const bool s2 = a.scheme == FDLBM_SCHEME_T2S2_2;
    const R bP = s2 ? a.c.b_phys : a.c.b_bar, cP = s2 ? a.c.c_phys : a.c.c_bar;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const R neq = geq[i] - g[i];
        R gb = g[i] + bP * neq;
        R gt = g[i] + a.c.b_til * neq;
        if (FORCE) {
            gb += cP * F[i];
            gt += a.c.c_til * F[i];
        }
        a.P[i * a.plane + o] = gb;
        a.Q[i * a.plane + o] = gt;
    }
}

template <class R, bool FORCE>
__device__ void star_node(const StepArgs<R> &a, int x, int y)
{
    if (is_wall_node(a, x, y)) return;
    const size_t o = (size_t)y * a.pitch + x;
    const R *src = a.scheme == FDLBM_SCHEME_T2S2_2 ? a.Q : a.P;
    R gs[9], geq[9], F[9];
#pragma unroll
    for (int i = 0; i < 9; ++i)
        gs[i] = src[i * a.plane + o] - a.c.h * xi_grad(a, src + i * a.plane, i, x, y);
    R drho, rho, ux, uy, Fx, Fy;
    node_macro<R, FORCE>(a, gs, a.c.half_h, o, drho, rho, ux, uy, Fx, Fy);
    equilibrium_dev(drho, rho, ux, uy, geq);
    if (FORCE) force_terms(a.c.rho0, geq, ux, uy, Fx, Fy, F, force_dshift(a.c, drho));
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        R v = gs[i] + a.c.b_star * (geq[i] - gs[i]);
        if (FORCE) v += a.c.c_star * F[i];
        a.S[i * a.plane + o] = v;
    }
}

template <class R>
__device__ void update_node(const StepArgs<R> &a, int x, int y)
{
    if (is_wall_node(a, x, y)) return;
    const size_t o = (size_t)y * a.pitch + x;
    if (a.scheme == FDLBM_SCHEME_T2S2_2) {
#pragma unroll
        for (int i = 0; i < 9; ++i)
            a.gout[i * a.plane + o] =
                a.Q[i * a.plane + o] - a.c.half_dt * (xi_grad(a, a.P + i * a.plane, i, x, y) +
                                                      xi_grad(a, a.S + i * a.plane, i, x, y));
        return;
    }
#pragma unroll
    for (int i = 0; i < 9; ++i)
        a.gout[i * a.plane + o] =
            a.Q[i * a.plane + o] - a.c.dt * xi_grad(a, a.S + i * a.plane, i, x, y);
}

// Number of wall nodes of a case (row walls first, then the column walls
// without the corners the rows already cover).
template <class R>
__host__ __device__ __forceinline__ int wall_count(const StepArgs<R> &a)
{
    const bool wy = a.bc_y == FDLBM_WALL, wx = a.bc_x == FDLBM_WALL;
    return (wy ? 2 * a.nx : 0) + (wx ? 2 * (wy ? a.ny - 2 : a.ny) : 0);
}

// Eq. 3.10 on wall node number k of `fld`: g_b = geq(rho_j, u_wall) + g_j -
// geq(rho_j, u_j), j the nearest interior node along the inward normal
// (diagonal at corners); the W/E walls own the corners.  `shift` is the force
// shift of the first moment of `fld` (dt/2 for f~, 0 for the physical-like f*).
template <class R, bool FORCE>
__device__ void wall_node(const StepArgs<R> &a, R *fld, R shift, int k)
{
    const bool wy = a.bc_y == FDLBM_WALL, wx = a.bc_x == FDLBM_WALL;
    const int nrow = wy ? 2 * a.nx : 0;
    const int ncol = wx ? 2 * (wy ? a.ny - 2 : a.ny) : 0;
    if (k >= nrow + ncol) return;
    int x, y;
    if (k < nrow) {
        x = k % a.nx;
        y = (k < a.nx) ? 0 : a.ny - 1;
    } else {
        const int m = k - nrow, len = ncol / 2;
        x = (m < len) ? 0 : a.nx - 1;
        y = (m % len) + (wy ? 1 : 0);
    }
    int jx = x, jy = y;
    if (wx) jx = x == 0 ? 1 : (x == a.nx - 1 ? a.nx - 2 : x);
    if (wy) jy = y == 0 ? 1 : (y == a.ny - 1 ? a.ny - 2 : y);
    int side;
    if (wx && x == 0) side = FDLBM_WALL_W;
    else if (wx && x == a.nx - 1) side = FDLBM_WALL_E;
    else if (y == 0) side = FDLBM_WALL_S;
    else side = FDLBM_WALL_N;
    const size_t ob = (size_t)y * a.pitch + x, oj = (size_t)jy * a.pitch + jx;
    R g[9], geqj[9], geqb[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) g[i] = fld[i * a.plane + oj];
    R drho, rho, ux, uy, Fx, Fy;
    node_macro<R, FORCE>(a, g, shift, oj, drho, rho, ux, uy, Fx, Fy);
    equilibrium_dev(drho, rho, ux, uy, geqj);
    equilibrium_dev(drho, rho, a.wall_u[side][0], a.wall_u[side][1], geqb);
#pragma unroll
    for (int i = 0; i < 9; ++i) fld[i * a.plane + ob] = geqb[i] + (g[i] - geqj[i]);
}

}  // namespace fdlbm
