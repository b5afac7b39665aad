// Fused T2S2-FDLBM2 step for grids periodic in x and y: the second computational
// sequence of Sec. 2D in one kernel, one read and one write of the
// distributions per node and step (the staged kernels move 9 x 7 values).
//
// Per node, with h = dt (Sec. 2D: fbar = f~ and fbar^{+,h} = f~+ at h = dt):
//   f^n      = Eq. 2.52 on f~^n (with the force term of Eq. 2.32)
//   f~+      = Eq. 2.20 on f~^n
//   fbar     = f~+ - dt xi.grad f~+                 (Eqs. 2.33, 2.35)
//   f^{n+1}  = Eq. 2.52 on fbar
//   f~^{n+1} = f~+ + dt/2 [L(f^n) + L(f^{n+1})]    (Eq. 5.23, L of Eq. 2.27)
//
// The layout is that of the T2S2-FDLBM1 sweep (step_fused.cu): a CTA owns NT - 8
// columns and a segment of rows, thread t owns one column and sweeps bottom to
// top; differences in y read per-thread register windows of five rows, in x
// shared-memory rings written by the neighbours.  Per row r:
//   A (row r)     f^n and f~+ of the newly loaded row (windows and x-rings)
//   B (row r-2)   L(f^n) (kept in a per-thread ring for stage C two rows on),
//                 fbar from the differences of f~+, then f^{n+1} (window, x-ring)
//   C (row r-4)   L(f^{n+1}) and the update of Eq. 5.23 with f~+ from the window
// Stage B carries the two differences the scheme needs at a point (of f^n and
// of f~+) against one in T2S2-FDLBM1.  One barrier per row: every ring slot a
// stage reads was written two rows earlier, and is rewritten five rows after
// it was written.
#include <cstdint>

#include "internal.h"
#include "frame.cuh"
#include "walls_nodes.cuh"

namespace fdlbm {
namespace {

constexpr int kHalo2 = 4;
constexpr int kRing2 = 5;

template <class R, int NT>
struct Smem2 {
    R P[kRing2][6][NT];   // f^n of the x-moving populations
    R Q[kRing2][6][NT];   // f~+ of the x-moving populations
    R S[kRing2][6][NT];   // f^{n+1} of the x-moving populations
    R LN[kRing2][9][NT];  // L(f^n), read back by the same thread two rows later
};

// Moments (Eq. 3.3 with the force shift `shift`), f^eq (Eq. 3.2 or the
// incompressible one) and the forcing terms (Eq. 3.12) of a deviation vector.
template <class R, bool FORCE>
__device__ __forceinline__ void node_maps(const Coeffs<R> &c, const R g[9], R Fx, R Fy, R shift,
                                          R geq[9], R F[9])
{
    R drho, jx, jy;
    moments_dev(g, drho, jx, jy);
    const R rho = macro_density(c, drho);
    if (FORCE) {
        jx += shift * rho * Fx;
        jy += shift * rho * Fy;
    }
    const R inv = node_reciprocal(rho);
    const R ux = jx * inv, uy = jy * inv;
    equilibrium_dev_j(drho, jx, jy, inv, geq);
    if (FORCE) force_terms(c.rho0, geq, ux, uy, Fx, Fy, F, force_dshift(c, drho));
}

template <class R, bool FORCE, int NT>
struct Sweep2 {
    const StepArgs<R> a;
    Smem2<R, NT> &sm;
    const int t, gx, xc;
    const bool act1, act2;
    const R mxc;
    const Coeffs<R> c;
    const Stencil<R> st;
    R Pw[9][kRing2];  // f^n of this column, slot = row mod 5
    R Qw[9][kRing2];  // f~+
    R Sw[9][kRing2];  // f^{n+1}
    R cur[9], nxt[9];
    int rl, rs, rq;   // wrapped global rows of the next load, stage B, stage C

    __device__ static int inc(int v, int n) { return v + 1 == n ? 0 : v + 1; }

    __device__ void load(R *dst, int row) const
    {
        const size_t off = (size_t)row * a.pitch + gx;
#pragma unroll
        for (int i = 0; i < 9; ++i) dst[i] = __ldg(a.gin + i * a.plane + off);
    }

    __device__ void force_at(int row, R &Fx, R &Fy) const
    {
        Fx = Fy = R(0);
        if (FORCE) {
            const size_t fo = (size_t)row * a.pitch + gx;
            Fx = __ldg(a.force + fo);
            Fy = __ldg(a.force + a.plane + fo);
        }
    }

    // sign(c) D_m f of population i at the centre of this column, in x from
    // the ring row `rw` and in y from the window w (slots of rows k-2 .. k+2).
    __device__ __forceinline__ R dx_of(int i, const R *rw, R v0) const
    {
        return apply_stencil(st, cx(i), rw[t - 2], rw[t - 1], v0, rw[t + 1], rw[t + 2]);
    }

    template <int PH>
    __device__ void row(int k, int iters)
    {
        constexpr int p0 = PH;                  // row r       (newest)
        constexpr int p1 = (PH + 4) % kRing2;   // row r-1
        constexpr int p2 = (PH + 3) % kRing2;   // row r-2  (stage B centre)
        constexpr int p3 = (PH + 2) % kRing2;   // row r-3
        constexpr int p4 = (PH + 1) % kRing2;   // row r-4  (stage C centre)
        const int rA = rl;
        if (k + 1 < iters) {
            rl = inc(rl, a.ny);
            load(nxt, rl);
        }
        // ------------------------------------------------------------ A (row r)
        {
            R Fx, Fy, geq[9], F[9];
            force_at(rA, Fx, Fy);
            node_maps<R, FORCE>(c, cur, Fx, Fy, c.half_dt, geq, F);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const R neq = geq[i] - cur[i];
                R fn = cur[i] + c.b_phys * neq;  // Eq. 2.52, h = dt
                R ft = cur[i] + c.b_til * neq;   // Eq. 2.20
                if (FORCE) {
                    fn += c.c_phys * F[i];
                    ft += c.c_til * F[i];
                }
                Pw[i][p0] = fn;
                Qw[i][p0] = ft;
                if (xslot(i) >= 0) {
                    sm.P[p0][xslot(i)][t] = fn;
                    sm.Q[p0][xslot(i)][t] = ft;
                }
            }
        }
        __syncthreads();
        // ------------------------------------------------------------ B (row r-2)
        if (k >= 4) {
            const int sg = rs;
            rs = inc(rs, a.ny);
            if (act1) {
                const R myr = __ldg(a.my + sg);
                const R hx = c.h * mxc, hy = c.h * myr;  // h = dt
                R fb[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    // L(f^n) = -xi.grad f^n and fbar = f~+ - dt xi.grad f~+
                    R dP = R(0), fbar = Qw[i][p2];
                    if (cx(i) != 0) {
                        dP += mxc * dx_of(i, sm.P[p2][xslot(i)], Pw[i][p2]);
                        fbar -= hx * dx_of(i, sm.Q[p2][xslot(i)], Qw[i][p2]);
                    }
                    if (cy(i) != 0) {
                        dP += myr * apply_stencil(st, cy(i), Pw[i][p4], Pw[i][p3], Pw[i][p2],
                                                  Pw[i][p1], Pw[i][p0]);
                        fbar -= hy * apply_stencil(st, cy(i), Qw[i][p4], Qw[i][p3], Qw[i][p2],
                                                   Qw[i][p1], Qw[i][p0]);
                    }
                    sm.LN[p0][i][t] = -dP;
                    fb[i] = fbar;
                }
                R Fx, Fy, geq[9], F[9];
                force_at(sg, Fx, Fy);
                node_maps<R, FORCE>(c, fb, Fx, Fy, c.half_h, geq, F);
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    R fnew = fb[i] + c.b_star * (geq[i] - fb[i]);  // Eq. 2.52, h = dt
                    if (FORCE) fnew += c.c_star * F[i];
                    Sw[i][p0] = fnew;
                    if (xslot(i) >= 0) sm.S[p0][xslot(i)][t] = fnew;
                }
            }
        }
        // ------------------------------------------------------------ C (row r-4)
        // f^{n+1} rows r-6 .. r-2 sit in slots p4 .. p0 of Sw, the centre row r-4
        // in slot p2; L(f^n) of row r-4 in ring slot p2; f~+ of row r-4 in Qw p4.
        if (k >= 8) {
            const int qg = rq;
            rq = inc(rq, a.ny);
            if (act2) {
                const R myr = __ldg(a.my + qg);
                const R hdt = c.half_dt;
                const size_t off = (size_t)qg * a.pitch + xc;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    R dS = R(0);
                    if (cx(i) != 0) dS += mxc * dx_of(i, sm.S[p2][xslot(i)], Sw[i][p2]);
                    if (cy(i) != 0)
                        dS += myr * apply_stencil(st, cy(i), Sw[i][p4], Sw[i][p3], Sw[i][p2],
                                                  Sw[i][p1], Sw[i][p0]);
                    a.gout[i * a.plane + off] = Qw[i][p4] + hdt * (sm.LN[p2][i][t] - dS);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) cur[i] = nxt[i];
    }
};

template <class R, bool FORCE, int NT>
__global__ void __launch_bounds__(NT, 2) k_step_fused_s2(const StepArgs<R> a)
{
    constexpr int W = NT - 2 * kHalo2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem2<R, NT> &sm = *reinterpret_cast<Smem2<R, NT> *>(smem_raw);

    const int t = threadIdx.x;
    const int x0 = blockIdx.x * W;
    const int xc = x0 - kHalo2 + t;
    const int y0 = blockIdx.y * a.rows;
    if (y0 >= a.ny) return;  // uniform over the block
    const int y1 = min(y0 + a.rows, a.ny);
    const int gx = wrap_index(xc, a.nx);
    Sweep2<R, FORCE, NT> sw{a,
                            sm,
                            t,
                            gx,
                            xc,
                            (t >= 2) && (t < NT - 2),
                            (t >= kHalo2) && (t < NT - kHalo2) && (xc < a.nx),
                            a.mx[gx],
                            a.c,
                            a.st};
    // iteration k loads row y0-4+k; stage B works on row y0-6+k (from k = 4),
    // stage C on row y0-8+k (from k = 8)
    sw.rl = wrap_index(y0 - kHalo2, a.ny);
    sw.rs = wrap_index(y0 - 2, a.ny);
    sw.rq = y0;
    sw.load(sw.cur, sw.rl);
    const int iters = (y1 - y0) + 2 * kHalo2;
    for (int k = 0; k < iters; k += kRing2) {
        sw.template row<0>(k, iters);
        if (k + 1 < iters) sw.template row<1>(k + 1, iters);
        if (k + 2 < iters) sw.template row<2>(k + 2, iters);
        if (k + 3 < iters) sw.template row<3>(k + 3, iters);
        if (k + 4 < iters) sw.template row<4>(k + 4, iters);
    }
}

// ---------------------------------------------------------------- walled grids
// The same sweep with Eq. 3.10 inside it, laid out like the FDLBM1 walls sweep
// (step_fused_walls.cu): on a walled axis loads outside the domain read the
// nearest row or column, stages B and C run at interior nodes only, and an
// interior node whose upwind tap would leave the domain takes the central
// difference.  The second sequence extrapolates three fields to the walls
// (shift 0 for f^n and f^{n+1}, dt/2 with the force for the new f~), each from
// the interior neighbour x_j:
//   f^n      of a W/E wall column: by the x_j thread into the wall column's
//            x-ring slot; of the S wall row: into the window slot of row 0 when
//            stage A reaches row 1; of the N wall row: in place at stage A;
//   f^{n+1}  as f* in the FDLBM1 walls sweep (x-ring slot, S-row window slot
//            at stage B of row 1, N row from the window row ny-2);
//   f~^{n+1} stored with x_j's own output at stage C (corners from the
//            diagonal x_j with the W/E wall velocity).
// f~+ of a wall node is its own (Eq. 2.20 on its f~), as in the staged path.
template <class R, bool FORCE, int NT>
struct SweepS2W {
    const StepArgs<R> a;
    Smem2<R, NT> &sm;
    const int t, xc, gx;
    const bool wx, wy;
    const bool colB, colC;
    const R mxc;
    const Coeffs<R> c;
    Stencil<R> sxp, sxn;  // x-differences at this column for sign + / -
    R Pw[9][kRing2];
    R Qw[9][kRing2];
    R Sw[9][kRing2];
    R cur[9], nxt[9];
    int rA;  // logical row of cur (may lie outside [0, ny))
    int y1;

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
    // wall velocities with constant indices only (see step_fused_walls.cu)
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
    __device__ __forceinline__ R dx_of(int i, const R *rw, R v0) const
    {
        return apply_stencil(cx(i) > 0 ? sxp : sxn, cx(i), rw[t - 2], rw[t - 1], v0, rw[t + 1],
                             rw[t + 2]);
    }

    template <int PH>
    __device__ void row(bool load_next, bool doB, bool doC)
    {
        constexpr int p0 = PH;
        constexpr int p1 = (PH + 4) % kRing2;
        constexpr int p2 = (PH + 3) % kRing2;
        constexpr int p3 = (PH + 2) % kRing2;
        constexpr int p4 = (PH + 1) % kRing2;
        const int r = rA;
        if (load_next) load(nxt, r + 1);
        const bool wallcol = wx && (xc == 0 || xc == a.nx - 1);
        // ------------------------------------------------------------ A (row r)
        {
            R Fx, Fy, geq[9], F[9];
            force_at(r, Fx, Fy);
            node_maps<R, FORCE>(c, cur, Fx, Fy, c.half_dt, geq, F);
            R fn[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const R neq = geq[i] - cur[i];
                R p = cur[i] + c.b_phys * neq;  // Eq. 2.52, h = dt
                R q = cur[i] + c.b_til * neq;   // Eq. 2.20
                if (FORCE) {
                    p += c.c_phys * F[i];
                    q += c.c_til * F[i];
                }
                fn[i] = p;
                Pw[i][p0] = p;
                Qw[i][p0] = q;
                if (xslot(i) >= 0) {
                    sm.Q[p0][xslot(i)][t] = q;
                    if (!wallcol) sm.P[p0][xslot(i)][t] = p;
                }
            }
            // Eq. 3.10 for f^n of the wall column next to x_j (this column)
            if (wx && (xc == 1 || xc == a.nx - 2)) {
                R wv[9];
                nee<R, false>(c, fn, R(0), R(0), R(0), uwx_side(xc == 1, 0), uwx_side(xc == 1, 1), wv);
                const int tw = xc == 1 ? t - 1 : t + 1;
#pragma unroll
                for (int i = 0; i < 9; ++i)
                    if (xslot(i) >= 0) sm.P[p0][xslot(i)][tw] = wv[i];
            }
            if (wy && r == 1) {  // the S wall row, into the window slot of row 0
                R wv[9];
                nee<R, false>(c, fn, R(0), R(0), R(0), uwy_side(true, 0), uwy_side(true, 1), wv);
#pragma unroll
                for (int i = 0; i < 9; ++i) Pw[i][p1] = wv[i];
            } else if (wy && r == a.ny - 1) {  // the N wall row, from the window row ny-2
                R pj[9], wv[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) pj[i] = Pw[i][p1];
                nee<R, false>(c, pj, R(0), R(0), R(0), uwy_side(false, 0), uwy_side(false, 1), wv);
#pragma unroll
                for (int i = 0; i < 9; ++i) Pw[i][p0] = wv[i];
            }
        }
        __syncthreads();
        // ------------------------------------------------------------ B (row r-2)
        if (doB) {
            const int rb = r - 2;
            const bool rowin = !wy || (rb >= 1 && rb <= a.ny - 2);
            if (colB && rowin) {
                const R myr = a.my[mem_row(rb)];
                const R hx = c.h * mxc, hy = c.h * myr;  // h = dt
                const Stencil<R> syp = (wy && rb == 1) ? a.stc : a.st;
                const Stencil<R> syn = (wy && rb == a.ny - 2) ? a.stc : a.st;
                R fb[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    R dP = R(0), fbar = Qw[i][p2];
                    if (cx(i) != 0) {
                        dP += mxc * dx_of(i, sm.P[p2][xslot(i)], Pw[i][p2]);
                        fbar -= hx * dx_of(i, sm.Q[p2][xslot(i)], Qw[i][p2]);
                    }
                    if (cy(i) != 0) {
                        const Stencil<R> &sy = cy(i) > 0 ? syp : syn;
                        dP += myr * apply_stencil(sy, cy(i), Pw[i][p4], Pw[i][p3], Pw[i][p2],
                                                  Pw[i][p1], Pw[i][p0]);
                        fbar -= hy * apply_stencil(sy, cy(i), Qw[i][p4], Qw[i][p3], Qw[i][p2],
                                                   Qw[i][p1], Qw[i][p0]);
                    }
                    sm.LN[p0][i][t] = -dP;
                    fb[i] = fbar;
                }
                R Fx, Fy, geq[9], F[9];
                force_at(rb, Fx, Fy);
                node_maps<R, FORCE>(c, fb, Fx, Fy, c.half_h, geq, F);
                R st[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    R v = fb[i] + c.b_star * (geq[i] - fb[i]);  // Eq. 2.52, h = dt
                    if (FORCE) v += c.c_star * F[i];
                    st[i] = v;
                    Sw[i][p0] = v;
                    if (xslot(i) >= 0) sm.S[p0][xslot(i)][t] = v;
                }
                if (wx && (xc == 1 || xc == a.nx - 2)) {
                    R wv[9];
                    nee<R, false>(c, st, R(0), R(0), R(0), uwx_side(xc == 1, 0), uwx_side(xc == 1, 1), wv);
                    const int tw = xc == 1 ? t - 1 : t + 1;
#pragma unroll
                    for (int i = 0; i < 9; ++i)
                        if (xslot(i) >= 0) sm.S[p0][xslot(i)][tw] = wv[i];
                }
                if (wy && rb == 1) {
                    R wv[9];
                    nee<R, false>(c, st, R(0), R(0), R(0), uwy_side(true, 0), uwy_side(true, 1), wv);
#pragma unroll
                    for (int i = 0; i < 9; ++i) Sw[i][p1] = wv[i];
                }
            } else if (colB && wy && rb == a.ny - 1) {
                R sj[9], wv[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) sj[i] = Sw[i][p1];
                nee<R, false>(c, sj, R(0), R(0), R(0), uwy_side(false, 0), uwy_side(false, 1), wv);
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    Sw[i][p0] = wv[i];
                    if (xslot(i) >= 0) sm.S[p0][xslot(i)][t] = wv[i];
                    sm.LN[p0][i][t] = R(0);
                }
            } else {
                // not evaluated here: finite zeros (wall columns keep the value
                // their interior neighbour writes into the ring)
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    Sw[i][p0] = R(0);
                    if (xslot(i) >= 0 && !wallcol) sm.S[p0][xslot(i)][t] = R(0);
                    sm.LN[p0][i][t] = R(0);
                }
            }
        }
        // ------------------------------------------------------------ C (row r-4)
        if (doC) {
            const int rc = r - 4;
            const bool rowin = !wy || (rc >= 1 && rc <= a.ny - 2);
            if (colC && rowin && rc < y1) {
                const R myr = a.my[mem_row(rc)];
                const Stencil<R> syp = (wy && rc == 1) ? a.stc : a.st;
                const Stencil<R> syn = (wy && rc == a.ny - 2) ? a.stc : a.st;
                R out[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    R dS = R(0);
                    if (cx(i) != 0) dS += mxc * dx_of(i, sm.S[p2][xslot(i)], Sw[i][p2]);
                    if (cy(i) != 0)
                        dS += myr * apply_stencil(cy(i) > 0 ? syp : syn, cy(i), Sw[i][p4], Sw[i][p3],
                                                  Sw[i][p2], Sw[i][p1], Sw[i][p0]);
                    out[i] = Qw[i][p4] + c.half_dt * (sm.LN[p2][i][t] - dS);
                }
                const int my_row = mem_row(rc);
                auto put = [&](int x, int y, const R *v) {
                    const size_t o = (size_t)y * a.pitch + x;
#pragma unroll
                    for (int i = 0; i < 9; ++i) a.gout[i * a.plane + o] = v[i];
                };
                put(gx, my_row, out);
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
                        if (bw) put(xw, 0, wv);
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

// One tile of the walls sweep: output columns x0 .. x0 + NT - 9 below xhi,
// rows y0 .. y1 - 1 (periodic axes wrap, walled axes clamp).
template <class R, bool FORCE, int NT>
__device__ __forceinline__ void sweep_tile_s2(const StepArgs<R> &a, Smem2<R, NT> &sm, int x0, int xhi,
                                              int y0, int y1)
{
    const int t = threadIdx.x;
    const int xc = x0 - kHalo2 + t;
    const bool wx = a.bc_x == FDLBM_WALL, wy = a.bc_y == FDLBM_WALL;
    const bool inside = !wx || (xc >= 0 && xc < a.nx);
    const int gx = wx ? min(max(xc, 0), a.nx - 1) : wrap_index(xc, a.nx);
    const bool colint = !wx || (xc >= 1 && xc <= a.nx - 2);
    const bool colB = (t >= 2) && (t < NT - 2) && inside && colint;
    const bool colC = (t >= kHalo2) && (t < NT - kHalo2) && xc < min(a.nx, xhi) && inside && colint;
    SweepS2W<R, FORCE, NT> sw{a,
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
    sw.rA = y0 - kHalo2;
    sw.load(sw.cur, sw.rA);
    const int iters = (y1 - y0) + 2 * kHalo2;
    for (int k = 0; k < iters; k += kRing2) {
        sw.template row<0>(k + 1 < iters, k >= 4, k >= 8);
        if (k + 1 < iters) sw.template row<1>(k + 2 < iters, k + 1 >= 4, k + 1 >= 8);
        if (k + 2 < iters) sw.template row<2>(k + 3 < iters, k + 2 >= 4, k + 2 >= 8);
        if (k + 3 < iters) sw.template row<3>(k + 4 < iters, k + 3 >= 4, k + 3 >= 8);
        if (k + 4 < iters) sw.template row<4>(k + 5 < iters, k + 4 >= 4, k + 4 >= 8);
    }
}

template <class R, bool FORCE, int NT>
__global__ void __launch_bounds__(NT, 2) k_step_fused_s2_walls(const StepArgs<R> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem2<R, NT> &sm = *reinterpret_cast<Smem2<R, NT> *>(smem_raw);
    const int y0 = blockIdx.y * a.rows;
    if (y0 >= a.ny) return;  // uniform over the block
    sweep_tile_s2<R, FORCE, NT>(a, sm, blockIdx.x * (NT - 2 * kHalo2), a.nx, y0, min(y0 + a.rows, a.ny));
}

// Batched: block b is tile (b + blk_off - blk_start[c]) of case c =
// blk_case[b + blk_off]; the T2S2-FDLBM2 cases' tiles follow those of the
// T2S2-FDLBM1 cases in the batch's tables, from blk_off on.  The case's
// arguments are copied into shared memory first.
template <class R, int NT>
__global__ void __launch_bounds__(NT, 2)
    kb_step_fused_s2(const StepArgs<R> *cases, const int *blk_case, const int *blk_start,
                     const int *strips, int blk_off)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem2<R, NT> &sm = *reinterpret_cast<Smem2<R, NT> *>(smem_raw);
    __shared__ __align__(16) unsigned char abuf[sizeof(StepArgs<R>)];
    static_assert(sizeof(StepArgs<R>) % 4 == 0, "argument block is copied as 32-bit words");
    const int b = blockIdx.x + blk_off;
    const int c = blk_case[b];
    {
        const int *src = reinterpret_cast<const int *>(cases + c);
        int *dst = reinterpret_cast<int *>(abuf);
        for (int q = threadIdx.x; q < (int)(sizeof(StepArgs<R>) / 4); q += blockDim.x) dst[q] = src[q];
    }
    __syncthreads();
    const StepArgs<R> &a = *reinterpret_cast<const StepArgs<R> *>(abuf);
    const int lb = b - blk_start[c], ns = strips[c];
    const int y0 = (lb / ns) * a.rows;
    if (y0 >= a.ny) return;  // uniform over the block
    sweep_tile_s2<R, true, NT>(a, sm, (lb % ns) * (NT - 2 * kHalo2), a.nx, y0, min(y0 + a.rows, a.ny));
}

// The frame of a walled FP32 grid whose interior runs the warp-tile kernel
// (T2S2-FDLBM2): this walls sweep in blocks of one warp on the frame tiles.
using FrameSmem2 = Smem2<float, frame::kFrameNT>;

template <bool FORCE>
__global__ void __launch_bounds__(frame::kFrameNT) k_frame_sweep_s2(const FrameGeom g, const StepArgs<float> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FrameSmem2 &sm = *reinterpret_cast<FrameSmem2 *>(smem_raw);
    frame::Tile tile;
    if (frame::frame_tile(g, blockIdx.x, tile) >= 0) return;
    sweep_tile_s2<float, FORCE, frame::kFrameNT>(a, sm, tile.x0, tile.xend, tile.y0, tile.y1);
}

template <class R, bool FORCE>
cudaError_t launch_s2_walls(const StepArgs<R> &a, cudaStream_t s)
{
    constexpr int NT = 128;
    constexpr int W = NT - 2 * kHalo2;
    constexpr size_t smem = sizeof(Smem2<R, NT>);
    cudaError_t e = cudaFuncSetAttribute(k_step_fused_s2_walls<R, FORCE, NT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((a.nx + W - 1) / W, (a.ny + a.rows - 1) / a.rows);
    k_step_fused_s2_walls<R, FORCE, NT><<<grid, NT, smem, s>>>(a);
    return cudaGetLastError();
}

template <class R, bool FORCE>
cudaError_t launch_s2(const StepArgs<R> &a, cudaStream_t s)
{
    constexpr int NT = 128;
    constexpr int W = NT - 2 * kHalo2;
    constexpr size_t smem = sizeof(Smem2<R, NT>);
    cudaError_t e = cudaFuncSetAttribute(k_step_fused_s2<R, FORCE, NT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((a.nx + W - 1) / W, (a.ny + a.rows - 1) / a.rows);
    k_step_fused_s2<R, FORCE, NT><<<grid, NT, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

template <class R>
cudaError_t launch_fused_s2(const StepArgs<R> &a, cudaStream_t s)
{
    if (a.bc_x == FDLBM_WALL || a.bc_y == FDLBM_WALL)
        return a.force ? launch_s2_walls<R, true>(a, s) : launch_s2_walls<R, false>(a, s);
    return a.force ? launch_s2<R, true>(a, s) : launch_s2<R, false>(a, s);
}

template <class R>
int fused_s2_blocks_per_sm()
{
    int n = 0;
    constexpr size_t smem = sizeof(Smem2<R, 128>);
    cudaFuncSetAttribute(k_step_fused_s2<R, false, 128>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_fused_s2<R, false, 128>, 128,
                                                      smem) != cudaSuccess)
        return 0;
    return n;
}

// The T2S2-FDLBM2 tiles of a batch (nblocks of them, from table entry blk_off).
template <class R>
cudaError_t launch_batched_fused_s2(const BatchTables &t, int parity, int blk_off, int nblocks,
                                    cudaStream_t s)
{
    if (nblocks <= 0) return cudaSuccess;
    constexpr int NT = 128;
    constexpr size_t smem = sizeof(Smem2<R, NT>);
    cudaError_t e = cudaFuncSetAttribute(kb_step_fused_s2<R, NT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kb_step_fused_s2<R, NT><<<nblocks, NT, smem, s>>>(
        static_cast<const StepArgs<R> *>(t.args[parity]), t.blk_case, t.blk_start, t.tiles_x,
        blk_off);
    return cudaGetLastError();
}

template cudaError_t launch_batched_fused_s2<float>(const BatchTables &, int, int, int, cudaStream_t);
template cudaError_t launch_batched_fused_s2<double>(const BatchTables &, int, int, int, cudaStream_t);
template cudaError_t launch_fused_s2<float>(const StepArgs<float> &, cudaStream_t);
template cudaError_t launch_fused_s2<double>(const StepArgs<double> &, cudaStream_t);
template int fused_s2_blocks_per_sm<float>();
template int fused_s2_blocks_per_sm<double>();

cudaError_t launch_frame_s2(const FrameGeom &g, const StepArgs<float> &a, cudaStream_t s)
{
    if (g.nframe <= 0) return cudaSuccess;
    constexpr size_t smem = sizeof(FrameSmem2);
    auto kern = a.force ? k_frame_sweep_s2<true> : k_frame_sweep_s2<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<g.nframe, frame::kFrameNT, smem, s>>>(g, a);
    return cudaGetLastError();
}

int frame_s2_blocks_per_sm()
{
    int n = 0;
    constexpr size_t smem = sizeof(FrameSmem2);
    cudaFuncSetAttribute(k_frame_sweep_s2<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_frame_sweep_s2<true>, frame::kFrameNT, smem) !=
        cudaSuccess)
        return 0;
    return n;
}

}  // namespace fdlbm
