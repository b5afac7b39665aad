// Discrete adjoint (reverse mode) of one T2S2-FDLBM1 step on a periodic grid,
// with the body-acceleration field as a differentiable parameter.
//
// Forward step in the terms used here (per node, all populations; see
// step_fused.cu for the equations):
//   A:  P = g + b1 (geq(g) - g) + c1 F(g),  Q = g + b2 (geq(g) - g) + c2 F(g)
//   B:  gs = P - h D(P),  S = gs + b3 (geq(gs) - gs) + c3 F(gs)
//   C:  g' = Q - dt D(S)
// with D_i f = m_x T_x f + m_y T_y f the metric-weighted mixed differences
// (Eqs. 2.36-2.38) and geq, F the node maps of Eqs. 3.2, 3.3, 3.12.  Given the
// cotangent lam' of g', the adjoint is
//   lam_Q = lam',  lam_S = -dt D^T lam'
//   lam_gs = (dS/dgs)^T lam_S                  (node-local)
//   lam_P = lam_gs - h D^T lam_gs
//   lam = (dP/dg)^T lam_P + (dQ/dg)^T lam_Q     (node-local)
// and the force cotangent collects (dS/dF)^T lam_S + (dP/dF)^T lam_P +
// (dQ/dF)^T lam_Q at every node.  The transposed difference gathers from the
// mirrored offsets, with the metric of the node it gathers from:
//   (T^T lam)(k) = sum_j w_j m(k + s j) lam(k + s j).
// Three kernels per step: recompute P; stage B adjoint (needs P and lam' in a
// +-2 neighbourhood); stage A adjoint (needs lam_gs in a +-2 neighbourhood).
#include <algorithm>
#include <type_traits>

#include "adjoint_node.cuh"
#include "internal.h"

namespace fdlbm {
namespace {

// ---------------------------------------------------------------- fused sweep
// One kernel per adjoint step, laid out like the forward sweep (step_fused.cu):
// a CTA of NT threads owns NT - 8 output columns and a segment of rows, thread
// t owns one column, and the sweep runs bottom to top with
//   A' (row r)    load g, lam', F; P = stage A of the forward step
//   B' (row r-2)  gs = P - h D(P); lam_S = -dt D^T lam'; node VJP of stage B
//                 -> lam_gs and the force cotangent of stage B
//   C' (row r-4)  lam_P = lam_gs - h D^T lam_gs; node VJP of stage A with
//                 lam_Q = lam' -> lam (stored) and the force cotangent (added
//                 to dforce in FP64)
// Differences in y read per-thread register windows of five rows; differences
// in x read shared-memory rings written by the neighbouring threads.  The
// transposed x-differences need the metric of the node they gather from, so
// the rings hold lam' m_x and lam_gs m_x, each multiplied by its writer's own
// column metric; the transposed y-differences weight the window rows by a
// window of m_y.  g and the force wait four rows in a per-thread ring for
// stages B' and C'.  The rows of g, lam' and the force arrive two rows ahead
// by asynchronous copies (cp.async) into a three-slot ring, each thread its
// own column, so that no row waits for its loads.
// One barrier per row, as in the forward sweep (5-slot rings, 5-row unroll):
// a ring slot is rewritten five rows after it was written, and every reader
// of it has passed a barrier in between (the copy ring: a slot is refilled one
// row, and one barrier, after its thread read it).

constexpr int kAdjNT = 128;
constexpr int kAdjHalo = 4;
constexpr int kAdjRing = 5;
constexpr int kAdjIn = 3;   // rows of the copy ring: this one and two ahead

template <class R>
struct AdjSmem {
    R P[kAdjRing][6][kAdjNT];   // fbar^{+,h} of the x-moving populations
    R L[kAdjRing][6][kAdjNT];   // lam' m_x of the x-moving populations
    R LG[kAdjRing][6][kAdjNT];  // lam_gs m_x of the x-moving populations
    R G[kAdjRing][11][kAdjNT];  // g and the force (own column only)
    R IN[kAdjIn][20][kAdjNT];   // rows in flight: g, lam', force (own column)
};

// Asynchronous global -> shared copy of one value (cp.async, cached in L1).
template <class R>
__device__ __forceinline__ void copy_async(R *dst, const R *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(src), "n"(sizeof(R)) : "memory");
}
__device__ __forceinline__ void copy_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void copy_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <class R>
struct AdjArgs {
    StepArgs<R> a;       // grid, metrics, coefficients (gin = state g^n)
    const R *lam_next;   // cotangent of g^{n+1}
    R *lam_prev;         // cotangent of g^n (output)
    double *dforce;      // [2][ny][nx] accumulated force cotangent, or nullptr
    int rows;            // tile height of the sweep
};

template <class R, bool FORCE>
__global__ void __launch_bounds__(kAdjNT, sizeof(R) == 4 ? 2 : 1) k_adj_fused(const AdjArgs<R> p)
{
    constexpr int NT = kAdjNT, W = NT - 2 * kAdjHalo;
    const StepArgs<R> &a = p.a;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AdjSmem<R> &sm = *reinterpret_cast<AdjSmem<R> *>(smem_raw);

    const int t = threadIdx.x;
    const int x0 = blockIdx.x * W;
    const int xc = x0 - kAdjHalo + t;
    const int y0 = blockIdx.y * p.rows;
    if (y0 >= a.ny) return;  // uniform over the block
    const int y1 = min(y0 + p.rows, a.ny);
    const int gx = wrap_index(xc, a.nx);
    const bool act1 = (t >= 2) && (t < NT - 2);
    const bool act2 = (t >= kAdjHalo) && (t < NT - kAdjHalo) && (xc < a.nx);
    const Coeffs<R> c = a.c;
    const Stencil<R> st = a.st;
    const R mxc = a.mx[gx];
    const R hx = c.h * mxc;
    const R wgt[4] = {st.wm1, st.w0, st.w1, st.w2};
    const size_t N = (size_t)a.nx * a.ny;

    R Pw[9][kAdjRing];   // P of this column, slot = iteration mod 5
    R Lw[9][kAdjRing];   // lam'
    R Gw[9][kAdjRing];   // lam_gs
    R Mw[kAdjRing];      // m_y of the rows in the windows above
    R Mg[kAdjRing];      // m_y of the rows of Gw
    R fBx[kAdjRing], fBy[kAdjRing];  // force cotangent of stage B, per row
    R gcur[9], lcur[9];
    int rl = wrap_index(y0 - kAdjHalo, a.ny);   // row of gcur / lcur
    int rn = rl;                                // next row to copy
    int rs = wrap_index(y0 - 6, a.ny);          // stage B' row at iteration k: y0 - 6 + k
    int rq = wrap_index(y0 - 8, a.ny);          // stage C' row: y0 - 8 + k
    // row `row` into copy slot `slot` (one commit group per row, empty past
    // the segment, so that the group count stays in step with the rows)
    auto issue = [&](int slot, bool any) {
        if (any) {
            const size_t off = (size_t)rn * a.pitch + gx;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                copy_async(&sm.IN[slot][i][t], a.gin + i * a.plane + off);
                copy_async(&sm.IN[slot][9 + i][t], p.lam_next + i * a.plane + off);
            }
            if (FORCE) {
                copy_async(&sm.IN[slot][18][t], a.force + off);
                copy_async(&sm.IN[slot][19][t], a.force + a.plane + off);
            }
            rn = rn + 1 == a.ny ? 0 : rn + 1;
        }
        copy_commit();
    };
    const int iters = (y1 - y0) + 2 * kAdjHalo;
    issue(0, true);
    issue(1, 1 < iters);

    auto row = [&](auto PHc, int k) {
        constexpr int PH = decltype(PHc)::value;
        constexpr int p0 = PH, p1 = (PH + 4) % 5, p2 = (PH + 3) % 5, p3 = (PH + 2) % 5,
                      p4 = (PH + 1) % 5;
        const int rA = rl;
        rl = rl + 1 == a.ny ? 0 : rl + 1;
        // the row two ahead into the slot read one row ago; then this row's
        const int slot = k % kAdjIn;
        issue((k + 2) % kAdjIn, k + 2 < iters);
        copy_wait<2>();
        R Fx = R(0), Fy = R(0);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            gcur[i] = sm.IN[slot][i][t];
            lcur[i] = sm.IN[slot][9 + i][t];
        }
        if (FORCE) {
            Fx = sm.IN[slot][18][t];
            Fy = sm.IN[slot][19][t];
        }
        const int rB = rs, rC = rq;
        rs = rs + 1 == a.ny ? 0 : rs + 1;
        rq = rq + 1 == a.ny ? 0 : rq + 1;
        const bool doC = k >= 8 && act2;
        const size_t nC = (size_t)rC * a.nx + xc;
        double dFx = 0.0, dFy = 0.0;
        if (p.dforce && doC) {
            dFx = p.dforce[nC];
            dFy = p.dforce[N + nC];
        }
        // ------------------------------------------------------------ A' (row r)
        {
            R drho, jx, jy;
            moments_dev(gcur, drho, jx, jy);
            const R rho = c.rho0 + drho;
            jx += c.half_dt * rho * Fx;
            jy += c.half_dt * rho * Fy;
            const R inv = node_recip(rho);
            const R ux = jx * inv, uy = jy * inv;
            R geq[9], F[9];
            equilibrium_dev_j(drho, jx, jy, inv, geq);
            if (FORCE) force_terms(c.rho0, geq, ux, uy, Fx, Fy, F);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                R P = gcur[i] + c.b_bar * (geq[i] - gcur[i]);
                if (FORCE) P += c.c_bar * F[i];
                Pw[i][p0] = P;
                Lw[i][p0] = lcur[i];
                sm.G[p0][i][t] = gcur[i];
                if (FORCE && i == 0) {
                    sm.G[p0][9][t] = Fx;
                    sm.G[p0][10][t] = Fy;
                }
                if (xslot(i) >= 0) {
                    sm.P[p0][xslot(i)][t] = P;
                    sm.L[p0][xslot(i)][t] = lcur[i] * mxc;
                }
            }
            Mw[p0] = a.my[rA];
        }
        __syncthreads();
        // ------------------------------------------------------------ B' (row r-2)
        // rows r-4 .. r sit in slots p4, p3, p2, p1, p0 of Pw, Lw and Mw
        if (k >= 4 && act1) {
            const R hy = c.h * Mw[p2];
            // transposed y weights: sign +: rows r-3, r-2, r-1, r (j = -1..2 at
            // rows rB + j); sign -: rows r-1, r-2, r-3, r-4 (rows rB - j)
            const R yp[4] = {wgt[0] * Mw[p3], wgt[1] * Mw[p2], wgt[2] * Mw[p1], wgt[3] * Mw[p0]};
            const R ym[4] = {wgt[0] * Mw[p1], wgt[1] * Mw[p2], wgt[2] * Mw[p3], wgt[3] * Mw[p4]};
            R gs[9], lS[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const R v0 = Pw[i][p2];
                R acc = v0, lt = R(0);
                if (cx(i) != 0) {
                    const R *rw = sm.P[p2][xslot(i)];
                    acc -= hx * apply_stencil(st, cx(i), rw[t - 2], rw[t - 1], v0, rw[t + 1], rw[t + 2]);
                    const R *lw = sm.L[p2][xslot(i)];
                    const int s = cx(i);
                    // sum_j w_j (lam' m_x)(x + s j), j = -1 .. 2
                    lt += wgt[0] * lw[t - s] + wgt[1] * lw[t] + wgt[2] * lw[t + s] + wgt[3] * lw[t + 2 * s];
                }
                if (cy(i) != 0) {
                    acc -= hy * apply_stencil(st, cy(i), Pw[i][p4], Pw[i][p3], v0, Pw[i][p1], Pw[i][p0]);
                    if (cy(i) > 0)
                        lt += yp[0] * Lw[i][p3] + yp[1] * Lw[i][p2] + yp[2] * Lw[i][p1] + yp[3] * Lw[i][p0];
                    else
                        lt += ym[0] * Lw[i][p1] + ym[1] * Lw[i][p2] + ym[2] * Lw[i][p3] + ym[3] * Lw[i][p4];
                }
                gs[i] = acc;
                lS[i] = -c.dt * lt;
            }
            R Fx = R(0), Fy = R(0);
            if (FORCE) {
                Fx = sm.G[p2][9][t];
                Fy = sm.G[p2][10][t];
            }
            NodeMap<R> m;
            m.eval(gs, c.rho0, Fx, Fy, c.half_h);
            R lgeq[9], lF[9], lg[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                lgeq[i] = c.b_star * lS[i];
                lF[i] = c.c_star * lS[i];
                lg[i] = (R(1) - c.b_star) * lS[i];
            }
            R lFx = R(0), lFy = R(0);
            m.vjp(lgeq, lF, Fx, Fy, c.half_h, lg, lFx, lFy);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                Gw[i][p0] = lg[i];
                if (xslot(i) >= 0) sm.LG[p0][xslot(i)][t] = lg[i] * mxc;
            }
            fBx[p0] = lFx;
            fBy[p0] = lFy;
        }
        Mg[p0] = Mw[p2];
        // ------------------------------------------------------------ C' (row r-4)
        // (the lam_gs ring slot read here was written two rows ago, before the
        // barrier of the previous row; no second barrier is needed)
        // lam_gs rows r-6 .. r-2 sit in slots p4, p3, p2, p1, p0 of Gw and Mg;
        // lam' of row r-4 in slot p4 of Lw; g of row r-4 in ring slot p4
        if (doC) {
            const R hyg = c.h;
            const R yp[4] = {wgt[0] * Mg[p3], wgt[1] * Mg[p2], wgt[2] * Mg[p1], wgt[3] * Mg[p0]};
            const R ym[4] = {wgt[0] * Mg[p1], wgt[1] * Mg[p2], wgt[2] * Mg[p3], wgt[3] * Mg[p4]};
            R lP[9], lQ[9], g[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                R lt = R(0);
                if (cx(i) != 0) {
                    const R *lw = sm.LG[p2][xslot(i)];
                    const int s = cx(i);
                    lt += wgt[0] * lw[t - s] + wgt[1] * lw[t] + wgt[2] * lw[t + s] + wgt[3] * lw[t + 2 * s];
                }
                if (cy(i) != 0) {
                    if (cy(i) > 0)
                        lt += yp[0] * Gw[i][p3] + yp[1] * Gw[i][p2] + yp[2] * Gw[i][p1] + yp[3] * Gw[i][p0];
                    else
                        lt += ym[0] * Gw[i][p1] + ym[1] * Gw[i][p2] + ym[2] * Gw[i][p3] + ym[3] * Gw[i][p4];
                }
                lP[i] = Gw[i][p2] - hyg * lt;
                lQ[i] = Lw[i][p4];
                g[i] = sm.G[p4][i][t];
            }
            R Fx = R(0), Fy = R(0);
            if (FORCE) {
                Fx = sm.G[p4][9][t];
                Fy = sm.G[p4][10][t];
            }
            NodeMap<R> m;
            m.eval(g, c.rho0, Fx, Fy, c.half_dt);
            R lgeq[9], lF[9], lg[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                lgeq[i] = c.b_bar * lP[i] + c.b_til * lQ[i];
                lF[i] = c.c_bar * lP[i] + c.c_til * lQ[i];
                lg[i] = (R(1) - c.b_bar) * lP[i] + (R(1) - c.b_til) * lQ[i];
            }
            R lFx = R(0), lFy = R(0);
            m.vjp(lgeq, lF, Fx, Fy, c.half_dt, lg, lFx, lFy);
            const size_t off = (size_t)rC * a.pitch + xc;
#pragma unroll
            for (int i = 0; i < 9; ++i) p.lam_prev[i * a.plane + off] = lg[i];
            if (p.dforce) {
                p.dforce[nC] = dFx + (double(lFx) + double(fBx[p2]));
                p.dforce[N + nC] = dFy + (double(lFy) + double(fBy[p2]));
            }
        }
    };
    for (int k = 0; k < iters; k += 5) {
        row(std::integral_constant<int, 0>{}, k);
        if (k + 1 < iters) row(std::integral_constant<int, 1>{}, k + 1);
        if (k + 2 < iters) row(std::integral_constant<int, 2>{}, k + 2);
        if (k + 3 < iters) row(std::integral_constant<int, 3>{}, k + 3);
        if (k + 4 < iters) row(std::integral_constant<int, 4>{}, k + 4);
    }
}

template <class R>
int adj_blocks_per_sm(bool force)
{
    int n = 0;
    const size_t smem = sizeof(AdjSmem<R>);
    auto fn = force ? k_adj_fused<R, true> : k_adj_fused<R, false>;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, kAdjNT, smem) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

// Tile height minimising (waves) x (rows + 8), as for the forward sweep.
int adj_rows(int nx, int ny, int per_sm)
{
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long slots = (long long)per_sm * sms;
    const long long strips = (nx + (kAdjNT - 2 * kAdjHalo) - 1) / (kAdjNT - 2 * kAdjHalo);
    int best = std::min(ny, 64);
    double best_cost = 1e300;
    for (int rows = 1; rows <= std::min(ny, 512); ++rows) {
        const long long ctas = strips * ((ny + rows - 1) / rows);
        const double cost = (double)((ctas + slots - 1) / slots) * (rows + 8);
        if (cost < best_cost - 1e-9) {
            best_cost = cost;
            best = rows;
        }
    }
    return std::max(1, std::min(best, ny));
}

template <class R>
__device__ __forceinline__ R force_at(const StepArgs<R> &a, int c, size_t o)
{
    return a.force ? a.force[c * a.plane + o] : R(0);
}

// Cotangent of the state from a cotangent du of the velocity of Eq. 3.3:
// u = (j + dt/2 rho F)/rho, so du/dg_i = (xi_i + dt/2 F - u)/rho and
// du/dF = dt/2.
template <class R>
__global__ void k_moments_vjp(const StepArgs<R> a, const double *du, R *lam, double *dforce)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    const size_t o = (size_t)y * a.pitch + x, n = (size_t)y * a.nx + x, N = (size_t)a.nx * a.ny;
    R g[9], drho, jx, jy;
#pragma unroll
    for (int i = 0; i < 9; ++i) g[i] = a.gin[i * a.plane + o];
    moments_dev(g, drho, jx, jy);
    const R rho = a.c.rho0 + drho;
    const R Fx = force_at(a, 0, o), Fy = force_at(a, 1, o);
    const R ux = (jx + a.c.half_dt * rho * Fx) / rho, uy = (jy + a.c.half_dt * rho * Fy) / rho;
    const R wx = R(du[n]), wy = R(du[N + n]);
#pragma unroll
    for (int i = 0; i < 9; ++i)
        lam[i * a.plane + o] =
            ((R(cx(i)) + a.c.half_dt * Fx - ux) * wx + (R(cy(i)) + a.c.half_dt * Fy - uy) * wy) / rho;
    if (dforce) {
        dforce[n] += double(a.c.half_dt * wx);
        dforce[N + n] += double(a.c.half_dt * wy);
    }
}

// Cotangents of the fields of the equilibrium initialisation, as written by
// k_init without the gradient term of Eq. 3.5: the physical f = f^eq (Eq. 3.2)
// and f~ = f - (dt/2) F_i (Eq. 2.19 with the forcing term of Eq. 3.12).  With
// e = xi_i.u, Phi_i = 3e + 4.5e^2 - 1.5u.u, E_i = w_i rho (1 + Phi_i) and
// q_i = 1.5 dt Fbar.(xi_i - u) (so that (dt/2) F_i = q_i E_i),
//   g_i = w_i [(rho - rho0) + rho Phi_i] - q_i E_i,
//   dg_i/drho  = w_i (1 + Phi_i)(1 - q_i),
//   dg_i/du_a  = w_i rho dPhi_i/du_a (1 - q_i) + 1.5 dt Fbar_a E_i,
//   dg_i/dFbar_a = -1.5 dt (xi_ia - u_a) E_i,
// with dPhi_i/du_a = (3 + 9e) xi_ia - 3 u_a.  Under the incompressible
// equilibrium rho0 replaces rho in the velocity terms and in E_i, and
// dg_i/drho = w_i.  The cotangents are added, in FP64.
template <class R>
__global__ void k_init_vjp(const StepArgs<R> a, const double *rho, const double *ux,
                           const double *uy, const R *lam, double dt, double *drho, double *dux,
                           double *duy, double *dforce)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    const size_t o = (size_t)y * a.pitch + x, n = (size_t)y * a.nx + x;
    const size_t N = (size_t)a.nx * a.ny;
    const double r = rho[n], u = ux[n], v = uy[n];
    const double rm = a.c.incomp ? double(a.c.rho0) : r;  // the density of the velocity terms
    const double Fx = a.force ? double(a.force[o]) : 0.0;
    const double Fy = a.force ? double(a.force[a.plane + o]) : 0.0;
    const double hq = 1.5 * dt;  // (dt/2) / cs^2
    const double uu = u * u + v * v;
    double gr = 0.0, gu = 0.0, gv = 0.0, gfx = 0.0, gfy = 0.0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const double w = wq<double>(i);
        const double l = double(lam[i * a.plane + o]);
        const double e = double(cx(i)) * u + double(cy(i)) * v;
        const double phi = e * (3.0 + 4.5 * e) - 1.5 * uu;
        const double E = w * rm * (1.0 + phi);
        const double q = hq * ((double(cx(i)) - u) * Fx + (double(cy(i)) - v) * Fy);
        gr += l * (a.c.incomp ? w : w * (1.0 + phi) * (1.0 - q));
        const double de = rm * (3.0 + 9.0 * e);
        gu += l * (w * (de * double(cx(i)) - 3.0 * rm * u) * (1.0 - q) + hq * Fx * E);
        gv += l * (w * (de * double(cy(i)) - 3.0 * rm * v) * (1.0 - q) + hq * Fy * E);
        gfx -= l * hq * (double(cx(i)) - u) * E;
        gfy -= l * hq * (double(cy(i)) - v) * E;
    }
    if (drho) drho[n] += gr;
    dux[n] += gu;
    duy[n] += gv;
    if (dforce) {
        dforce[n] += gfx;
        dforce[N + n] += gfy;
    }
}

}  // namespace

template <class R>
cudaError_t launch_init_vjp(const StepArgs<R> &a, const double *rho, const double *ux,
                            const double *uy, const R *lam, double dt, double *drho, double *dux,
                            double *duy, double *dforce, cudaStream_t s)
{
    const dim3 blk(32, 8), grd((a.nx + 31) / 32, (a.ny + 7) / 8);
    k_init_vjp<R><<<grd, blk, 0, s>>>(a, rho, ux, uy, lam, dt, drho, dux, duy, dforce);
    return cudaGetLastError();
}

template cudaError_t launch_init_vjp<float>(const StepArgs<float> &, const double *, const double *,
                                            const double *, const float *, double, double *,
                                            double *, double *, double *, cudaStream_t);
template cudaError_t launch_init_vjp<double>(const StepArgs<double> &, const double *,
                                             const double *, const double *, const double *, double,
                                             double *, double *, double *, double *, cudaStream_t);

template <class R>
cudaError_t launch_adjoint(const StepArgs<R> &a, const R *lam_next, R *lam_prev, R *, R *,
                           double *, double *dforce, cudaStream_t s)
{
    const bool force = a.force != nullptr;
    AdjArgs<R> p{a, lam_next, lam_prev, dforce, adj_rows(a.nx, a.ny, adj_blocks_per_sm<R>(force))};
    const size_t smem = sizeof(AdjSmem<R>);
    const dim3 grid((a.nx + kAdjNT - 2 * kAdjHalo - 1) / (kAdjNT - 2 * kAdjHalo),
                    (a.ny + p.rows - 1) / p.rows);
    auto fn = force ? k_adj_fused<R, true> : k_adj_fused<R, false>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, kAdjNT, smem, s>>>(p);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_moments_vjp(const StepArgs<R> &a, const double *du, R *lam, double *dforce,
                               cudaStream_t s)
{
    const dim3 blk(32, 8), grd((a.nx + 31) / 32, (a.ny + 7) / 8);
    k_moments_vjp<R><<<grd, blk, 0, s>>>(a, du, lam, dforce);
    return cudaGetLastError();
}

template cudaError_t launch_adjoint<float>(const StepArgs<float> &, const float *, float *, float *,
                                           float *, double *, double *, cudaStream_t);
template cudaError_t launch_adjoint<double>(const StepArgs<double> &, const double *, double *,
                                            double *, double *, double *, double *, cudaStream_t);
template cudaError_t launch_moments_vjp<float>(const StepArgs<float> &, const double *, float *,
                                               double *, cudaStream_t);
template cudaError_t launch_moments_vjp<double>(const StepArgs<double> &, const double *, double *,
                                                double *, cudaStream_t);

}  // namespace fdlbm
