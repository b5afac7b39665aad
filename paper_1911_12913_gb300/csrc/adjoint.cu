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
#include "internal.h"

namespace fdlbm {
namespace {

// Node map of stage A or B: moments (with force shift `sh`), equilibrium and
// forcing, and the derivatives needed by its vector-Jacobian product.
template <class R>
struct NodeMap {
    R drho, rho, ux, uy, eu[9], t[9], feq[9], s[9];

    __device__ void eval(const R g[9], R rho0, R Fx, R Fy, R sh)
    {
        R jx, jy;
        moments_dev(g, drho, jx, jy);
        rho = rho0 + drho;
        jx += sh * rho * Fx;
        jy += sh * rho * Fy;
        ux = jx / rho;
        uy = jy / rho;
        const R usq = R(1.5) * (ux * ux + uy * uy);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            eu[i] = xi_dot<R>(i, ux, uy);
            t[i] = eu[i] * (R(3) + R(4.5) * eu[i]) - usq;
            feq[i] = wq<R>(i) * rho0 + wq<R>(i) * (drho + rho * t[i]);
            s[i] = (R(cx(i)) - ux) * Fx + (R(cy(i)) - uy) * Fy;
        }
    }

    // Given lam_geq and lam_F (per population), add the cotangent of g (lam_g)
    // and of the force (lFx, lFy).
    __device__ void vjp(const R lgeq_in[9], const R lF[9], R Fx, R Fy, R sh, R lam_g[9], R &lFx,
                        R &lFy) const
    {
        R lux = R(0), luy = R(0), lrho = R(0), ldrho = R(0), lusq = R(0);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            // F_i = 3 s_i feq_i
            const R lgeq = lgeq_in[i] + R(3) * s[i] * lF[i];
            const R ls = R(3) * feq[i] * lF[i];
            lux -= Fx * ls;
            luy -= Fy * ls;
            lFx += (R(cx(i)) - ux) * ls;
            lFy += (R(cy(i)) - uy) * ls;
            // geq_i = w_i (drho + rho t_i), t_i = eu_i (3 + 4.5 eu_i) - usq
            ldrho += wq<R>(i) * lgeq;
            lrho += wq<R>(i) * t[i] * lgeq;
            const R lt = wq<R>(i) * rho * lgeq;
            const R leu = (R(3) + R(9) * eu[i]) * lt;
            lusq -= lt;
            lux += R(cx(i)) * leu;
            luy += R(cy(i)) * leu;
        }
        // usq = 1.5 (ux^2 + uy^2)
        lux += R(3) * ux * lusq;
        luy += R(3) * uy * lusq;
        // u = j'/rho, j' = j + sh rho F
        const R ljx = lux / rho, ljy = luy / rho;
        lrho -= (ux * lux + uy * luy) / rho;
        lrho += sh * (Fx * ljx + Fy * ljy);
        lFx += sh * rho * ljx;
        lFy += sh * rho * ljy;
        ldrho += lrho;
#pragma unroll
        for (int i = 0; i < 9; ++i) lam_g[i] += ldrho + R(cx(i)) * ljx + R(cy(i)) * ljy;
    }
};

template <class R>
struct AdjArgs {
    StepArgs<R> a;       // grid, metrics, coefficients (gin = state g^n)
    const R *lam_next;   // cotangent of g^{n+1}
    R *lam_prev;         // cotangent of g^n (output)
    R *P;                // recomputed fbar^{+,h}
    R *lgs;              // cotangent of gs
    double *fB;          // [2][N] force cotangent of stage B (scratch)
    double *dforce;      // [2][ny][nx] accumulated force cotangent, or nullptr
};

template <class R>
__device__ __forceinline__ R force_at(const StepArgs<R> &a, int c, size_t o)
{
    return a.force ? a.force[c * a.plane + o] : R(0);
}

// D_i f at (x, y) on a periodic grid.
template <class R>
__device__ R dop(const StepArgs<R> &a, const R *fld, int i, int x, int y)
{
    R out = R(0);
    if (cx(i) != 0) {
        const int s = cx(i);
        const R *row = fld + (size_t)y * a.pitch;
        auto at = [&](int d) { return row[wrap_index(x + d, a.nx)]; };
        out += a.mx[x] * apply_stencil(a.st, s, at(-2), at(-1), at(0), at(1), at(2));
    }
    if (cy(i) != 0) {
        const int s = cy(i);
        auto at = [&](int d) { return fld[(size_t)wrap_index(y + d, a.ny) * a.pitch + x]; };
        out += a.my[y] * apply_stencil(a.st, s, at(-2), at(-1), at(0), at(1), at(2));
    }
    return out;
}

// D_i^T lam at (x, y): sum_j w_j m(k + s j) lam(k + s j) along each axis, with
// w_{-1}, w_0, w_1, w_2 the weights of sign(c) * D_m (lattice.cuh).
template <class R>
__device__ R dop_t(const StepArgs<R> &a, const R *lam, int i, int x, int y)
{
    R out = R(0);
    const R w[4] = {a.st.wm1, a.st.w0, a.st.w1, a.st.w2};
    if (cx(i) != 0) {
        const int s = cx(i);
        const R *row = lam + (size_t)y * a.pitch;
#pragma unroll
        for (int j = -1; j <= 2; ++j) {
            const int xx = wrap_index(x + s * j, a.nx);
            out += w[j + 1] * a.mx[xx] * row[xx];
        }
    }
    if (cy(i) != 0) {
        const int s = cy(i);
#pragma unroll
        for (int j = -1; j <= 2; ++j) {
            const int yy = wrap_index(y + s * j, a.ny);
            out += w[j + 1] * a.my[yy] * lam[(size_t)yy * a.pitch + x];
        }
    }
    return out;
}

// Recompute P = fbar^{+,h}(g^n) at every node.
template <class R>
__global__ void k_adj_recompute(const AdjArgs<R> p)
{
    const StepArgs<R> &a = p.a;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    const size_t o = (size_t)y * a.pitch + x;
    R g[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) g[i] = a.gin[i * a.plane + o];
    const R Fx = force_at(a, 0, o), Fy = force_at(a, 1, o);
    NodeMap<R> m;
    m.eval(g, a.c.rho0, Fx, Fy, a.c.half_dt);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const R geq = m.feq[i] - wq<R>(i) * a.c.rho0;
        const R F = R(3) * m.s[i] * m.feq[i];
        p.P[i * a.plane + o] = g[i] + a.c.b_bar * (geq - g[i]) + a.c.c_bar * F;
    }
}

// Stage B adjoint at every node: lam_S = -dt D^T lam', gs = P - h D(P),
// lam_gs = (dS/dgs)^T lam_S, force cotangent of stage B.
template <class R>
__global__ void k_adj_stage_b(const AdjArgs<R> p)
{
    const StepArgs<R> &a = p.a;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    const size_t o = (size_t)y * a.pitch + x;
    R gs[9], lS[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        gs[i] = p.P[i * a.plane + o] - a.c.h * dop(a, p.P + i * a.plane, i, x, y);
        lS[i] = -a.c.dt * dop_t(a, p.lam_next + i * a.plane, i, x, y);
    }
    const R Fx = force_at(a, 0, o), Fy = force_at(a, 1, o);
    NodeMap<R> m;
    m.eval(gs, a.c.rho0, Fx, Fy, a.c.half_h);
    R lgeq[9], lF[9], lg[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        lgeq[i] = a.c.b_star * lS[i];
        lF[i] = a.c.c_star * lS[i];
        lg[i] = (R(1) - a.c.b_star) * lS[i];
    }
    R lFx = R(0), lFy = R(0);
    m.vjp(lgeq, lF, Fx, Fy, a.c.half_h, lg, lFx, lFy);
#pragma unroll
    for (int i = 0; i < 9; ++i) p.lgs[i * a.plane + o] = lg[i];
    const size_t n = (size_t)y * a.nx + x, N = (size_t)a.nx * a.ny;
    p.fB[n] = double(lFx);
    p.fB[N + n] = double(lFy);
}

// Stage A adjoint at every node: lam_P = lam_gs - h D^T lam_gs, lam_Q = lam',
// lam = (dP/dg)^T lam_P + (dQ/dg)^T lam_Q; accumulate the force cotangent.
template <class R>
__global__ void k_adj_stage_a(const AdjArgs<R> p)
{
    const StepArgs<R> &a = p.a;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    const size_t o = (size_t)y * a.pitch + x;
    R g[9], lP[9], lQ[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        g[i] = a.gin[i * a.plane + o];
        lP[i] = p.lgs[i * a.plane + o] - a.c.h * dop_t(a, p.lgs + i * a.plane, i, x, y);
        lQ[i] = p.lam_next[i * a.plane + o];
    }
    const R Fx = force_at(a, 0, o), Fy = force_at(a, 1, o);
    NodeMap<R> m;
    m.eval(g, a.c.rho0, Fx, Fy, a.c.half_dt);
    R lgeq[9], lF[9], lg[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        lgeq[i] = a.c.b_bar * lP[i] + a.c.b_til * lQ[i];
        lF[i] = a.c.c_bar * lP[i] + a.c.c_til * lQ[i];
        lg[i] = (R(1) - a.c.b_bar) * lP[i] + (R(1) - a.c.b_til) * lQ[i];
    }
    R lFx = R(0), lFy = R(0);
    m.vjp(lgeq, lF, Fx, Fy, a.c.half_dt, lg, lFx, lFy);
#pragma unroll
    for (int i = 0; i < 9; ++i) p.lam_prev[i * a.plane + o] = lg[i];
    if (p.dforce) {
        const size_t n = (size_t)y * a.nx + x, N = (size_t)a.nx * a.ny;
        p.dforce[n] += double(lFx) + p.fB[n];
        p.dforce[N + n] += double(lFy) + p.fB[N + n];
    }
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

}  // namespace

template <class R>
cudaError_t launch_adjoint(const StepArgs<R> &a, const R *lam_next, R *lam_prev, R *P, R *lgs,
                           double *fB, double *dforce, cudaStream_t s)
{
    AdjArgs<R> p{a, lam_next, lam_prev, P, lgs, fB, dforce};
    const dim3 blk(32, 8), grd((a.nx + 31) / 32, (a.ny + 7) / 8);
    k_adj_recompute<R><<<grd, blk, 0, s>>>(p);
    k_adj_stage_b<R><<<grd, blk, 0, s>>>(p);
    k_adj_stage_a<R><<<grd, blk, 0, s>>>(p);
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
