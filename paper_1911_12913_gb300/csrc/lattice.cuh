// D2Q9 lattice and node-local arithmetic of the T2S2-FDLBM, device side.
//
// Distributions are stored as deviations from the rest equilibrium,
// g_i = f~_i - w_i rho0.  The transforms of the scheme are affine with
// coefficients that sum to one (Eqs. 2.20, 2.32, 2.34), and the differences
// annihilate constants, so every step carries over to g unchanged; in FP32 this
// keeps the small O(u) part of f~ away from the O(1) rest value.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

namespace fdlbm {

// Velocity set of Sec. 3 with xi = 1 (population order 0..8 of the paper).
__host__ __device__ constexpr int cx(int i)
{
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cy(int i)
{
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
// Weights 4/9, 1/9, 1/36 (Sec. 3).
template <class R>
__host__ __device__ constexpr R wq(int i)
{
    return i == 0 ? R(4) / R(9) : (i < 5 ? R(1) / R(9) : R(1) / R(36));
}

// Populations with a nonzero x (y) velocity and their slot in compact arrays.
__host__ __device__ constexpr int xslot(int i)
{
    return i == 1 ? 0 : i == 3 ? 1 : i == 5 ? 2 : i == 6 ? 3 : i == 7 ? 4 : i == 8 ? 5 : -1;
}
__host__ __device__ constexpr int yslot(int i)
{
    return i == 2 ? 0 : i == 4 ? 1 : i == 5 ? 2 : i == 6 ? 3 : i == 7 ? 4 : i == 8 ? 5 : -1;
}

// xi_i . u with the zero/sign cases folded at compile time (i is unrolled).
template <class R>
__device__ __forceinline__ R xi_dot(int i, R ux, R uy)
{
    if (cx(i) == 0 && cy(i) == 0) return R(0);
    if (cx(i) == 0) return cy(i) > 0 ? uy : -uy;
    if (cy(i) == 0) return cx(i) > 0 ? ux : -ux;
    return (cx(i) > 0 ? ux : -ux) + (cy(i) > 0 ? uy : -uy);
}

// Zeroth and first moments of a deviation vector: sum g, sum xi g.
template <class R>
__device__ __forceinline__ void moments_dev(const R g[9], R &drho, R &jx, R &jy)
{
    drho = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
    jx = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]);
    jy = (g[2] - g[4]) + (g[5] + g[6]) - (g[7] + g[8]);
}

// Eq. 3.2 with cs^2 = 1/3 as a deviation from w_i rho0:
//   f_i^eq - w_i rho0 = w_i [ (rho - rho0) + rho (3 xi.u + 4.5 (xi.u)^2 - 1.5 u.u) ].
template <class R>
__device__ __forceinline__ void equilibrium_dev(R drho, R rho, R ux, R uy, R geq[9])
{
    const R usq = R(1.5) * (ux * ux + uy * uy);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const R eu = xi_dot<R>(i, ux, uy);
        geq[i] = wq<R>(i) * (drho + rho * (eu * (R(3) + R(4.5) * eu) - usq));
    }
}

// The same deviation from the momentum j = rho u (with any force shift of
// Eq. 3.3 already in it) and inv = 1/rho, or 1/rho0 under the incompressible
// equilibrium (whose velocity terms rho0 (3 xi.u + 4.5 (xi.u)^2 - 1.5 u.u) are
// the same expression in j = rho0 u):
//   f_i^eq - w_i rho0 = w_i [ drho + 3 e_i + (4.5 e_i^2 - 1.5 j.j) inv ],  e_i = xi_i.j.
// Only the quadratic term needs 1/rho, and opposite velocities share it.  The
// linear coefficients 3 w_i are c1 = fl(1/3) (axis velocities) and c2 =
// (1 - 2 c1)/4 (diagonals): 2 c1 + 4 c2 = 1 exactly, so the first moment of
// the equilibrium is j with no rounding bias (a fixed bias would act like a
// force proportional to u, which a slowly decaying flow accumulates).
template <class R>
struct LinearCoef {
    static constexpr R c1 = R(1) / R(3);
    static constexpr R c2 = (R(1) - R(2) * c1) * R(0.25);
};

template <class R>
__device__ __forceinline__ void equilibrium_dev_j(R drho, R jx, R jy, R inv, R geq[9])
{
    const R qn = R(-1.5) * (jx * jx + jy * jy);
    geq[0] = wq<R>(0) * (drho + qn * inv);
    auto pair = [&](R e, R w, R c, int ip, int im) {
        const R ws = w * (drho + (R(4.5) * e * e + qn) * inv);
        const R lin = c * e;
        geq[ip] = ws + lin;
        geq[im] = ws - lin;
    };
    pair(jx, wq<R>(1), LinearCoef<R>::c1, 1, 3);
    pair(jy, wq<R>(2), LinearCoef<R>::c1, 2, 4);
    pair(jx + jy, wq<R>(5), LinearCoef<R>::c2, 5, 7);
    pair(jy - jx, wq<R>(6), LinearCoef<R>::c2, 6, 8);
}

// 1/rho for the momentum-form equilibrium, where it scales only the O(u^2)
// quadratic term, so a reciprocal within a few ulp serves.  FP32: the
// hardware approximation (about one ulp for normal x).  FP64: the same
// instruction's FP64 form as a seed, refined by two Newton-Raphson steps for
// f(y) = 1/y - x, y <- y + y (1 - x y), each of which squares the relative
// error (e.g. J.-M. Muller et al., Handbook of Floating-Point Arithmetic,
// division by Newton-Raphson iteration); the density is O(1) and finite.
template <class R>
__device__ __forceinline__ R node_reciprocal(R x);

template <>
__device__ __forceinline__ float node_reciprocal<float>(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <>
__device__ __forceinline__ double node_reciprocal<double>(double x)
{
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
#pragma unroll
    for (int k = 0; k < 2; ++k) y = fma(y, fma(-x, y, 1.0), y);
    return y;
}

// Eq. 3.12: F_i = Fbar.(xi_i - u) f_i^eq / cs^2, with f_i^eq = w_i rho0 + geq_i
// - w_i dshift.  dshift = 0 takes the equilibrium of the node (Eq. 3.2); under
// the incompressible equilibrium dshift = rho - rho0, which takes it at rho0.
template <class R>
__device__ __forceinline__ void force_terms(R rho0, const R geq[9], R ux, R uy, R Fx, R Fy,
                                            R F[9], R dshift = R(0))
{
    const R base = -(ux * Fx + uy * Fy);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const R xf = base + xi_dot<R>(i, Fx, Fy);
        F[i] = R(3) * xf * (wq<R>(i) * (rho0 - dshift) + geq[i]);
    }
}

// Mixed difference of Eq. 2.36 (blend beta = upwind weight) in the index
// coordinate, pre-multiplied by the sign of the velocity component:
//   sign(c) * D_m f(k) = sum_j w_j f(k - sign(c) * j),   j = -1, 0, 1, 2,
// w_{-1} = (1-beta)/2, w_0 = 3 beta/2, w_1 = -(1-beta)/2 - 2 beta, w_2 = beta/2.
// (Central part Eq. 2.37, second-order upwind part Eq. 2.38 and its mirror.)
template <class R>
struct Stencil {
    R wm1, w0, w1, w2;
};

// The weights sum to zero, so the difference of a constant vanishes and the
// update conserves mass and momentum on a periodic uniform grid.  Rounded
// separately they would not (for beta = 0.1 in FP32 the sum is 1.9e-8), and
// every step would then scale each moving population by 1 - CFL x that sum: a
// damping that adds up linearly over a long run.  So the weights are put on a
// grid of 2^-22 (FP32) or 2^-51 (FP64), fine enough to move beta by no more
// than that, and coarse enough that w0 = -(wm1 + w1 + w2) and every partial sum
// are exact (|w| <= 2).
template <class R>
__host__ inline Stencil<R> make_stencil(double beta)
{
    const double g = sizeof(R) == 4 ? 4194304.0 : 2251799813685248.0;  // 2^22, 2^51
    auto on_grid = [g](double v) { return std::nearbyint(v * g) / g; };
    const double wm1 = on_grid(0.5 * (1.0 - beta));
    const double w1 = on_grid(-0.5 * (1.0 - beta) - 2.0 * beta);
    const double w2 = on_grid(0.5 * beta);
    Stencil<R> s;
    s.wm1 = R(wm1);
    s.w1 = R(w1);
    s.w2 = R(w2);
    s.w0 = R(-(wm1 + w1 + w2));
    return s;
}

// Products s w of a weight (|w| <= 2) and a scale s != 0 (for instance -dt m)
// rounded to a multiple of q = 2^(e - 21), where 2^e <= |s| < 2^(e+1).  The
// rounding moves a product by at most 2^-22 |s|, and every sum of up to three
// such products, or of two such sums with the same q, is exact in FP32.  So a
// centre coefficient set to minus the sum of the taps gives a difference whose
// coefficients sum to exactly zero, as the exact ones do.
struct WeightGrid {
    float q, inv_q;
};

__device__ __forceinline__ WeightGrid weight_grid(float s)
{
    const int b = (__float_as_int(s) & 0x7f800000) - (21 << 23);  // exponent field of q
    return {__int_as_float(b), __int_as_float(0x7f000000 - b)};
}

__device__ __forceinline__ float on_weight_grid(float v, WeightGrid g)
{
    return rintf(v * g.inv_q) * g.q;
}

// Apply to values v(k-2..k+2) given as vm2..vp2 for a population moving in the
// + direction (sgn > 0) or - direction (sgn < 0).
template <class R>
__device__ __forceinline__ R apply_stencil(const Stencil<R> &s, int sgn, R vm2, R vm1, R v0,
                                           R vp1, R vp2)
{
    if (sgn > 0) return s.wm1 * vp1 + (s.w0 * v0 + (s.w1 * vm1 + s.w2 * vm2));
    return s.wm1 * vm1 + (s.w0 * v0 + (s.w1 * vp1 + s.w2 * vp2));
}

// Node-local coefficients of one step (all from Eqs. 2.20, 2.32, 2.34), with
// h = A dt.  Each transform is written g + b (geq - g) + c F since a + b = 1.
template <class R>
struct Coeffs {
    R rho0, dt, h;
    R b_bar, c_bar;     // fbar^{+,h} from f~ (Eq. 2.19 inverted, then Eq. 2.34)
    R b_til, c_til;     // f~+ (Eq. 2.20)
    R b_star, c_star;   // f* from fbar* (Eq. 2.32)
    R b_phys, c_phys;   // physical f from f~ (Eq. 2.19 inverted; Eq. 2.32 with h = dt)
    R half_dt, half_h;  // force shifts of the first moment (Eq. 3.3 and its h analogue)
    int incomp;         // 1: incompressible equilibrium of He and Luo (cited in Sec. 2)
};

template <class R>
__host__ inline Coeffs<R> make_coeffs(double tau, double dt, double A, double rho0)
{
    const double h = A * dt;
    Coeffs<R> c;
    c.rho0 = R(rho0);
    c.dt = R(dt);
    c.h = R(h);
    // physical f = (2 tau f~ + dt feq + tau dt F)/(2 tau + dt);
    // fbar^{+,h} = (1 - h/2tau) f + (h/2tau) feq + (h/2) F
    const double k = 1.0 - h / (2.0 * tau);
    c.b_bar = R(k * dt / (2.0 * tau + dt) + h / (2.0 * tau));
    c.c_bar = R(k * tau * dt / (2.0 * tau + dt) + 0.5 * h);
    c.b_til = R(2.0 * dt / (2.0 * tau + dt));
    c.c_til = R(2.0 * tau * dt / (2.0 * tau + dt));
    c.b_star = R(h / (2.0 * tau + h));
    c.c_star = R(h * tau / (2.0 * tau + h));
    c.b_phys = R(dt / (2.0 * tau + dt));
    c.c_phys = R(tau * dt / (2.0 * tau + dt));
    c.half_dt = R(0.5 * dt);
    c.half_h = R(0.5 * h);
    c.incomp = 0;
    return c;
}

// The density that carries the momentum and multiplies the velocity terms of
// the equilibrium: rho itself (Eqs. 3.2, 3.3), or the constant rho0 under the
// incompressible equilibrium, f_i^eq = w_i [rho + rho0 (3 xi.u + 4.5 (xi.u)^2
// - 1.5 u.u)] with rho0 u = sum xi f.
template <class R>
__host__ __device__ __forceinline__ R macro_density(const Coeffs<R> &c, R drho)
{
    return c.incomp ? c.rho0 : c.rho0 + drho;
}

// The argument of force_terms that selects the equilibrium of the forcing term.
template <class R>
__host__ __device__ __forceinline__ R force_dshift(const Coeffs<R> &c, R drho)
{
    return c.incomp ? drho : R(0);
}

__host__ __device__ __forceinline__ int wrap_index(int k, int n)
{
    k %= n;
    return k < 0 ? k + n : k;
}

}  // namespace fdlbm
