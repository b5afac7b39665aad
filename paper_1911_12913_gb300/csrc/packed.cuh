// Node-local T2S2-FDLBM arithmetic on pairs of nodes in packed FP32x2
// (sm_100-family f32x2 FMA/ADD/MUL): moments (Eq. 3.3), the equilibrium of
// Eq. 3.2 as a deviation from w_i rho0, and the mixed difference of Eq. 2.36.
#pragma once

#include <cuda_runtime.h>

#include "lattice.cuh"

namespace fdlbm {
namespace packed {

typedef float2 f2;

__device__ __forceinline__ f2 bc(float s) { return make_float2(s, s); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 sub2(f2 a, f2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }



// 1/x from the hardware approximation (about one ulp for normal x), enough
// for FP32 storage; the density is O(1).
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

struct Macro {
    f2 drho, rho, ux, uy;
};

// Eq. 3.3 on deviations (no force): drho = sum g, rho u = sum xi g.
__device__ __forceinline__ Macro moments2(const f2 g[9], f2 rho0)
{
    Macro m;
    m.drho = add2(add2(add2(g[0], g[1]), add2(g[2], g[3])),
                  add2(add2(g[4], g[5]), add2(add2(g[6], g[7]), g[8])));
    const f2 jx = add2(add2(sub2(g[1], g[3]), sub2(g[5], g[6])), sub2(g[8], g[7]));
    const f2 jy = add2(sub2(g[2], g[4]), sub2(add2(g[5], g[6]), add2(g[7], g[8])));
    m.rho = add2(rho0, m.drho);
    const f2 inv = make_float2(rcp_approx(m.rho.x), rcp_approx(m.rho.y));
    m.ux = mul2(jx, inv);
    m.uy = mul2(jy, inv);
    return m;
}

// The same under the incompressible equilibrium of He and Luo: rho0 u = sum xi
// g, and rho0 (not rho) multiplies the velocity terms of the equilibrium.
__device__ __forceinline__ Macro moments2_incomp(const f2 g[9], f2 rho0, f2 inv_rho0)
{
    Macro m;
    m.drho = add2(add2(add2(g[0], g[1]), add2(g[2], g[3])),
                  add2(add2(g[4], g[5]), add2(add2(g[6], g[7]), g[8])));
    const f2 jx = add2(add2(sub2(g[1], g[3]), sub2(g[5], g[6])), sub2(g[8], g[7]));
    const f2 jy = add2(sub2(g[2], g[4]), sub2(add2(g[5], g[6]), add2(g[7], g[8])));
    m.rho = rho0;
    m.ux = mul2(jx, inv_rho0);
    m.uy = mul2(jy, inv_rho0);
    return m;
}

// Eq. 3.2 minus w_i rho0, written pairwise for opposite velocities: with
// e = xi_i.u,  f_i^eq - w_i rho0 = w_i drho + w_i rho (A +- 3e),
// A = 4.5 e^2 - 1.5 u.u.
__device__ __forceinline__ void equilibrium2(const Macro &m, f2 geq[9])
{
    const f2 nusq = mul2(fma2(m.ux, m.ux, mul2(m.uy, m.uy)), bc(-1.5f));
    const f2 w0r = mul2(bc(4.f / 9.f), m.rho), w1r = mul2(bc(1.f / 9.f), m.rho),
             w2r = mul2(bc(1.f / 36.f), m.rho);
    const f2 w0d = mul2(bc(4.f / 9.f), m.drho), w1d = mul2(bc(1.f / 9.f), m.drho),
             w2d = mul2(bc(1.f / 36.f), m.drho);
    geq[0] = fma2(w0r, nusq, w0d);
    auto pair = [&](f2 e, f2 wr, f2 wd, f2 &plus, f2 &minus) {
        const f2 A = fma2(mul2(e, bc(4.5f)), e, nusq);
        plus = fma2(wr, fma2(bc(3.f), e, A), wd);
        minus = fma2(wr, fma2(bc(-3.f), e, A), wd);
    };
    pair(m.ux, w1r, w1d, geq[1], geq[3]);
    pair(m.uy, w1r, w1d, geq[2], geq[4]);
    pair(add2(m.ux, m.uy), w2r, w2d, geq[5], geq[7]);
    pair(sub2(m.uy, m.ux), w2r, w2d, geq[6], geq[8]);
}

// sign(c) * D_m f at the centre from f(k-2..k+2); w = {wm1, w0, w1, w2} of
// make_stencil (lattice.cuh).
__device__ __forceinline__ f2 stencil2(const float w[4], int sgn, f2 vm2, f2 vm1, f2 v0, f2 vp1,
                                       f2 vp2)
{
    if (sgn > 0)
        return fma2(bc(w[3]), vm2, fma2(bc(w[2]), vm1, fma2(bc(w[1]), v0, mul2(bc(w[0]), vp1))));
    return fma2(bc(w[3]), vp2, fma2(bc(w[2]), vp1, fma2(bc(w[1]), v0, mul2(bc(w[0]), vm1))));
}

}  // namespace packed
}  // namespace fdlbm
