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

// ---- Eq. 3.2 from the momentum j = rho u instead of the velocity.  With
// e_i = xi_i . j, Eq. 3.2 minus w_i rho0 is
//     w_i [drho + 3 e_i + (4.5 e_i^2 - 1.5 j.j) / rho],
// the same value as equilibrium2 written out: only the quadratic term waits
// for the reciprocal of rho, so the linear terms and the squares are formed
// while it is in flight, and no velocity is formed at all.  Under the
// incompressible equilibrium of He and Luo, j = rho0 u and 1/rho0 replaces
// 1/rho (the terms rho0 (3 xi.u + 4.5 (xi.u)^2 - 1.5 u.u) are the same
// expression in j).
struct MacroJ {
    f2 drho, jx, jy, inv;  // inv: 1/rho, or 1/rho0 under the incompressible equilibrium
};

__device__ __forceinline__ MacroJ moments2_j(const f2 g[9], f2 rho0)
{
    MacroJ m;
    m.drho = add2(add2(add2(g[0], g[1]), add2(g[2], g[3])),
                  add2(add2(g[4], g[5]), add2(add2(g[6], g[7]), g[8])));
    m.jx = add2(add2(sub2(g[1], g[3]), sub2(g[5], g[6])), sub2(g[8], g[7]));
    m.jy = add2(sub2(g[2], g[4]), sub2(add2(g[5], g[6]), add2(g[7], g[8])));
    const f2 rho = add2(rho0, m.drho);
    m.inv = make_float2(rcp_approx(rho.x), rcp_approx(rho.y));
    return m;
}

__device__ __forceinline__ MacroJ moments2_j_incomp(const f2 g[9], f2 inv_rho0)
{
    MacroJ m;
    m.drho = add2(add2(add2(g[0], g[1]), add2(g[2], g[3])),
                  add2(add2(g[4], g[5]), add2(add2(g[6], g[7]), g[8])));
    m.jx = add2(add2(sub2(g[1], g[3]), sub2(g[5], g[6])), sub2(g[8], g[7]));
    m.jy = add2(sub2(g[2], g[4]), sub2(add2(g[5], g[6]), add2(g[7], g[8])));
    m.inv = inv_rho0;
    return m;
}

// Coefficients 3 w_i of the linear term: c1 = fl(1/3) on the axis velocities
// and c2 = (1 - 2 c1)/4 on the diagonal ones, so that 2 c1 + 4 c2 = 1 holds
// exactly and the first moment of the equilibrium is j with no rounding bias.
// A fixed relative bias d there acts, every step, like a force d j / tau; in
// a slowly decaying flow (the cavity near steady state) it shifts the state
// by about d over the decay rate per step.
constexpr float kLin1 = 1.f / 3.f;
constexpr float kLin2 = (1.f - 2.f * kLin1) * 0.25f;
static_assert(2.f * kLin1 + 4.f * kLin2 == 1.f, "momentum of the linear term");

// f_i^eq - w_i rho0 in the momentum form above; velocity pairs as in
// equilibrium2 (xi_1 / xi_3 on e = jx, xi_2 / xi_4 on jy, xi_5 / xi_7 on
// jx + jy, xi_6 / xi_8 on jy - jx).
__device__ __forceinline__ void equilibrium2_j(const MacroJ &m, f2 geq[9])
{
    const f2 qn = mul2(fma2(m.jx, m.jx, mul2(m.jy, m.jy)), bc(-1.5f));
    geq[0] = mul2(bc(4.f / 9.f), fma2(qn, m.inv, m.drho));
    auto pair = [&](f2 e, float w, float c, f2 &plus, f2 &minus) {
        const f2 s = fma2(fma2(mul2(e, bc(4.5f)), e, qn), m.inv, m.drho);
        const f2 ws = mul2(bc(w), s);
        plus = fma2(bc(c), e, ws);
        minus = fma2(bc(-c), e, ws);
    };
    pair(m.jx, 1.f / 9.f, kLin1, geq[1], geq[3]);
    pair(m.jy, 1.f / 9.f, kLin1, geq[2], geq[4]);
    pair(add2(m.jx, m.jy), 1.f / 36.f, kLin2, geq[5], geq[7]);
    pair(sub2(m.jy, m.jx), 1.f / 36.f, kLin2, geq[6], geq[8]);
}

// Weights of the relaxation g + b (f^eq - g) = (1 - b) g + b f^eq (Eq. 2.52
// and Eq. 2.51 are of this form) folded into the momentum-form equilibrium,
// as pairs: b w_i for the three weight classes, +-b c1 and +-b c2 for the
// linear term, and 1 - b.  The unfolded form conserves mass and momentum for
// any b; the folded one does so only if (1 - b) + b = 1 and the linear
// weights sum to b exactly.  So b is taken as b' = 1 - fl(1 - b) (within
// 3e-8 of b, and 1 - b' is exact) and b c2 = (b' - 2 b c1)/4 (exact).
struct RelaxK {
    float2 bw0, bw1, bw2, bc1, bc2, nbc1, nbc2, omb;
};

inline RelaxK make_relax(float b)
{
    auto p = [](float v) { return make_float2(v, v); };
    const float omb = 1.f - b;
    const float bp = 1.f - omb;
    const float bc1 = bp / 3.f;
    const float bc2 = (bp - 2.f * bc1) * 0.25f;
    RelaxK k;
    k.bw0 = p((float)((double)bp * 4.0 / 9.0));
    k.bw1 = p((float)((double)bp / 9.0));
    k.bw2 = p((float)((double)bp / 36.0));
    k.bc1 = p(bc1);
    k.bc2 = p(bc2);
    k.nbc1 = p(-bc1);
    k.nbc2 = p(-bc2);
    k.omb = p(omb);
    return k;
}

// out_i = (1 - b') g_i + b' (f_i^eq - w_i rho0) with f^eq from m (the moments of
// g or of another population set): two packed FMAs per population.
__device__ __forceinline__ void relax2_j(const MacroJ &m, const f2 g[9], const RelaxK &k, f2 out[9])
{
    const f2 qn = mul2(fma2(m.jx, m.jx, mul2(m.jy, m.jy)), bc(-1.5f));
    out[0] = fma2(k.omb, g[0], mul2(k.bw0, fma2(qn, m.inv, m.drho)));
    auto pair = [&](f2 e, f2 bw, f2 bcl, f2 nbcl, int ip, int im) {
        const f2 s = fma2(fma2(mul2(e, bc(4.5f)), e, qn), m.inv, m.drho);
        const f2 bws = mul2(bw, s);
        out[ip] = fma2(bcl, e, fma2(k.omb, g[ip], bws));
        out[im] = fma2(nbcl, e, fma2(k.omb, g[im], bws));
    };
    pair(m.jx, k.bw1, k.bc1, k.nbc1, 1, 3);
    pair(m.jy, k.bw1, k.bc1, k.nbc1, 2, 4);
    pair(add2(m.jx, m.jy), k.bw2, k.bc2, k.nbc2, 5, 7);
    pair(sub2(m.jy, m.jx), k.bw2, k.bc2, k.nbc2, 6, 8);
}

// The forcing term of Eq. 3.12 for the pair, premultiplied by k = 3 c for the
// weight c of the transform it enters (Eqs. 2.20, 2.32, 2.34):
//   k/3 F_i = k (xi_i.F - u.F) f_i^eq,   f_i^eq = w_i rf + geq_i,
// with rf = rho0 (f^eq of Eq. 3.2; geq is its deviation from w_i rho0) or
// rf = rho0 - drho under the incompressible equilibrium, whose forcing term
// takes the equilibrium at rho0.  uF = u.F.  out_i += (k/3) F_i for two
// transforms (k1, k2) at once; q returns f_i^eq for reuse.
__device__ __forceinline__ void force_add2(const f2 geq[9], f2 rf, f2 Fx, f2 Fy, f2 uF, f2 k1,
                                           f2 k2, f2 out1[9], f2 out2[9])
{
    const float w[3] = {4.f / 9.f, 1.f / 9.f, 1.f / 36.f};
    auto one = [&](int i, f2 tF, int wc) {
        const f2 q = fma2(bc(w[wc]), rf, geq[i]);
        out1[i] = fma2(mul2(k1, tF), q, out1[i]);
        out2[i] = fma2(mul2(k2, tF), q, out2[i]);
    };
    const f2 nuF = mul2(bc(-1.f), uF);
    one(0, nuF, 0);
    one(1, sub2(Fx, uF), 1);
    one(3, sub2(nuF, Fx), 1);
    one(2, sub2(Fy, uF), 1);
    one(4, sub2(nuF, Fy), 1);
    const f2 s = add2(Fx, Fy), d = sub2(Fy, Fx);
    one(5, sub2(s, uF), 2);
    one(7, sub2(nuF, s), 2);
    one(6, sub2(d, uF), 2);
    one(8, sub2(nuF, d), 2);
}

// The same for one transform.
__device__ __forceinline__ void force_add1(const f2 geq[9], f2 rf, f2 Fx, f2 Fy, f2 uF, f2 k1,
                                           f2 out1[9])
{
    const float w[3] = {4.f / 9.f, 1.f / 9.f, 1.f / 36.f};
    auto one = [&](int i, f2 tF, int wc) {
        const f2 q = fma2(bc(w[wc]), rf, geq[i]);
        out1[i] = fma2(mul2(k1, tF), q, out1[i]);
    };
    const f2 nuF = mul2(bc(-1.f), uF);
    one(0, nuF, 0);
    one(1, sub2(Fx, uF), 1);
    one(3, sub2(nuF, Fx), 1);
    one(2, sub2(Fy, uF), 1);
    one(4, sub2(nuF, Fy), 1);
    const f2 s = add2(Fx, Fy), d = sub2(Fy, Fx);
    one(5, sub2(s, uF), 2);
    one(7, sub2(nuF, s), 2);
    one(6, sub2(d, uF), 2);
    one(8, sub2(nuF, d), 2);
}

}  // namespace packed
}  // namespace fdlbm
