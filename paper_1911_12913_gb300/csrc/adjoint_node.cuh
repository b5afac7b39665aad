// Node maps of the T2S2-FDLBM step and their vector-Jacobian products, for the
// discrete adjoint: moments (Eq. 3.3, with the force shift of the stage),
// equilibrium (Eq. 3.2) and forcing (Eq. 3.12).
#pragma once

#include "lattice.cuh"

namespace fdlbm {

// Node map of stage A or B: moments (with force shift `sh`), equilibrium and
// forcing, and the derivatives needed by its vector-Jacobian product.
// 1/rho: the forward sweeps' fast reciprocal (within 1 ulp in FP32, equal to
// 1/x on the samples tested in FP64).
template <class R>
__device__ __forceinline__ R node_recip(R v)
{
    return node_reciprocal<R>(v);
}

template <class R>
struct NodeMap {
    R drho, rho, inv, ux, uy, eu[9], t[9], feq[9], s[9];

    __device__ __forceinline__ void eval(const R g[9], R rho0, R Fx, R Fy, R sh)
    {
        R jx, jy;
        moments_dev(g, drho, jx, jy);
        rho = rho0 + drho;
        jx += sh * rho * Fx;
        jy += sh * rho * Fy;
        inv = node_recip(rho);
        ux = jx * inv;
        uy = jy * inv;
        const R usq = R(1.5) * (ux * ux + uy * uy);
        const R uF = ux * Fx + uy * Fy;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            eu[i] = xi_dot<R>(i, ux, uy);
            t[i] = eu[i] * (R(3) + R(4.5) * eu[i]) - usq;
            feq[i] = wq<R>(i) * rho0 + wq<R>(i) * (drho + rho * t[i]);
            s[i] = xi_dot<R>(i, Fx, Fy) - uF;  // (xi_i - u).F
        }
    }

    // Given lam_geq and lam_F (per population), add the cotangent of g (lam_g)
    // and of the force (lFx, lFy).
    __device__ __forceinline__ void vjp(const R lgeq_in[9], const R lF[9], R Fx, R Fy, R sh, R lam_g[9], R &lFx,
                        R &lFy) const
    {
        R lux = R(0), luy = R(0), lrho = R(0), ldrho = R(0), lusq = R(0);
        // the cotangents of s_i = (xi_i - u).F summed first: sum ls, sum xi ls
        R ls0 = R(0), lsx = R(0), lsy = R(0);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            // F_i = 3 s_i feq_i
            const R lgeq = lgeq_in[i] + R(3) * s[i] * lF[i];
            const R ls = R(3) * feq[i] * lF[i];
            ls0 += ls;
            lsx += R(cx(i)) * ls;
            lsy += R(cy(i)) * ls;
            // geq_i = w_i (drho + rho t_i), t_i = eu_i (3 + 4.5 eu_i) - usq
            const R wl = wq<R>(i) * lgeq;
            ldrho += wl;
            lrho += t[i] * wl;
            const R lt = rho * wl;
            const R leu = (R(3) + R(9) * eu[i]) * lt;
            lusq -= lt;
            lux += R(cx(i)) * leu;
            luy += R(cy(i)) * leu;
        }
        lux -= Fx * ls0;
        luy -= Fy * ls0;
        lFx += lsx - ux * ls0;
        lFy += lsy - uy * ls0;
        // usq = 1.5 (ux^2 + uy^2)
        lux += R(3) * ux * lusq;
        luy += R(3) * uy * lusq;
        // u = j'/rho, j' = j + sh rho F
        const R ljx = lux * inv, ljy = luy * inv;
        lrho -= (ux * lux + uy * luy) * inv;
        lrho += sh * (Fx * ljx + Fy * ljy);
        lFx += sh * rho * ljx;
        lFy += sh * rho * ljy;
        ldrho += lrho;
#pragma unroll
        for (int i = 0; i < 9; ++i) lam_g[i] += ldrho + R(cx(i)) * ljx + R(cy(i)) * ljy;
    }
};

}  // namespace fdlbm
