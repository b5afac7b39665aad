// Node-local pieces of the fused sweeps with walls: the moments and
// equilibrium of a deviation vector, and the non-equilibrium extrapolation of
// Eq. 3.10.
#pragma once

#include "internal.h"

namespace fdlbm {
namespace {

// Eq. 3.3 and Eq. 3.2 for a 9-vector of deviations; `shift` is the force
// shift of its first moment (FORCE only).
template <class R, bool FORCE>
__device__ __forceinline__ void node_eq(const Coeffs<R> &c, const R g[9], R Fx, R Fy, R shift,
                                        R &drho, R &rho, R &ux, R &uy, R geq[9])
{
    R jx, jy;
    moments_dev(g, drho, jx, jy);
    rho = macro_density(c, drho);
    if (FORCE) {
        jx += shift * rho * Fx;
        jy += shift * rho * Fy;
    }
    const R inv = node_reciprocal(rho);
    ux = jx * inv;
    uy = jy * inv;
    equilibrium_dev_j(drho, jx, jy, inv, geq);
}

// Eq. 3.10: the wall value of every population from node x_j's vector g.
template <class R, bool FORCE>
__device__ __forceinline__ void nee(const Coeffs<R> &c, const R g[9], R Fx, R Fy, R shift, R uwx,
                                    R uwy, R out[9])
{
    R drho, rho, ux, uy, geqj[9], geqb[9];
    node_eq<R, FORCE>(c, g, Fx, Fy, shift, drho, rho, ux, uy, geqj);
    equilibrium_dev(drho, rho, uwx, uwy, geqb);
#pragma unroll
    for (int i = 0; i < 9; ++i) out[i] = geqb[i] + (g[i] - geqj[i]);
}

}  // namespace
}  // namespace fdlbm
