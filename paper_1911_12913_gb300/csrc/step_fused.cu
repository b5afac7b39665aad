// Fused T2S2-FDLBM step for grids periodic in x and y: both stages of Sec. 2D
// (Steps 1-3) in one kernel, one read and one write of the distributions per
// node and step.
//
// Work decomposition: a CTA owns a strip of W = NT - 8 columns and a segment of
// `rows` rows, and sweeps the segment from bottom to top.  Thread t owns column
// x0 - 4 + t for the whole sweep, so every difference in y (Eqs. 2.36-2.38)
// reads a register window of the thread's own column; differences in x read
// shared-memory row buffers written by the neighbouring threads.  Per row r:
//   A  (all NT columns)       load f~(r), moments (Eq. 3.3), f^eq (Eq. 3.2),
//                             force (Eq. 3.12) -> fbar^{+,h}(r) (Eqs. 2.19, 2.34)
//                             and f~+(r) (Eq. 2.20)
//   B  (NT-4 columns, row r-2) fbar* = fbar^{+,h} - h xi.grad fbar^{+,h}
//                             (Eqs. 2.33, 2.35), its moments, f* (Eq. 2.32)
//   C  (W columns, row r-4)    f~(t+dt) = f~+ - dt xi.grad f* (Eqs. 2.23, 2.27)
// A row of f* needs fbar^{+,h} two rows further on, and the update needs f* two
// rows further on, hence the lag of 2 + 2 rows and the 4-row y-halo of a
// segment.  The recomputed halo is 8 of NT columns and 8 of `rows` rows.
#include <cstdint>

#include "internal.h"

namespace fdlbm {
namespace {

constexpr int kHalo = 4;

template <class R, bool FORCE, int NT>
__global__ void __launch_bounds__(NT, sizeof(R) == 4 ? 3 : 2) k_step_fused(const StepArgs<R> a)
{
    constexpr int W = NT - 2 * kHalo;
    // Dynamic shared memory (83 KB for FP64 exceeds the static limit):
    //   sP[3][6][NT]  fbar^{+,h} of the x-moving populations, rows r-2..r
    //   sS[3][6][NT]  f* of the x-moving populations, rows s-2..s
    //   sQ[5][9][NT]  f~+ of the thread's own column, rows r-4..r
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R (*sP)[6][NT] = reinterpret_cast<R (*)[6][NT]>(smem_raw);
    R (*sS)[6][NT] = reinterpret_cast<R (*)[6][NT]>(smem_raw + sizeof(R) * 3 * 6 * NT);
    R (*sQ)[9][NT] = reinterpret_cast<R (*)[9][NT]>(smem_raw + sizeof(R) * 6 * 6 * NT);

    const R *__restrict__ gin = a.gin;
    R *__restrict__ gout = a.gout;
    const int t = threadIdx.x;
    const int x0 = blockIdx.x * W;
    const int xc = x0 - kHalo + t;
    const int gx = wrap_index(xc, a.nx);
    const int y0 = blockIdx.y * a.rows;
    if (y0 >= a.ny) return;  // uniform over the block
    const int y1 = min(y0 + a.rows, a.ny);
    const bool act1 = (t >= 2) && (t < NT - 2);
    const bool act2 = (t >= kHalo) && (t < NT - kHalo) && (xc < a.nx);
    const R mxc = a.mx[gx];
    const Coeffs<R> c = a.c;
    const Stencil<R> st = a.st;
    const size_t plane = a.plane;

    R Pw[9][5];  // fbar^{+,h} window of this column: [4] = row r, [2] = row r-2
    R Sw[9][5];  // f* window of this column: [4] = row s = r-2, [2] = row r-4
    R cur[9], nxt[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            Pw[i][k] = R(0);
            Sw[i][k] = R(0);
        }
    }

    const int rfirst = y0 - kHalo, rlast = y1 + kHalo - 1;
    {
        const size_t off = (size_t)wrap_index(rfirst, a.ny) * a.pitch + gx;
#pragma unroll
        for (int i = 0; i < 9; ++i) cur[i] = __ldg(gin + i * plane + off);
    }

    int it = 0;
    for (int r = rfirst; r <= rlast; ++r, ++it) {
        if (r < rlast) {
            const size_t off = (size_t)wrap_index(r + 1, a.ny) * a.pitch + gx;
#pragma unroll
            for (int i = 0; i < 9; ++i) nxt[i] = __ldg(gin + i * plane + off);
        }
        // ---------------------------------------------------------------- A
        {
            R drho, jx, jy;
            moments_dev(cur, drho, jx, jy);
            const R rho = c.rho0 + drho;
            R Fx = R(0), Fy = R(0);
            if (FORCE) {
                const size_t fo = (size_t)wrap_index(r, a.ny) * a.pitch + gx;
                Fx = __ldg(a.force + fo);
                Fy = __ldg(a.force + plane + fo);
                jx += c.half_dt * rho * Fx;
                jy += c.half_dt * rho * Fy;
            }
            const R inv = R(1) / rho;
            const R ux = jx * inv, uy = jy * inv;
            R geq[9], F[9];
            equilibrium_dev(drho, rho, ux, uy, geq);
            if (FORCE) force_terms(c.rho0, geq, ux, uy, Fx, Fy, F);
            const int sp = it % 3, sq = it % 5;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const R neq = geq[i] - cur[i];
                R gb = cur[i] + c.b_bar * neq;
                R gt = cur[i] + c.b_til * neq;
                if (FORCE) {
                    gb += c.c_bar * F[i];
                    gt += c.c_til * F[i];
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) Pw[i][k] = Pw[i][k + 1];
                Pw[i][4] = gb;
                if (xslot(i) >= 0) sP[sp][xslot(i)][t] = gb;
                sQ[sq][i][t] = gt;
            }
        }
        __syncthreads();
        // ---------------------------------------------------------------- B
        if (r >= y0 && act1) {
            const int sg = wrap_index(r - 2, a.ny);
            const int sp = (it + 1) % 3;  // slot of row r-2 in sP
            const R hx = c.h * mxc, hy = c.h * __ldg(a.my + sg);
            R gs[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                R acc = Pw[i][2];
                if (cx(i) != 0) {
                    const R *row = sP[sp][xslot(i)];
                    acc -= hx * apply_stencil(st, cx(i), row[t - 2], row[t - 1], row[t], row[t + 1],
                                              row[t + 2]);
                }
                if (cy(i) != 0)
                    acc -= hy * apply_stencil(st, cy(i), Pw[i][0], Pw[i][1], Pw[i][2], Pw[i][3],
                                              Pw[i][4]);
                gs[i] = acc;
            }
            R drho, jx, jy;
            moments_dev(gs, drho, jx, jy);
            const R rho = c.rho0 + drho;
            R Fx = R(0), Fy = R(0);
            if (FORCE) {
                const size_t fo = (size_t)sg * a.pitch + gx;
                Fx = __ldg(a.force + fo);
                Fy = __ldg(a.force + plane + fo);
                jx += c.half_h * rho * Fx;
                jy += c.half_h * rho * Fy;
            }
            const R inv = R(1) / rho;
            const R ux = jx * inv, uy = jy * inv;
            R geq[9], F[9];
            equilibrium_dev(drho, rho, ux, uy, geq);
            if (FORCE) force_terms(c.rho0, geq, ux, uy, Fx, Fy, F);
            const int ss = it % 3;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                R gst = gs[i] + c.b_star * (geq[i] - gs[i]);
                if (FORCE) gst += c.c_star * F[i];
#pragma unroll
                for (int k = 0; k < 4; ++k) Sw[i][k] = Sw[i][k + 1];
                Sw[i][4] = gst;
                if (xslot(i) >= 0) sS[ss][xslot(i)][t] = gst;
            }
        }
        __syncthreads();
        // ---------------------------------------------------------------- C
        if (r >= y0 + kHalo && act2) {
            const int qg = wrap_index(r - kHalo, a.ny);
            const int ss = (it + 1) % 3;  // slot of row r-4 in sS
            const int sq = (it + 1) % 5;  // slot of row r-4 in sQ
            const R dx = c.dt * mxc, dy = c.dt * __ldg(a.my + qg);
            const size_t off = (size_t)qg * a.pitch + xc;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                R acc = sQ[sq][i][t];
                if (cx(i) != 0) {
                    const R *row = sS[ss][xslot(i)];
                    acc -= dx * apply_stencil(st, cx(i), row[t - 2], row[t - 1], row[t], row[t + 1],
                                              row[t + 2]);
                }
                if (cy(i) != 0)
                    acc -= dy * apply_stencil(st, cy(i), Sw[i][0], Sw[i][1], Sw[i][2], Sw[i][3],
                                              Sw[i][4]);
                gout[i * plane + off] = acc;
            }
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) cur[i] = nxt[i];
    }
}

}  // namespace

template <class R>
cudaError_t launch_fused(const StepArgs<R> &a, cudaStream_t s)
{
    constexpr int NT = 128;
    constexpr int W = NT - 2 * kHalo;
    constexpr size_t smem = sizeof(R) * (2 * 3 * 6 + 5 * 9) * NT;
    dim3 grid((a.nx + W - 1) / W, (a.ny + a.rows - 1) / a.rows);
    cudaError_t e;
    if (a.force) {
        e = cudaFuncSetAttribute(k_step_fused<R, true, NT>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_step_fused<R, true, NT><<<grid, NT, smem, s>>>(a);
    } else {
        e = cudaFuncSetAttribute(k_step_fused<R, false, NT>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_step_fused<R, false, NT><<<grid, NT, smem, s>>>(a);
    }
    return cudaGetLastError();
}

template cudaError_t launch_fused<float>(const StepArgs<float> &, cudaStream_t);
template cudaError_t launch_fused<double>(const StepArgs<double> &, cudaStream_t);

}  // namespace fdlbm
