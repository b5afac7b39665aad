// Fused T2S2-FDLBM step for grids periodic in x and y: both stages of Sec. 2D
// (Steps 1-3) in one kernel, one read and one write of the distributions per
// node and step.
//
// Work decomposition: a CTA owns a strip of W = NT - 8 columns and a segment of
// `rows` rows, and sweeps the segment from bottom to top.  Thread t owns column
// x0 - 4 + t for the whole sweep, so every difference in y (Eqs. 2.36-2.38)
// reads a register window of the thread's own column; differences in x read
// shared-memory row buffers written by the neighbouring threads.  Per row r:
//   A  (all NT columns)        load f~(r), moments (Eq. 3.3), f^eq (Eq. 3.2),
//                              force (Eq. 3.12) -> fbar^{+,h}(r) (Eqs. 2.19, 2.34)
//                              and f~+(r) (Eq. 2.20)
//   B  (NT-4 columns, row r-2) fbar* = fbar^{+,h} - h xi.grad fbar^{+,h}
//                              (Eqs. 2.33, 2.35), its moments, f* (Eq. 2.32)
//   C  (W columns, row r-4)    f~(t+dt) = f~+ - dt xi.grad f* (Eqs. 2.23, 2.27)
// A row of f* needs fbar^{+,h} two rows further on, and the update needs f* two
// rows further on, hence the lag of 2 + 2 rows and the 4-row y-halo of a
// segment.  The recomputed halo is 8 of NT columns and 8 of `rows` rows.
//
// The register windows and the shared-memory rings hold 5 rows and the row
// loop is unrolled by 5, so every window slot and ring slot is a compile-time
// index (no register shuffling), and one barrier per row suffices: a ring slot
// is rewritten 5 rows after it was written, and every reader of it has passed
// at least one barrier in between.
#include <cstdint>

#include "internal.h"

namespace fdlbm {
namespace {

constexpr int kHalo = 4;
constexpr int kRing = 5;

template <class R, int NT>
struct Smem {
    R P[kRing][6][NT];   // fbar^{+,h} of the x-moving populations
    R S[kRing][6][NT];   // f* of the x-moving populations
    R Q[kRing][9][NT];   // f~+ (read back by the same thread only)
};

template <class R, bool FORCE, int NT>
struct Sweep {
    const StepArgs<R> a;
    Smem<R, NT> &sm;
    const int t, gx, xc;
    const bool act1, act2;
    const R mxc;
    const Coeffs<R> c;
    const Stencil<R> st;
    R Pw[9][kRing];  // fbar^{+,h} of this column, slot = row mod 5 (phase)
    R Sw[9][kRing];  // f* of this column
    R cur[9], nxt[9];
    int rl, rs, rq;  // wrapped global rows of the next load, stage B, stage C

    __device__ static int inc(int v, int n) { return v + 1 == n ? 0 : v + 1; }

    __device__ void load(R *dst, int row) const
    {
        const size_t off = (size_t)row * a.pitch + gx;
#pragma unroll
        for (int i = 0; i < 9; ++i) dst[i] = __ldg(a.gin + i * a.plane + off);
    }

    // One row of the sweep at compile-time phase PH (= iteration mod 5).
    // doA/doB/doC: which stages run (uniform over the block).
    template <int PH>
    __device__ void row(bool load_next, bool doB, bool doC)
    {
        constexpr int p0 = PH;                 // row r       (newest)
        constexpr int p1 = (PH + 4) % kRing;   // row r-1
        constexpr int p2 = (PH + 3) % kRing;   // row r-2  (stage B centre)
        constexpr int p3 = (PH + 2) % kRing;   // row r-3
        constexpr int p4 = (PH + 1) % kRing;   // row r-4  (stage C centre)
        const int rA = rl;                     // row being loaded now is cur's row
        if (load_next) {
            rl = inc(rl, a.ny);
            load(nxt, rl);
        }
        // ------------------------------------------------------------ A
        {
            R drho, jx, jy;
            moments_dev(cur, drho, jx, jy);
            const R rho = macro_density(c, drho);
            R Fx = R(0), Fy = R(0);
            if (FORCE) {
                const size_t fo = (size_t)rA * a.pitch + gx;
                Fx = __ldg(a.force + fo);
                Fy = __ldg(a.force + a.plane + fo);
                jx += c.half_dt * rho * Fx;
                jy += c.half_dt * rho * Fy;
            }
            const R inv = node_reciprocal(rho);
            const R ux = jx * inv, uy = jy * inv;
            R geq[9], F[9];
            equilibrium_dev_j(drho, jx, jy, inv, geq);
            if (FORCE) force_terms(c.rho0, geq, ux, uy, Fx, Fy, F, force_dshift(c, drho));
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const R neq = geq[i] - cur[i];
                R gb = cur[i] + c.b_bar * neq;
                R gt = cur[i] + c.b_til * neq;
                if (FORCE) {
                    gb += c.c_bar * F[i];
                    gt += c.c_til * F[i];
                }
                Pw[i][p0] = gb;
                if (xslot(i) >= 0) sm.P[p0][xslot(i)][t] = gb;
                sm.Q[p0][i][t] = gt;
            }
        }
        __syncthreads();
        // ------------------------------------------------------------ B
        if (doB) {
            const int sg = rs;
            rs = inc(rs, a.ny);
            if (act1) {
                const R hx = c.h * mxc, hy = c.h * __ldg(a.my + sg);
                R gs[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const R v0 = Pw[i][p2];
                    R acc = v0;
                    if (cx(i) != 0) {
                        const R *rw = sm.P[p2][xslot(i)];
                        acc -= hx * apply_stencil(st, cx(i), rw[t - 2], rw[t - 1], v0, rw[t + 1],
                                                  rw[t + 2]);
                    }
                    if (cy(i) != 0)
                        acc -= hy * apply_stencil(st, cy(i), Pw[i][p4], Pw[i][p3], v0, Pw[i][p1],
                                                  Pw[i][p0]);
                    gs[i] = acc;
                }
                R drho, jx, jy;
                moments_dev(gs, drho, jx, jy);
                const R rho = macro_density(c, drho);
                R Fx = R(0), Fy = R(0);
                if (FORCE) {
                    const size_t fo = (size_t)sg * a.pitch + gx;
                    Fx = __ldg(a.force + fo);
                    Fy = __ldg(a.force + a.plane + fo);
                    jx += c.half_h * rho * Fx;
                    jy += c.half_h * rho * Fy;
                }
                const R inv = node_reciprocal(rho);
                const R ux = jx * inv, uy = jy * inv;
                R geq[9], F[9];
                equilibrium_dev_j(drho, jx, jy, inv, geq);
                if (FORCE) force_terms(c.rho0, geq, ux, uy, Fx, Fy, F, force_dshift(c, drho));
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    R gst = gs[i] + c.b_star * (geq[i] - gs[i]);
                    if (FORCE) gst += c.c_star * F[i];
                    Sw[i][p0] = gst;  // f* of row r-2 lives in slot PH
                    if (xslot(i) >= 0) sm.S[p0][xslot(i)][t] = gst;
                }
            }
        }
        // ------------------------------------------------------------ C
        // f* rows (r-6 .. r-2) sit in slots (p4, p3, p2, p1, p0) of Sw; the
        // centre row r-4 is slot p2 (written two rows ago, behind a barrier).
        if (doC) {
            const int qg = rq;
            rq = inc(rq, a.ny);
            if (act2) {
                const R dx = c.dt * mxc, dy = c.dt * __ldg(a.my + qg);
                const size_t off = (size_t)qg * a.pitch + xc;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const R v0 = Sw[i][p2];
                    R acc = sm.Q[p4][i][t];
                    if (cx(i) != 0) {
                        const R *rw = sm.S[p2][xslot(i)];
                        acc -= dx * apply_stencil(st, cx(i), rw[t - 2], rw[t - 1], v0, rw[t + 1],
                                                  rw[t + 2]);
                    }
                    if (cy(i) != 0)
                        acc -= dy * apply_stencil(st, cy(i), Sw[i][p4], Sw[i][p3], v0, Sw[i][p1],
                                                  Sw[i][p0]);
                    a.gout[i * a.plane + off] = acc;
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) cur[i] = nxt[i];
    }
};

template <class R, bool FORCE, int NT>
__global__ void __launch_bounds__(NT, sizeof(R) == 4 ? 4 : 2) k_step_fused(const StepArgs<R> a)
{
    constexpr int W = NT - 2 * kHalo;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<R, NT> &sm = *reinterpret_cast<Smem<R, NT> *>(smem_raw);

    const int t = threadIdx.x;
    const int x0 = blockIdx.x * W;
    const int xc = x0 - kHalo + t;
    const int y0 = blockIdx.y * a.rows;
    if (y0 >= a.ny) return;  // uniform over the block
    const int y1 = min(y0 + a.rows, a.ny);
    const int gx = wrap_index(xc, a.nx);
    Sweep<R, FORCE, NT> sw{a,
                           sm,
                           t,
                           gx,
                           xc,
                           (t >= 2) && (t < NT - 2),
                           (t >= kHalo) && (t < NT - kHalo) && (xc < a.nx),
                           a.mx[gx],
                           a.c,
                           a.st};
    // rows y0-4 .. y1+3: iteration k handles load row y0-4+k, stage B row
    // y0-6+k (from k = 4), stage C row y0-8+k (from k = 8)
    const int first = wrap_index(y0 - kHalo, a.ny);
    sw.rl = first;
    sw.rs = wrap_index(y0 - 2, a.ny);
    sw.rq = y0;
    sw.load(sw.cur, first);
    const int iters = (y1 - y0) + 2 * kHalo;
    // iteration k loads row y0-4+k; stage B from k = 4, stage C from k = 8.
    // Full blocks of five rows first (one straight-line body, which lets the
    // compiler hoist the next row's loads), then the remaining 0..4 rows.
    int k = 0;
    for (; k + kRing <= iters; k += kRing) {
        sw.template row<0>(k + 1 < iters, k >= 4, k >= 8);
        sw.template row<1>(k + 2 < iters, k + 1 >= 4, k + 1 >= 8);
        sw.template row<2>(k + 3 < iters, k + 2 >= 4, k + 2 >= 8);
        sw.template row<3>(k + 4 < iters, k + 3 >= 4, k + 3 >= 8);
        sw.template row<4>(k + 5 < iters, k + 4 >= 4, k + 4 >= 8);
    }
    if (k < iters) sw.template row<0>(k + 1 < iters, true, k >= 8);
    if (k + 1 < iters) sw.template row<1>(k + 2 < iters, true, k + 1 >= 8);
    if (k + 2 < iters) sw.template row<2>(k + 3 < iters, true, k + 2 >= 8);
    if (k + 3 < iters) sw.template row<3>(k + 4 < iters, true, k + 3 >= 8);
}

}  // namespace

template <class R>
cudaError_t launch_fused(const StepArgs<R> &a, cudaStream_t s)
{
    constexpr int NT = 128;
    constexpr int W = NT - 2 * kHalo;
    constexpr size_t smem = sizeof(Smem<R, NT>);
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

int fused_tile_width() { return 128 - 2 * kHalo; }

template <class R>
int fused_blocks_per_sm()
{
    int n = 0;
    constexpr size_t smem = sizeof(Smem<R, 128>);
    cudaFuncSetAttribute(k_step_fused<R, false, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_fused<R, false, 128>, 128, smem) !=
        cudaSuccess)
        return 0;
    return n;
}
template int fused_blocks_per_sm<float>();
template int fused_blocks_per_sm<double>();

template cudaError_t launch_fused<float>(const StepArgs<float> &, cudaStream_t);
template cudaError_t launch_fused<double>(const StepArgs<double> &, cudaStream_t);

}  // namespace fdlbm
