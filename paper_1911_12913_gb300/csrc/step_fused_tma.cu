// Fused T2S2-FDLBM step for periodic grids with TMA row loads.
//
// Same sweep as step_fused.cu (per row r: stage A at row r, stage B at r-2,
// stage C at r-4; y-differences from per-thread register windows, x-differences
// from shared-memory rows; see the comment there), but rows of f~ no longer
// pass through registers: one warp issues 1-D bulk copies (cp.async.bulk,
// completion on an mbarrier) three rows ahead into a 3-stage shared buffer, so
// DRAM latency is covered by the pipeline instead of by occupancy.
//
// Ring sizes: stage buffers, fbar^{+,h} rows and f* rows rotate with period 3
// and need two barriers per row (after A, after B); the f~+ ring of the
// thread's own column has period 5 like the register windows.  With FP32 the
// shared memory is 55 KB per CTA, so four CTAs of 128 threads fit an SM.
//
// Requirements (host-checked): every row piece must start and end on 16 bytes
// (nx a multiple of 16 / sizeof(R)) and a strip wraps at most once (nx >= 128).
#include <cstdint>

#include "internal.h"
#include "tma.cuh"

namespace fdlbm {
namespace {

constexpr int kHalo = 4;
constexpr int kStages = 3;

template <class R, int NT>
struct SmemT {
    R stage[kStages][9][NT];  // f~ rows delivered by the bulk copies
    R P[kStages][6][NT];      // fbar^{+,h} of the x-moving populations
    R S[kStages][6][NT];      // f* of the x-moving populations
    R Q[5][9][NT];            // f~+ of the thread's own column
    uint64_t bar[kStages];
};

template <class R>
__device__ __forceinline__ R recip(R v)
{
    return R(1) / v;
}
template <>
__device__ __forceinline__ float recip<float>(float v)
{
    return __frcp_rn(v);
}

template <class R, bool FORCE, int NT>
struct SweepT {
    const StepArgs<R> a;
    SmemT<R, NT> &sm;
    const int t, gx, xc;
    const bool act1, act2;
    const R mxc;
    const Coeffs<R> c;
    const Stencil<R> st;
    const int iters;
    R Pw[9][5];
    R Sw[9][5];
    int ra, rs, rq;        // rows of stage A, B, C (wrapped)
    R myB, myC;            // metric of the next B / C row
    int ring = 0;          // iteration mod 3
    uint32_t parity = 0;   // mbarrier phase of stage `ring`
    bool timed_out = false;
    // producer (warp 0): lane j < ncp owns one bulk copy per row
    int ld_row = 0, ld_it = 0, ncp = 0;
    uint32_t cp_dst = 0, cp_bytes = 0;
    size_t cp_src = 0;

    __device__ void issue(int stage)
    {
        if (t == 0) mbar_expect_tx(&sm.bar[stage], 9u * NT * sizeof(R));
        __syncwarp();
        if (t < ncp)
            bulk_copy(cp_dst + (uint32_t)(stage * 9 * NT * sizeof(R)),
                      a.gin + (size_t)ld_row * a.pitch + cp_src, cp_bytes,
                      smem_addr(&sm.bar[stage]));
        ld_row = ld_row + 1 == a.ny ? 0 : ld_row + 1;
        ++ld_it;
    }

    template <int PH>
    __device__ void row(bool doB, bool doC)
    {
        constexpr int p0 = PH, p1 = (PH + 4) % 5, p2 = (PH + 3) % 5, p3 = (PH + 2) % 5,
                      p4 = (PH + 1) % 5;
        const int rP = ring == 2 ? 0 : ring + 1;  // slot of rows r-2 (P) and r-4 (S)
        // ------------------------------------------------------------ A (row r)
        if (!mbar_wait_bounded(&sm.bar[ring], parity)) timed_out = true;
        {
            R g[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) g[i] = sm.stage[ring][i][t];
            R drho, jx, jy;
            moments_dev(g, drho, jx, jy);
            const R rho = c.rho0 + drho;
            R Fx = R(0), Fy = R(0);
            if (FORCE) {
                const size_t fo = (size_t)ra * a.pitch + gx;
                Fx = __ldg(a.force + fo);
                Fy = __ldg(a.force + a.plane + fo);
                jx += c.half_dt * rho * Fx;
                jy += c.half_dt * rho * Fy;
            }
            ra = ra + 1 == a.ny ? 0 : ra + 1;
            const R inv = recip(rho);
            const R ux = jx * inv, uy = jy * inv;
            R geq[9], F[9];
            equilibrium_dev(drho, rho, ux, uy, geq);
            if (FORCE) force_terms(c.rho0, geq, ux, uy, Fx, Fy, F);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const R neq = geq[i] - g[i];
                R gb = g[i] + c.b_bar * neq;
                R gt = g[i] + c.b_til * neq;
                if (FORCE) {
                    gb += c.c_bar * F[i];
                    gt += c.c_til * F[i];
                }
                Pw[i][p0] = gb;
                if (xslot(i) >= 0) sm.P[ring][xslot(i)][t] = gb;
                sm.Q[PH][i][t] = gt;
            }
        }
        __syncthreads();
        // the stage just consumed is free: request the row three iterations ahead
        if (t < 32 && ld_it < iters) {
            fence_proxy_async();
            issue(ring);
        }
        // ------------------------------------------------------------ B (row r-2)
        if (doB) {
            const int sg = rs;
            rs = rs + 1 == a.ny ? 0 : rs + 1;
            const R my_now = myB;
            myB = __ldg(a.my + rs);
            if (act1) {
                const R hx = c.h * mxc, hy = c.h * my_now;
                R gs[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const R v0 = Pw[i][p2];
                    R acc = v0;
                    if (cx(i) != 0) {
                        const R *rw = sm.P[rP][xslot(i)];
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
                const R rho = c.rho0 + drho;
                R Fx = R(0), Fy = R(0);
                if (FORCE) {
                    const size_t fo = (size_t)sg * a.pitch + gx;
                    Fx = __ldg(a.force + fo);
                    Fy = __ldg(a.force + a.plane + fo);
                    jx += c.half_h * rho * Fx;
                    jy += c.half_h * rho * Fy;
                }
                const R inv = recip(rho);
                const R ux = jx * inv, uy = jy * inv;
                R geq[9], F[9];
                equilibrium_dev(drho, rho, ux, uy, geq);
                if (FORCE) force_terms(c.rho0, geq, ux, uy, Fx, Fy, F);
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    R gst = gs[i] + c.b_star * (geq[i] - gs[i]);
                    if (FORCE) gst += c.c_star * F[i];
                    Sw[i][p0] = gst;
                    if (xslot(i) >= 0) sm.S[ring][xslot(i)][t] = gst;
                }
            }
        }
        __syncthreads();
        // ------------------------------------------------------------ C (row r-4)
        if (doC) {
            const int qg = rq;
            rq = rq + 1 == a.ny ? 0 : rq + 1;
            const R my_now = myC;
            myC = __ldg(a.my + rq);
            if (act2) {
                const R dx = c.dt * mxc, dy = c.dt * my_now;
                const size_t off = (size_t)qg * a.pitch + xc;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const R v0 = Sw[i][p2];
                    R acc = sm.Q[p4][i][t];
                    if (cx(i) != 0) {
                        const R *rw = sm.S[rP][xslot(i)];
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
        if (++ring == kStages) {
            ring = 0;
            parity ^= 1u;
        }
    }
};

template <class R, bool FORCE, int NT>
__global__ void __launch_bounds__(NT, sizeof(R) == 4 ? 4 : 2) k_step_fused_tma(const StepArgs<R> a)
{
    constexpr int W = NT - 2 * kHalo;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SmemT<R, NT> &sm = *reinterpret_cast<SmemT<R, NT> *>(smem_raw);

    const int t = threadIdx.x;
    const int x0 = blockIdx.x * W;
    const int xc = x0 - kHalo + t;
    const int y0 = blockIdx.y * a.rows;
    if (y0 >= a.ny) return;  // uniform over the block
    const int y1 = min(y0 + a.rows, a.ny);
    const int gx = wrap_index(xc, a.nx);
    const int iters = (y1 - y0) + 2 * kHalo;
    SweepT<R, FORCE, NT> sw{a, sm, t, gx, xc, (t >= 2) && (t < NT - 2),
                            (t >= kHalo) && (t < NT - kHalo) && (xc < a.nx), a.mx[gx], a.c, a.st,
                            iters};
    sw.ra = wrap_index(y0 - kHalo, a.ny);
    sw.rs = wrap_index(y0 - 2, a.ny);
    sw.rq = y0;
    sw.myB = __ldg(a.my + sw.rs);
    sw.myC = __ldg(a.my + sw.rq);
    sw.ld_row = sw.ra;
    // copy descriptors: 9 pops x (1 or 2 pieces of the wrapped strip)
    if (t < 32) {
        int c, g, len;
        const int np = wrap_piece(x0 - kHalo, NT, a.nx, 1, c, g, len) ? 2 : 1;
        sw.ncp = 9 * np;
        if (t < sw.ncp) {
            const int i = t % 9;
            wrap_piece(x0 - kHalo, NT, a.nx, t / 9, c, g, len);
            sw.cp_dst = smem_addr(&sm.stage[0][i][c]);
            sw.cp_bytes = (uint32_t)len * sizeof(R);
            sw.cp_src = (size_t)i * a.plane + g;
        }
    }
    if (t == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&sm.bar[s], 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (t < 32)
        for (int s = 0; s < kStages && s < iters; ++s) sw.issue(s);

    int k = 0;
    for (; k + 5 <= iters; k += 5) {
        sw.template row<0>(k >= 4, k >= 8);
        sw.template row<1>(k + 1 >= 4, k + 1 >= 8);
        sw.template row<2>(k + 2 >= 4, k + 2 >= 8);
        sw.template row<3>(k + 3 >= 4, k + 3 >= 8);
        sw.template row<4>(k + 4 >= 4, k + 4 >= 8);
    }
    if (k < iters) sw.template row<0>(true, k >= 8);
    if (k + 1 < iters) sw.template row<1>(true, k + 1 >= 8);
    if (k + 2 < iters) sw.template row<2>(true, k + 2 >= 8);
    if (k + 3 < iters) sw.template row<3>(true, k + 3 >= 8);
    if (sw.timed_out) {
        // let copies that may still be in flight land before the CTA exits
        if (t == 0)
            for (int s = 0; s < kStages; ++s) (void)mbar_wait_bounded(&sm.bar[s], sw.parity ^ 1u);
        atomicOr(a.err, 1);
    }
}

template <class R, bool FORCE>
cudaError_t launch_t(const StepArgs<R> &a, cudaStream_t s)
{
    constexpr int NT = 128, W = NT - 2 * kHalo;
    constexpr size_t smem = sizeof(SmemT<R, NT>);
    cudaError_t e = cudaFuncSetAttribute(k_step_fused_tma<R, FORCE, NT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((a.nx + W - 1) / W, (a.ny + a.rows - 1) / a.rows);
    k_step_fused_tma<R, FORCE, NT><<<grid, NT, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

template <class R>
bool fused_tma_ok(int nx, int ny)
{
    return nx % (16 / (int)sizeof(R)) == 0 && nx >= 128 && ny >= 4;
}

template <class R>
cudaError_t launch_fused_tma(const StepArgs<R> &a, cudaStream_t s)
{
    return a.force ? launch_t<R, true>(a, s) : launch_t<R, false>(a, s);
}

template <class R>
int fused_tma_blocks_per_sm()
{
    int n = 0;
    constexpr size_t smem = sizeof(SmemT<R, 128>);
    cudaFuncSetAttribute(k_step_fused_tma<R, false, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_fused_tma<R, false, 128>, 128,
                                                      smem) != cudaSuccess)
        return 0;
    return n;
}

template bool fused_tma_ok<float>(int, int);
template bool fused_tma_ok<double>(int, int);
template cudaError_t launch_fused_tma<float>(const StepArgs<float> &, cudaStream_t);
template cudaError_t launch_fused_tma<double>(const StepArgs<double> &, cudaStream_t);
template int fused_tma_blocks_per_sm<float>();
template int fused_tma_blocks_per_sm<double>();

}  // namespace fdlbm
