// Fused T2S2-FDLBM step for periodic grids, each thread prefetching its own
// column two rows ahead with cp.async.
//
// Same sweep as step_fused.cu (per row r: stage A at row r, stage B at r-2,
// stage C at r-4; see the comment there).  Rows of f~ do not pass through
// registers: every thread copies the 9 values of its own column for row r+2
// into a shared-memory slot with cp.async (one commit group per row) and
// waits for row r's group before stage A.  A thread only ever reads what it
// copied itself, so the load pipeline needs no barrier and no producer warp.
// Stage A overwrites the slot with f~+ of the same row, which stage C reads
// four rows later, so one 7-slot ring (rows r-4 .. r+2) holds both.
//
// Shared rings with one barrier per row (after A): fbar^{+,h} needs 4 slots
// (written by A(k), read by B(k+2), rewritten by A(k+4) after barrier k+3);
// f* needs 3 (written by B(k), read by C(k+2), rewritten by B(k+3) after
// barrier k+3).  FP32 totals 53.8 KB, so four 128-thread CTAs fit an SM.
#include <cstdint>

#include "internal.h"
#include "tma.cuh"

namespace fdlbm {
namespace {

constexpr int kHalo = 4;
constexpr int kAhead = 2;          // rows in flight ahead of stage A
constexpr int kQ = 5 + kAhead;     // own-column ring: rows r-4 .. r+2
constexpr int kP = 4, kS = 3;

template <class R, int NT>
struct SmemA {
    R P[kP][6][NT];   // fbar^{+,h} of the x-moving populations
    R S[kS][6][NT];   // f* of the x-moving populations
    R Q[kQ][9][NT];   // own column: f~ as copied, then f~+ of the same row
};

template <class R>
__device__ __forceinline__ R recip_a(R v)
{
    return R(1) / v;
}
template <>
__device__ __forceinline__ float recip_a<float>(float v)
{
    return __frcp_rn(v);
}

template <int BYTES>
__device__ __forceinline__ void cp_async(uint32_t dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(dst), "l"(src), "n"(BYTES)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <class R, bool FORCE, int NT>
struct SweepA {
    const StepArgs<R> a;
    SmemA<R, NT> &sm;
    const int t, gx, xc;
    const bool act1, act2;
    const R mxc;
    const Coeffs<R> c;
    const Stencil<R> st;
    const int iters;
    R Pw[9][5];
    R Sw[9][5];
    int ra, rs, rq, rl;          // rows of stage A, B, C and of the next copy (wrapped)
    int ld_it = 0;               // iteration index of the next copy
    R myB, myC;
    int qa = 0, pa = 0, sa = 0;  // ring slots of the current row in Q, P, S
    int ql = 0;                  // Q slot of the next copy

    // copy the 9 values of this thread's column of row `rl` into Q slot `ql`
    __device__ void fetch()
    {
        const R *src = a.gin + (size_t)rl * a.pitch + gx;
#pragma unroll
        for (int i = 0; i < 9; ++i)
            cp_async<sizeof(R)>(smem_addr(&sm.Q[ql][i][t]), src + i * a.plane);
        cp_commit();
        rl = rl + 1 == a.ny ? 0 : rl + 1;
        ql = ql + 1 == kQ ? 0 : ql + 1;
        ++ld_it;
    }

    template <int PH>
    __device__ void row(bool doB, bool doC)
    {
        constexpr int p0 = PH, p1 = (PH + 4) % 5, p2 = (PH + 3) % 5, p3 = (PH + 2) % 5,
                      p4 = (PH + 1) % 5;
        // keep kAhead rows in flight (an empty group past the last row keeps
        // the wait count uniform)
        if (ld_it < iters) fetch();
        else cp_commit();
        cp_wait<kAhead>();
        // ------------------------------------------------------------ A (row r)
        {
            R g[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) g[i] = sm.Q[qa][i][t];
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
            const R inv = recip_a(rho);
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
                if (xslot(i) >= 0) sm.P[pa][xslot(i)][t] = gb;
                sm.Q[qa][i][t] = gt;
            }
        }
        __syncthreads();
        // ------------------------------------------------------------ B (row r-2)
        if (doB) {
            const int sg = rs;
            rs = rs + 1 == a.ny ? 0 : rs + 1;
            const R my_now = myB;
            myB = __ldg(a.my + rs);
            if (act1) {
                const int pb = pa >= 2 ? pa - 2 : pa + kP - 2;  // slot of row r-2
                const R hx = c.h * mxc, hy = c.h * my_now;
                R gs[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const R v0 = Pw[i][p2];
                    R acc = v0;
                    if (cx(i) != 0) {
                        const R *rw = sm.P[pb][xslot(i)];
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
                const R inv = recip_a(rho);
                const R ux = jx * inv, uy = jy * inv;
                R geq[9], F[9];
                equilibrium_dev(drho, rho, ux, uy, geq);
                if (FORCE) force_terms(c.rho0, geq, ux, uy, Fx, Fy, F);
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    R gst = gs[i] + c.b_star * (geq[i] - gs[i]);
                    if (FORCE) gst += c.c_star * F[i];
                    Sw[i][p0] = gst;
                    if (xslot(i) >= 0) sm.S[sa][xslot(i)][t] = gst;
                }
            }
        }
        // ------------------------------------------------------------ C (row r-4)
        // f* of row r-4 was written by B two rows ago (slot sa-2 mod 3), f~+ of
        // row r-4 by A four rows ago (slot qa-4 mod 7).
        if (doC) {
            const int qg = rq;
            rq = rq + 1 == a.ny ? 0 : rq + 1;
            const R my_now = myC;
            myC = __ldg(a.my + rq);
            if (act2) {
                const int sc = sa == 2 ? 0 : sa + 1;
                const int qc = qa >= 4 ? qa - 4 : qa + kQ - 4;
                const R dx = c.dt * mxc, dy = c.dt * my_now;
                const size_t off = (size_t)qg * a.pitch + xc;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const R v0 = Sw[i][p2];
                    R acc = sm.Q[qc][i][t];
                    if (cx(i) != 0) {
                        const R *rw = sm.S[sc][xslot(i)];
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
        qa = qa + 1 == kQ ? 0 : qa + 1;
        pa = pa + 1 == kP ? 0 : pa + 1;
        sa = sa + 1 == kS ? 0 : sa + 1;
    }
};

template <class R, bool FORCE, int NT>
__global__ void __launch_bounds__(NT, sizeof(R) == 4 ? 4 : 2) k_step_fused_async(const StepArgs<R> a)
{
    constexpr int W = NT - 2 * kHalo;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SmemA<R, NT> &sm = *reinterpret_cast<SmemA<R, NT> *>(smem_raw);

    const int t = threadIdx.x;
    const int x0 = blockIdx.x * W;
    const int xc = x0 - kHalo + t;
    const int y0 = blockIdx.y * a.rows;
    if (y0 >= a.ny) return;  // uniform over the block
    const int y1 = min(y0 + a.rows, a.ny);
    const int gx = wrap_index(xc, a.nx);
    const int iters = (y1 - y0) + 2 * kHalo;
    SweepA<R, FORCE, NT> sw{a, sm, t, gx, xc, (t >= 2) && (t < NT - 2),
                            (t >= kHalo) && (t < NT - kHalo) && (xc < a.nx), a.mx[gx], a.c, a.st,
                            iters};
    sw.ra = wrap_index(y0 - kHalo, a.ny);
    sw.rl = sw.ra;
    sw.rs = wrap_index(y0 - 2, a.ny);
    sw.rq = y0;
    sw.myB = __ldg(a.my + sw.rs);
    sw.myC = __ldg(a.my + sw.rq);
    // rows 0 .. kAhead-1 in flight before the first row (iters >= 9 > kAhead)
    for (int k = 0; k < kAhead; ++k) sw.fetch();

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
    cp_wait<0>();
}

template <class R, bool FORCE>
cudaError_t launch_a(const StepArgs<R> &a, cudaStream_t s)
{
    constexpr int NT = 128, W = NT - 2 * kHalo;
    constexpr size_t smem = sizeof(SmemA<R, NT>);
    cudaError_t e = cudaFuncSetAttribute(k_step_fused_async<R, FORCE, NT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((a.nx + W - 1) / W, (a.ny + a.rows - 1) / a.rows);
    k_step_fused_async<R, FORCE, NT><<<grid, NT, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

template <class R>
cudaError_t launch_fused_async(const StepArgs<R> &a, cudaStream_t s)
{
    return a.force ? launch_a<R, true>(a, s) : launch_a<R, false>(a, s);
}

template <class R>
int fused_async_blocks_per_sm()
{
    int n = 0;
    constexpr size_t smem = sizeof(SmemA<R, 128>);
    cudaFuncSetAttribute(k_step_fused_async<R, false, 128>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_fused_async<R, false, 128>, 128,
                                                      smem) != cudaSuccess)
        return 0;
    return n;
}

template cudaError_t launch_fused_async<float>(const StepArgs<float> &, cudaStream_t);
template cudaError_t launch_fused_async<double>(const StepArgs<double> &, cudaStream_t);
template int fused_async_blocks_per_sm<float>();
template int fused_async_blocks_per_sm<double>();

}  // namespace fdlbm
