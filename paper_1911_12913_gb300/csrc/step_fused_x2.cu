// Fused FP32-deviation T2S2-FDLBM step for periodic grids, two strips per CTA
// in packed FP32x2 arithmetic (sm_100-family f32x2 FMA/ADD/MUL).
//
// The scheme is the same as in step_fused.cu (stages A, B, C of Sec. 2D per
// row of a bottom-to-top sweep; see there), but each thread carries the same
// column of two 128-column strips ("lanes" .x and .y of a float2), so every
// node-local formula and every difference (Eqs. 2.36-2.38) is one packed
// instruction for two nodes.  Strip A covers global columns x0-4 .. x0+123,
// strip B the next 120 columns; each strip keeps its own 4-column x-halo.
//
// Rows of f~ arrive in shared memory by 1-D bulk copies (TMA,
// cp.async.bulk + mbarrier complete_tx) issued by one thread three rows ahead
// of their use; a stage buffer is refilled only after the barrier that follows
// its consumption.  Every wait on an mbarrier is bounded: on timeout the kernel
// records an error flag and carries on (the host reports the flag), so no
// barrier is ever left waiting for an absent thread.
//
// Requirements (checked by the host): nx % 4 == 0 and nx >= 256, so that every
// bulk copy starts and ends on a 16-byte boundary and wraps at most once.
#include <cstdint>
#include <type_traits>

#include "internal.h"
#include "packed.cuh"
#include "tma.cuh"

namespace fdlbm {
namespace {

constexpr int NT = 128;              // threads = columns per strip
constexpr int kHalo = 4;
constexpr int W1 = NT - 2 * kHalo;   // output columns per strip
constexpr int kStages = 3;           // bulk-copy pipeline depth (rows)
constexpr int kRing = 3;             // fbar^{+,h} and f* row rings
constexpr int kQRing = 5;            // f~+ ring (rows r-4 .. r)

using namespace packed;

// ------------------------------------------------------------------ shared memory
struct Smem {
    float stage[kStages][9][2][NT];  // f~ rows, [pop][strip][column]
    f2 P[kRing][6][NT];              // fbar^{+,h} of the x-moving populations
    f2 S[kRing][6][NT];              // f* of the x-moving populations
    f2 Q[kQRing][9][NT];             // f~+ (own column only)
    uint64_t bar[kStages];
};

// ------------------------------------------------------------------ the kernel
struct Args2 {
    const float *gin;
    float *gout;
    const float *mx, *my;
    int nx, ny, pitch;
    size_t plane;
    int rows;
    float rho0, h, dt, b_bar, b_til, b_star;
    float w[4];  // wm1, w0, w1, w2
    int *err;
};

__global__ void __launch_bounds__(NT, 2) k_step_fused_x2(const Args2 a)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);

    const int t = threadIdx.x;
    const int x0 = blockIdx.x * (2 * W1);      // first output column of strip A
    const int y0 = blockIdx.y * a.rows;
    if (y0 >= a.ny) return;                     // uniform over the block
    const int y1 = min(y0 + a.rows, a.ny);
    const int iters = (y1 - y0) + 2 * kHalo;
    // strip s (0 = A, 1 = B) starts at global column xs[s] (before wrapping)
    const int xsA = x0 - kHalo, xsB = x0 + W1 - kHalo;
    const int gxA = wrap_index(xsA + t, a.nx), gxB = wrap_index(xsB + t, a.nx);
    const bool act1 = (t >= 2) && (t < NT - 2);
    const bool inA = (x0 + t - kHalo) < a.nx, inB = (x0 + W1 + t - kHalo) < a.nx;
    const bool act2 = (t >= kHalo) && (t < NT - kHalo);
    const f2 rho0 = bc(a.rho0);
    const f2 mx2 = make_float2(a.mx[gxA], a.mx[gxB]);
    const f2 nhx = mul2(bc(-a.h), mx2), ndx = mul2(bc(-a.dt), mx2);
    const f2 bbar = bc(a.b_bar), btil = bc(a.b_til), bstar = bc(a.b_star);

    // -------- bulk-copy producer: warp 0, one copy per lane.  Each strip's
    // 128 columns wrap at most once, so a row is 9 pops x (1 or 2 pieces) x 2
    // strips <= 36 copies; lane j owns copies j and j + 32.
    int ld_row = wrap_index(y0 - kHalo, a.ny);  // next row to request
    int ld_it = 0;                              // iteration index of that row
    uint32_t cp_dst0 = 0u, cp_dst1 = 0u, cp_bytes0 = 0u, cp_bytes1 = 0u;
    size_t cp_src0 = 0, cp_src1 = 0;            // element offsets within a row block
    int ncp = 0;
    if (t < 32) {
        int j = 0;
        for (int sidx = 0; sidx < 2; ++sidx) {
            const int xs = sidx == 0 ? xsA : xsB;
            int c0 = 0;
            while (c0 < NT) {
                const int g = wrap_index(xs + c0, a.nx);
                const int len = min(NT - c0, a.nx - g);
                for (int i = 0; i < 9; ++i, ++j) {
                    if (j == t) {
                        cp_dst0 = smem_addr(&sm.stage[0][i][sidx][c0]);
                        cp_bytes0 = (uint32_t)len * sizeof(float);
                        cp_src0 = (size_t)i * a.plane + g;
                    } else if (j == t + 32) {
                        cp_dst1 = smem_addr(&sm.stage[0][i][sidx][c0]);
                        cp_bytes1 = (uint32_t)len * sizeof(float);
                        cp_src1 = (size_t)i * a.plane + g;
                    }
                }
                c0 += len;
            }
        }
        ncp = j;
    }
    constexpr uint32_t kStageBytes = 9u * 2u * NT * sizeof(float);
    auto issue = [&](int stage) {
        // warp 0: lane 0 announces the bytes, then every lane issues its copies
        if (t == 0) mbar_expect_tx(&sm.bar[stage], kStageBytes);
        __syncwarp();
        const float *rowbase = a.gin + (size_t)ld_row * a.pitch;
        const uint32_t soff = (uint32_t)stage * 9u * 2u * NT * sizeof(float);
        const uint32_t bar = smem_addr(&sm.bar[stage]);
        if (t < ncp) bulk_copy(cp_dst0 + soff, rowbase + cp_src0, cp_bytes0, bar);
        if (t + 32 < ncp) bulk_copy(cp_dst1 + soff, rowbase + cp_src1, cp_bytes1, bar);
        ld_row = ld_row + 1 == a.ny ? 0 : ld_row + 1;
        ++ld_it;
    };

    if (t == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&sm.bar[s], 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (t < 32)
        for (int s = 0; s < kStages && s < iters; ++s) issue(s);

    f2 Pw[9][5];  // fbar^{+,h} window, slot = iteration mod 5
    f2 Sw[9][5];  // f* window
    int rs = wrap_index(y0 - 2, a.ny), rq = y0;
    float myB = __ldg(a.my + rs), myC = __ldg(a.my + rq);  // metric of the next B / C row
    int ring = 0;           // iteration mod 3 (P/S rings, stage buffers)
    uint32_t parity = 0;    // mbarrier phase of the current stage
    bool timed_out = false;

    auto row = [&](auto PHc, int k) {
        constexpr int PH = decltype(PHc)::value;
        constexpr int p0 = PH, p1 = (PH + 4) % 5, p2 = (PH + 3) % 5, p3 = (PH + 2) % 5,
                      p4 = (PH + 1) % 5;
        // ------------------------------------------------------------ A
        if (!mbar_wait_bounded(&sm.bar[ring], parity)) timed_out = true;
        {
            f2 g[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) g[i] = make_float2(sm.stage[ring][i][0][t], sm.stage[ring][i][1][t]);
            const Macro m = moments2(g, rho0);
            f2 geq[9];
            equilibrium2(m, geq);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const f2 neq = sub2(geq[i], g[i]);
                const f2 gb = fma2(bbar, neq, g[i]);
                const f2 gt = fma2(btil, neq, g[i]);
                Pw[i][p0] = gb;
                if (xslot(i) >= 0) sm.P[ring][xslot(i)][t] = gb;
                sm.Q[PH][i][t] = gt;
            }
        }
        __syncthreads();
        // stage `ring` is free: request the row three iterations ahead into it
        if (t < 32 && ld_it < iters) {
            fence_proxy_async();
            issue(ring);
        }
        // ------------------------------------------------------------ B (row r-2)
        const int rP = ring == 0 ? 1 : (ring == 1 ? 2 : 0);  // (k-2) mod 3 = (k+1) mod 3
        if (k >= 4) {
            rs = rs + 1 == a.ny ? 0 : rs + 1;
            const float my_now = myB;
            myB = __ldg(a.my + rs);
            if (act1) {
                const f2 nhy = bc(-a.h * my_now);
                f2 gs[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const f2 v0 = Pw[i][p2];
                    f2 acc = v0;
                    if (cx(i) != 0) {
                        const f2 *rw = sm.P[rP][xslot(i)];
                        acc = fma2(nhx, stencil2(a.w, cx(i), rw[t - 2], rw[t - 1], v0, rw[t + 1], rw[t + 2]), acc);
                    }
                    if (cy(i) != 0)
                        acc = fma2(nhy, stencil2(a.w, cy(i), Pw[i][p4], Pw[i][p3], v0, Pw[i][p1], Pw[i][p0]), acc);
                    gs[i] = acc;
                }
                const Macro m = moments2(gs, rho0);
                f2 geq[9];
                equilibrium2(m, geq);
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const f2 gst = fma2(bstar, sub2(geq[i], gs[i]), gs[i]);
                    Sw[i][p0] = gst;
                    if (xslot(i) >= 0) sm.S[ring][xslot(i)][t] = gst;
                }
            }
        }
        __syncthreads();
        // ------------------------------------------------------------ C (row r-4)
        if (k >= 8) {
            const int qg = rq;
            rq = rq + 1 == a.ny ? 0 : rq + 1;
            const float my_now = myC;
            myC = __ldg(a.my + rq);
            if (act2) {
                const f2 ndy = bc(-a.dt * my_now);
                const size_t off = (size_t)qg * a.pitch;
                const int xA = x0 + t - kHalo, xB = x0 + W1 + t - kHalo;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const f2 v0 = Sw[i][p2];
                    f2 acc = sm.Q[p4][i][t];
                    if (cx(i) != 0) {
                        const f2 *rw = sm.S[rP][xslot(i)];
                        acc = fma2(ndx, stencil2(a.w, cx(i), rw[t - 2], rw[t - 1], v0, rw[t + 1], rw[t + 2]), acc);
                    }
                    if (cy(i) != 0)
                        acc = fma2(ndy, stencil2(a.w, cy(i), Sw[i][p4], Sw[i][p3], v0, Sw[i][p1], Sw[i][p0]), acc);
                    float *dst = a.gout + i * a.plane + off;
                    if (inA) dst[xA] = acc.x;
                    if (inB) dst[xB] = acc.y;
                }
            }
        }
        // advance the stage ring (and the mbarrier phase when it wraps)
        if (++ring == kStages) {
            ring = 0;
            parity ^= 1u;
        }
    };

    for (int k = 0; k < iters; k += 5) {
        row(std::integral_constant<int, 0>{}, k);
        if (k + 1 < iters) row(std::integral_constant<int, 1>{}, k + 1);
        if (k + 2 < iters) row(std::integral_constant<int, 2>{}, k + 2);
        if (k + 3 < iters) row(std::integral_constant<int, 3>{}, k + 3);
        if (k + 4 < iters) row(std::integral_constant<int, 4>{}, k + 4);
    }
    if (timed_out) {
        // give copies that may still be in flight a last bounded chance to land
        // before the CTA's shared memory is released
        if (t == 0)
            for (int s = 0; s < kStages; ++s) (void)mbar_wait_bounded(&sm.bar[s], parity ^ 1u);
        atomicOr(a.err, 1);
    }
}

}  // namespace

bool fused_x2_ok(int nx, int ny) { return nx % 4 == 0 && nx >= 256 && ny >= 4; }

cudaError_t launch_fused_x2(const StepArgs<float> &s, int *err, cudaStream_t stream)
{
    Args2 a;
    a.gin = s.gin;
    a.gout = s.gout;
    a.mx = s.mx;
    a.my = s.my;
    a.nx = s.nx;
    a.ny = s.ny;
    a.pitch = s.pitch;
    a.plane = s.plane;
    a.rows = s.rows;
    a.rho0 = s.c.rho0;
    a.h = s.c.h;
    a.dt = s.c.dt;
    a.b_bar = s.c.b_bar;
    a.b_til = s.c.b_til;
    a.b_star = s.c.b_star;
    a.w[0] = s.st.wm1;
    a.w[1] = s.st.w0;
    a.w[2] = s.st.w1;
    a.w[3] = s.st.w2;
    a.err = err;
    constexpr size_t smem = sizeof(Smem);
    cudaError_t e = cudaFuncSetAttribute(k_step_fused_x2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((s.nx + 2 * W1 - 1) / (2 * W1), (s.ny + s.rows - 1) / s.rows);
    k_step_fused_x2<<<grid, NT, smem, stream>>>(a);
    return cudaGetLastError();
}

int fused_x2_tile_width() { return 2 * W1; }

int fused_x2_blocks_per_sm()
{
    int n = 0;
    constexpr size_t smem = sizeof(Smem);
    cudaFuncSetAttribute(k_step_fused_x2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_fused_x2, NT, smem) != cudaSuccess)
        return 0;
    return n;
}

}  // namespace fdlbm
