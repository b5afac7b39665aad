// Fused FP32-deviation T2S2-FDLBM step for periodic grids: one warp per tile,
// two adjacent columns per lane in packed FP32x2 arithmetic, no block-level
// barrier anywhere.
//
// The scheme is the one of step_fused.cu (stages A, B, C of Sec. 2D per row of
// a bottom-to-top sweep, lags of 2 + 2 rows), laid out so that a warp needs
// nothing from any other warp:
//   - a warp owns a window of 64 columns (lane l: columns 2l and 2l+1 as the
//     .x and .y halves of a float2), of which the middle 56 are its output;
//     the 4 columns on either side are the x-halo of the two difference stages;
//   - every difference in y (Eqs. 2.36-2.38) reads the lane's own register
//     window of the last five rows;
//   - every difference in x reads the neighbouring lanes' centre values by
//     warp shuffle: for the pair (2l, 2l+1) the taps 2l-2 .. 2l+3 are the
//     lane's own pair and the halves of lanes l-1 and l+1;
//   - a row of f~ (all nine populations of the window) arrives in a per-warp
//     shared-memory ring by one tiled tensor copy (TMA, 3-D box 64 x 1 x 9)
//     issued at the end of the row that freed its slot, for the row three
//     ahead; a window that crosses the periodic seam gets its wrapped columns
//     by a second copy into a side ring;
//   - f~+ waits four rows in a per-lane shared-memory ring.
// Lanes 0 and 31 have one neighbour only, so their stage-B values are wrong;
// the stage-C output of lanes 2..29 reads f* of lanes 1..30 only.
//
// Every row runs all three stages with no branch in between: before stage B
// (C) has valid input, in the first 4 (8) rows of a segment, it computes on
// the zero-initialised windows and its results are discarded (stage-C stores
// start at row 8; the stage-B rows it then reads were all written from row 4).
//
// The x-differences use weights pre-multiplied by the column's metric and the
// half step (stage B) or step (stage C), with the centre taps of the x and y
// differences merged into one coefficient.  The equilibria are formed from the
// momentum rho u (packed.cuh), so that only their quadratic term waits for
// 1/rho, and stage B folds the relaxation of Eq. 2.52 into the equilibrium
// (two packed FMAs per population).
//
// Every wait on an mbarrier is bounded: on timeout the warp records an error
// flag, keeps its control flow, waits (bounded) for its copies in flight
// before it exits, and the host reports the flag.
//
// Requirements (checked by the host): nx % 4 == 0 and nx >= 64, so that every
// copy starts on a 16-byte boundary, a window crosses the seam at most once,
// and the two columns of a lane never straddle it; the state holds fewer than
// 2^32 values, so that element offsets fit 32 bits.
#include <cstddef>
#include <cstdint>
#include <cmath>
#include <cstring>
#include <type_traits>

#include <cuda.h>

#include "internal.h"
#include "packed.cuh"
#include "tma.cuh"

namespace fdlbm {
namespace {

using namespace packed;

constexpr int kLanes = 32;
constexpr int kCols = 2 * kLanes;          // window columns per warp
constexpr int kHalo = 4;
constexpr int kW = kCols - 2 * kHalo;      // output columns per warp
constexpr int kStages = 3;                 // rows of f~ buffered / in flight
constexpr int kQRing = 5;                  // f~+ rows r-4 .. r
constexpr unsigned kFull = 0xffffffffu;
// Resident warps per SM the register allocation is sized for: 8 (two per
// scheduler) leaves ptxas up to 255 registers; 12 caps it at 168.
#ifndef FDLBM_WARP_MIN_BLOCKS
#define FDLBM_WARP_MIN_BLOCKS 8
#endif
constexpr uint32_t kRowBytes = 9u * kCols * sizeof(float);

// Columns of the other side of the seam that a seam window needs: 4 (the
// x-halo); with a force field the side rings hold just these (a tensor copy
// of box 4 x 1 x 9, or 4 x 1 x 2 for the force), which keeps the forced
// kernel's shared memory within eight warps per SM.
constexpr int kSide = 4;
constexpr int kFRing = 5;                        // force rows r-2 .. r+2
constexpr uint32_t kSideSlot = 256;              // bytes per side-ring slot (144 used)
constexpr uint32_t kFSideSlot = 128;             // bytes per force side-ring slot (32 used)
constexpr uint32_t kFRowBytes = 2u * kCols * sizeof(float);

template <bool FORCE>
struct WarpSmem {
    float ring[kStages][9][kCols];                // f~ rows of the window, [pop][window column]
    // the same rows at the other side of the seam: 64 columns, or with a force
    // field the 4 columns next to the seam ([pop][4], one 256-byte slot per row)
    float wrap[kStages][FORCE ? kSideSlot / 4 : 9 * kCols];
    float fring[FORCE ? kFRing : 1][2][kCols];    // force rows, [component][window column]
    float fwrap[FORCE ? kFRing : 1][kFSideSlot / 4];  // force columns next to the seam, [2][4]
    f2 Q[kQRing][9][kLanes];                      // f~+ of the lane's two columns
    uint64_t bar[kStages];
};
static_assert(offsetof(WarpSmem<false>, wrap) % 128 == 0, "tensor-copy destinations are 128-B aligned");
static_assert(offsetof(WarpSmem<true>, wrap) % 128 == 0, "tensor-copy destinations are 128-B aligned");
static_assert(offsetof(WarpSmem<true>, fring) % 128 == 0, "tensor-copy destinations are 128-B aligned");
static_assert(offsetof(WarpSmem<true>, fwrap) % 128 == 0, "tensor-copy destinations are 128-B aligned");

// Scalars and pointers of one step of one grid.
struct ArgsS {
    float *gout;
    const float *mx, *my;
    const float *force;  // [2][ny][pitch] (walled grids read it directly at Eq. 3.10)
    int nx, ny, pitch;
    size_t plane;
    int rows;
    // output rectangle: columns [xoff + 56 bx, ...) below xend, rows [yoff + rows by,
    // ...) below yend (the whole grid on a periodic one)
    int xoff, xend, yoff, yend;
    float rho0, h, dt, b_bar, b_til, b_star;
    float w[4];  // wm1, w0, w1, w2
    int *err;
    float inv_rho0;  // incompressible equilibrium only
    RelaxK kstar;    // the relaxation of Eq. 2.52 (b = b_star) as packed weights
    // force field: shifts dt/2 and h/2 of the first moments (Eq. 3.3 and its
    // analogue for fbar), and 3 x the weights of the forcing term in fbar^{+,h}
    // (Eq. 2.34 after Eq. 2.19), f~+ (Eq. 2.20) and f* (Eq. 2.32)
    float hdt, hh, k_bar, k_til, k_star;
    // walled axes (WALLS instances): the velocities of the W, E, S, N walls (Eq. 3.10)
    int wx, wy;
    float uw[4][2];
};

// The arguments of one grid: its tensor maps (kernel parameters, or entries
// of a table in global memory for a batch) and the scalars.
struct ArgsW {
    CUtensorMap tin;    // the input state: dims (nx, ny, 9), box (64, 1, 9)
    CUtensorMap tside;  // the same with box (4, 1, 9) (force field only)
    CUtensorMap tf;     // the force field: dims (nx, ny, 2), box (64, 1, 2)
    CUtensorMap tfside; // the same with box (4, 1, 2)
    ArgsS s;
};

// The weights of the update's differences (stage C) for a scale s = -dt m:
// the taps (offsets +1, -1, -2 for sgn > 0) in t[0..2] and the centre in c,
// with c + t[0] + t[1] + t[2] = 0 exactly, as for the exact weights, so that
// the update of a constant is zero and a periodic uniform grid conserves mass
// and momentum to rounding (separately rounded weights leave a sum of order
// 1e-8 s, a damping that adds up linearly over a long run).
//   GRID = false (requires wm1 >= 0.55 |w1|, beta <= 0.16): t0 = s wm1,
//     t1 = s w1 and c = s w0 rounded; t0 + t1 is exact by Sterbenz's lemma
//     (t0 and -t1 within a factor 2), so is (t0 + t1) + c (ratio 3/4), and
//     t2 = -((t0 + t1) + c) takes up their rounding (1e-8 |s| at most).
//   GRID = true (any beta): each tap rounded to the weight grid of s and c
//     minus their sum, exact on that grid.
// Both sides of a square uniform grid get bit-identical weights, so the
// merged centre of a diagonal population, c_x + c_y = 2c, is exact too.
template <bool GRID>
__device__ __forceinline__ void update_weights(float s, const float w[4], float t[3], float &c)
{
    if (GRID) {
        const WeightGrid g = weight_grid(s);
        t[0] = on_weight_grid(s * w[0], g);
        t[1] = on_weight_grid(s * w[2], g);
        t[2] = on_weight_grid(s * w[3], g);
        c = -((t[0] + t[1]) + t[2]);
    } else {
        t[0] = s * w[0];
        t[1] = s * w[2];
        c = s * w[1];
        t[2] = -((t[0] + t[1]) + c);
    }
}

// The taps other than the centre of sign(c) * D_m f in x for the lane's pair
// (Eq. 2.36 with Eqs. 2.37-2.38), weighted by c[0..2] = weights of the taps
// at offsets +1, -1, -2 (sgn > 0) or -1, +1, +2 (sgn < 0), added to acc.  The
// neighbours' halves come by shuffle from lanes l - 1 and l + 1.
__device__ __forceinline__ f2 xtaps(const f2 c[3], int sgn, f2 v0, f2 acc)
{
    if (sgn > 0) {
        const float Llo = __shfl_up_sync(kFull, v0.x, 1);
        const float Lhi = __shfl_up_sync(kFull, v0.y, 1);
        const float Rlo = __shfl_down_sync(kFull, v0.x, 1);
        acc = fma2(c[0], make_float2(v0.y, Rlo), acc);
        acc = fma2(c[1], make_float2(Lhi, v0.x), acc);
        return fma2(c[2], make_float2(Llo, Lhi), acc);
    }
    const float Lhi = __shfl_up_sync(kFull, v0.y, 1);
    const float Rlo = __shfl_down_sync(kFull, v0.x, 1);
    const float Rhi = __shfl_down_sync(kFull, v0.y, 1);
    acc = fma2(c[0], make_float2(Lhi, v0.x), acc);
    acc = fma2(c[1], make_float2(v0.y, Rlo), acc);
    return fma2(c[2], make_float2(Rlo, Rhi), acc);
}

// Next to a wall (Eq. 3.10 grids) an interior node whose upwind tap would
// reach past the wall takes the central difference alone.  With the value
// past the wall replaced by the quadratic extrapolation 3 f(0) - 3 f(1) + f(2)
// of the three nearest values, the mixed weights of Eq. 2.36 give exactly the
// central difference (the upwind part is exact on quadratics), so every node
// keeps the same weights and the stencil loops the same code.  ghost_x puts
// that value into the column past a wall of x, held by a lane outside the
// grid (or, for an odd width, the padding column of the lane at the east
// wall); all lanes take part in the shuffles.  gw: the lane holds columns -2
// and -1; ge: nx and nx+1 (nx even); go: nx-1 and nx (nx odd).
__device__ __forceinline__ void ghost_x(f2 &v, bool gw, bool ge, bool go)
{
    const float d0 = __shfl_down_sync(kFull, v.x, 1);   // columns xc+2, xc+3, xc+4
    const float d1 = __shfl_down_sync(kFull, v.y, 1);
    const float d2 = __shfl_down_sync(kFull, v.x, 2);
    const float u0 = __shfl_up_sync(kFull, v.x, 1);     // columns xc-2, xc-1, xc-3
    const float u1 = __shfl_up_sync(kFull, v.y, 1);
    const float u2 = __shfl_up_sync(kFull, v.y, 2);
    if (gw) v.y = fmaf(3.f, d0 - d1, d2);   // column -1 from columns 0, 1, 2
    if (ge) v.x = fmaf(3.f, u1 - u0, u2);   // column nx from columns nx-1, nx-2, nx-3
    if (go) v.y = fmaf(3.f, v.x - u1, u0);  // column nx from columns nx-1, nx-2, nx-3
}

// The same in y from the lane's own window (rows k-2 .. k+2 as vm2 .. vp2).
__device__ __forceinline__ f2 ytaps(const f2 c[3], int sgn, f2 vm2, f2 vm1, f2 vp1, f2 vp2, f2 acc)
{
    if (sgn > 0) return fma2(c[2], vm2, fma2(c[1], vm1, fma2(c[0], vp1, acc)));
    return fma2(c[2], vp2, fma2(c[1], vp1, fma2(c[0], vm1, acc)));
}

// INC: the incompressible equilibrium of He and Luo (velocity from rho0 u).
// GRID: how the update's weights are made to sum to zero (update_weights).
// FORCE: a body-acceleration field (Eqs. 3.3 and 3.12), whose rows arrive by
// tensor copy with the rows of f~ into a 5-row ring (stage B reads row r-2).
// WALLS: walled axes (a.wx, a.wy) with Eq. 3.10, by the rules of the scalar
// walls sweep: wall nodes take no part in stages B and C, their f* and new f~
// come from Eq. 3.10 at the nearest interior node (the diagonal one at
// corners, with the W/E wall velocity), and interior nodes whose upwind tap
// would reach past a wall take the central difference alone (here through a
// quadratic ghost value, ghost_x).  Rows and columns past a wall arrive as
// the tensor copy's zero fill and feed no stored value.
template <bool INC, bool GRID, bool FORCE, bool WALLS>
__device__ __forceinline__ void warp_tile(const ArgsS &a, const CUtensorMap *tin,
                                          const CUtensorMap *tside, const CUtensorMap *tf,
                                          const CUtensorMap *tfside, int bx, int by,
                                          unsigned char *smem_raw)
{
    WarpSmem<FORCE> &sm = *reinterpret_cast<WarpSmem<FORCE> *>(smem_raw);

    const int l = threadIdx.x;
    const int x0 = a.xoff + bx * kW;  // first output column
    const int y0 = a.yoff + by * a.rows;
    if (y0 >= a.yend) return;              // uniform over the warp
    const int y1 = min(y0 + a.rows, a.yend);
    const int iters = (y1 - y0) + 2 * kHalo;
    const int xs = x0 - kHalo;             // window start before wrapping
    const int xc = xs + 2 * l;             // the lane's first column
    const bool wxl = WALLS && a.wx, wyl = WALLS && a.wy;
    const int gx = wrap_index(xc, a.nx);   // even, and gx + 1 < nx
    const bool store = (l >= 2) && (l < kLanes - 2) && (xc < a.xend);
    // lanes at a wall of x: west holds columns (0, 1); with nx even east holds
    // (nx-2, nx-1); with nx odd easto holds (nx-1, nx),
    // whose interior neighbour x_j = nx-2 sits in the previous lane (the window
    // that holds column nx-1 shuffles it over: hase)
    const bool odd = (a.nx & 1) != 0;
    const bool west = wxl && xc == 0, east = wxl && !odd && xc == a.nx - 2;
    const bool easto = wxl && odd && xc == a.nx - 1;
    const bool hase = wxl && odd && xs <= a.nx - 1 && a.nx - 1 < xs + kCols;
    // the window holds a wall column (warp-uniform: the wall code that needs
    // every lane, shuffles and warp barriers, runs under these)
    const bool winx = wxl && ((xs <= 0 && 0 < xs + kCols) || (xs <= a.nx - 1 && a.nx - 1 < xs + kCols));
    // lanes that hold the ghost column past a wall of x (ghost_x)
    const bool gw = wxl && xc == -2, ge = wxl && !odd && xc == a.nx, go = easto;

    // ---- where the lane's pair lands: the main ring, or the side ring filled
    // from x = nx - 4 (first window) or x = 0 (last window); a walled x axis
    // has no seam
    const bool wrap_lo = !wxl && xs < 0, wrap_hi = !wxl && xs + kCols > a.nx;
    const int wrap_x = wrap_lo ? a.nx - kHalo : 0;
    uint32_t rd = (uint32_t)offsetof(WarpSmem<FORCE>, ring) + 8u * (uint32_t)l;
    uint32_t pstride = kCols * sizeof(float);  // bytes between populations
    uint32_t frd = (uint32_t)offsetof(WarpSmem<FORCE>, fring) + 8u * (uint32_t)l;
    uint32_t fstride = kCols * sizeof(float);  // bytes between force components
    if (!FORCE) {
        if (!wxl && xc < 0) rd = (uint32_t)offsetof(WarpSmem<FORCE>, wrap) + 4u * (uint32_t)(xc + kHalo);
        if (!wxl && xc >= a.nx) rd = (uint32_t)offsetof(WarpSmem<FORCE>, wrap) + 4u * (uint32_t)(xc - a.nx);
    } else {
        // side rings of 4 columns; lanes further past the seam read the main
        // ring's zero fill (their values reach no output)
        const int side = wxl ? -1 : (xc < 0 ? xc + kHalo : (xc >= a.nx && xc < a.nx + kSide ? xc - a.nx : -1));
        if (side >= 0) {
            rd = (uint32_t)offsetof(WarpSmem<FORCE>, wrap) + 4u * (uint32_t)side;
            pstride = kSide * sizeof(float);
            frd = (uint32_t)offsetof(WarpSmem<FORCE>, fwrap) + 4u * (uint32_t)side;
            fstride = kSide * sizeof(float);
        }
    }
    const unsigned char *rd_base = smem_raw + rd;
    const unsigned char *frd_base = smem_raw + frd;

    // ---- constants: the x weights carry -h m_x (stage B) and -dt m_x (stage C)
    const f2 rho0 = bc(a.rho0);
    const f2 mx2 = make_float2(__ldg(a.mx + gx), __ldg(a.mx + (gx + 1 < a.nx ? gx + 1 : gx)));
    const f2 nhx = mul2(bc(-a.h), mx2), ndx = mul2(bc(-a.dt), mx2);
    const f2 axB[3] = {mul2(nhx, bc(a.w[0])), mul2(nhx, bc(a.w[2])), mul2(nhx, bc(a.w[3]))};
    // stage C: taps on the weight grid of each column and the centre as minus
    // their sum, so that the x weights of the update sum to exactly zero
    // (stage B needs no such care: its result enters the update only through
    // differences)
    f2 axC[3], cxC;
    {
        float tl[3], th[3];
        update_weights<GRID>(ndx.x, a.w, tl, cxC.x);
        update_weights<GRID>(ndx.y, a.w, th, cxC.y);
#pragma unroll
        for (int k = 0; k < 3; ++k) axC[k] = make_float2(tl[k], th[k]);
    }
    const f2 cxB = mul2(nhx, bc(a.w[1]));
    const f2 c_xB = add2(bc(1.f), cxB);
    const f2 bbar = bc(a.b_bar), btil = bc(a.b_til);

    const uint32_t bar0 = smem_addr(&sm.bar[0]);
    const uint32_t ring0 = smem_addr(&sm.ring[0][0][0]), wrap0 = smem_addr(&sm.wrap[0][0]);
    const uint32_t fring0 = smem_addr(&sm.fring[0][0][0]), fwrap0 = smem_addr(&sm.fwrap[0][0]);
    const bool seam = wrap_lo || wrap_hi;
    const uint32_t tx = FORCE ? kRowBytes + kFRowBytes + (seam ? 9u * kSide * 4u + 2u * kSide * 4u : 0u)
                              : (seam ? 2u * kRowBytes : kRowBytes);
    // next row to request (a walled y axis: the logical row, whose copies
    // past the walls are zero-filled)
    int ld_row = wyl ? y0 - kHalo : wrap_index(y0 - kHalo, a.ny);
    // rows into f~ slot `slot` and (force field) force slot `fslot`
    auto issue = [&](int slot, int fslot) {
        if (l == 0) {
            fence_proxy_async();
            const uint32_t bar = bar0 + 8u * (uint32_t)slot;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(tx)
                         : "memory");
            tensor_copy_3d(ring0 + (uint32_t)slot * kRowBytes, tin, xs, ld_row, 0, bar);
            if (!FORCE) {
                if (seam)
                    tensor_copy_3d(wrap0 + (uint32_t)slot * kRowBytes, tin, wrap_x, ld_row, 0, bar);
            } else {
                tensor_copy_3d(fring0 + (uint32_t)fslot * kFRowBytes, tf, xs, ld_row, 0, bar);
                if (seam) {
                    tensor_copy_3d(wrap0 + (uint32_t)slot * kSideSlot, tside, wrap_x, ld_row, 0, bar);
                    tensor_copy_3d(fwrap0 + (uint32_t)fslot * kFSideSlot, tfside, wrap_x, ld_row, 0,
                                   bar);
                }
            }
        }
        ld_row = (!wyl && ld_row + 1 == a.ny) ? 0 : ld_row + 1;
    };

    if (l == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&sm.bar[s], 1);
        mbar_init_fence();
    }
    __syncwarp();
    for (int s = 0; s < kStages && s < iters; ++s) issue(s, s);

    f2 Pw[9][5];  // fbar^{+,h} of the lane's columns, slot = iteration mod 5
    f2 Sw[9][5];  // f*
#pragma unroll
    for (int i = 0; i < 9; ++i)
#pragma unroll
        for (int j = 0; j < 5; ++j) Pw[i][j] = Sw[i][j] = bc(0.f);
    // rows of stage B (y0 - 6 + k) and C (y0 - 8 + k) at iteration k: wrapped
    // (metric and store rows) and logical (walls)
    int rs = wrap_index(y0 - 6, a.ny), rq = wrap_index(y0 - 8, a.ny);
    int rbL = y0 - 6, rcL = y0 - 8;
    float myB = __ldg(a.my + rs), myC = __ldg(a.my + rq);
    int slot = 0;          // iteration mod 3
    uint32_t parity = 0;   // mbarrier phase parity of the current slot
    bool timed_out = false;
    // wall velocities as pairs (both halves alike; corner halves get their own)
    auto uwp = [&](int side, int k) { return bc(a.uw[side][k]); };

    // force of the lane's pair from force slot fs (components x, y)
    auto force_of = [&](int fs, f2 &Fx, f2 &Fy) {
        const unsigned char *src = frd_base + fs * kFRowBytes;
        if (FORCE && fstride != kCols * sizeof(float)) src = frd_base + fs * kFSideSlot;
        Fx = *reinterpret_cast<const f2 *>(src);
        Fy = *reinterpret_cast<const f2 *>(src + fstride);
    };

    auto row = [&](auto PHc, int k) {
        constexpr int PH = decltype(PHc)::value;
        constexpr int p0 = PH, p1 = (PH + 4) % 5, p2 = (PH + 3) % 5, p3 = (PH + 2) % 5,
                      p4 = (PH + 1) % 5;
        // ------------------------------------------------------------ A (row r)
        if (!mbar_wait_bounded(&sm.bar[slot], parity)) timed_out = true;
        {
            const unsigned char *src =
                rd_base + slot * (FORCE && pstride != kCols * sizeof(float) ? kSideSlot : kRowBytes);
            f2 g[9];
#pragma unroll
            for (int i = 0; i < 9; ++i)
                g[i] = *reinterpret_cast<const f2 *>(src + i * (FORCE ? pstride : kCols * sizeof(float)));
            f2 geq[9];
            if (!FORCE) {
                equilibrium2_j(INC ? moments2_j_incomp(g, bc(a.inv_rho0)) : moments2_j(g, rho0), geq);
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const f2 neq = sub2(geq[i], g[i]);
                    Pw[i][p0] = fma2(bbar, neq, g[i]);
                    sm.Q[PH][i][l] = fma2(btil, neq, g[i]);
                }
            } else {
                f2 Fx, Fy;
                force_of(p0, Fx, Fy);
                // Eq. 3.3: rho u = sum xi f~ + (dt/2) rho F
                MacroJ m = INC ? moments2_j_incomp(g, bc(a.inv_rho0)) : moments2_j(g, rho0);
                const f2 hr = mul2(bc(a.hdt), INC ? rho0 : add2(rho0, m.drho));
                m.jx = fma2(hr, Fx, m.jx);
                m.jy = fma2(hr, Fy, m.jy);
                equilibrium2_j(m, geq);
                const f2 uF = mul2(fma2(m.jx, Fx, mul2(m.jy, Fy)), m.inv);
                f2 P[9], Qv[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const f2 neq = sub2(geq[i], g[i]);
                    P[i] = fma2(bbar, neq, g[i]);
                    Qv[i] = fma2(btil, neq, g[i]);
                }
                // Eq. 3.12 at the equilibrium of Eq. 3.2 (at rho0 under the
                // incompressible one)
                force_add2(geq, INC ? sub2(rho0, m.drho) : rho0, Fx, Fy, uF, bc(a.k_bar),
                           bc(a.k_til), P, Qv);
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    Pw[i][p0] = P[i];
                    sm.Q[PH][i][l] = Qv[i];
                }
            }
        }
        // ------------------------------------------------------------ B (row r-2)
        {
            const float nhy = -a.h * myB;
            rs = rs + 1 == a.ny ? 0 : rs + 1;
            myB = __ldg(a.my + rs);
            const f2 ay[3] = {bc(nhy * a.w[0]), bc(nhy * a.w[2]), bc(nhy * a.w[3])};
            // centre coefficients: 1 + the centre weights of the differences taken
            const f2 c_y = bc(1.f + nhy * a.w[1]);
            const f2 c_d = add2(c_y, cxB);
            // next to a wall: the quadratic ghost values past it (ghost_x); the
            // slots they overwrite (rows -1 and ny, columns past the walls) feed
            // no stored value otherwise
            if (WALLS && wyl && rbL == 1) {
#pragma unroll
                for (int i = 0; i < 9; ++i)
                    if (cy(i) > 0) Pw[i][p4] = fma2(bc(3.f), sub2(Pw[i][p3], Pw[i][p2]), Pw[i][p1]);
            }
            if (WALLS && wyl && rbL == a.ny - 2) {
#pragma unroll
                for (int i = 0; i < 9; ++i)
                    if (cy(i) < 0) Pw[i][p0] = fma2(bc(3.f), sub2(Pw[i][p1], Pw[i][p2]), Pw[i][p3]);
            }
            if (WALLS && winx) {
#pragma unroll
                for (int i = 0; i < 9; ++i)
                    if (cx(i) != 0) ghost_x(Pw[i][p2], gw, ge, go);
            }
            f2 gs[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const f2 v0 = Pw[i][p2];
                f2 acc;
                if (cx(i) != 0 && cy(i) != 0) acc = mul2(c_d, v0);
                else if (cx(i) != 0) acc = mul2(c_xB, v0);
                else if (cy(i) != 0) acc = mul2(c_y, v0);
                else acc = v0;
                if (cx(i) != 0) acc = xtaps(axB, cx(i), v0, acc);
                if (cy(i) != 0) acc = ytaps(ay, cy(i), Pw[i][p4], Pw[i][p3], Pw[i][p1], Pw[i][p0], acc);
                gs[i] = acc;
            }
            f2 fs[9];
            if (!FORCE) {
                // Eq. 2.52: f* = f-bar* + b* (f^eq* - f-bar*), folded into the equilibrium
                relax2_j(INC ? moments2_j_incomp(gs, bc(a.inv_rho0)) : moments2_j(gs, rho0), gs, a.kstar, fs);
            } else {
                // Eq. 2.32 with the force of row r-2: rho u = sum xi fbar + (h/2) rho F
                f2 Fx, Fy;
                force_of(p2, Fx, Fy);
                MacroJ m = INC ? moments2_j_incomp(gs, bc(a.inv_rho0)) : moments2_j(gs, rho0);
                const f2 hr = mul2(bc(a.hh), INC ? rho0 : add2(rho0, m.drho));
                m.jx = fma2(hr, Fx, m.jx);
                m.jy = fma2(hr, Fy, m.jy);
                f2 ge[9];
                equilibrium2_j(m, ge);
                const f2 uF = mul2(fma2(m.jx, Fx, mul2(m.jy, Fy)), m.inv);
                const f2 bst = bc(a.b_star);
#pragma unroll
                for (int i = 0; i < 9; ++i) fs[i] = fma2(bst, sub2(ge[i], gs[i]), gs[i]);
                force_add1(ge, INC ? sub2(rho0, m.drho) : rho0, Fx, Fy, uF, bc(a.k_star), fs);
            }
            if (WALLS && wyl && rbL == a.ny - 1) {
                // the N wall row's f*, from the window row ny-2 (Eq. 3.10 on the
                // physical distribution: no force shift)
#pragma unroll
                for (int i = 0; i < 9; ++i) fs[i] = Sw[i][p1];
                const f2 z = bc(0.f);
                nee2<INC, false>(fs, rho0, bc(a.inv_rho0), z, z, z, uwp(FDLBM_WALL_N, 0),
                                 uwp(FDLBM_WALL_N, 1));
            }
#pragma unroll
            for (int i = 0; i < 9; ++i) Sw[i][p0] = fs[i];
            if (WALLS && winx) {
                // the W (E) wall column's f* from column 1 (nx-2): the same lane,
                // or for nx odd the previous one (a shuffle over the whole warp:
                // winx is uniform)
                f2 t[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const float nb = __shfl_up_sync(kFull, Sw[i][p0].y, 1);
                    t[i] = west ? bc(Sw[i][p0].y) : (east ? bc(Sw[i][p0].x) : bc(nb));
                }
                if (west || east || easto) {
                    const f2 z = bc(0.f);
                    const int sd = west ? FDLBM_WALL_W : FDLBM_WALL_E;
                    nee2<INC, false>(t, rho0, bc(a.inv_rho0), z, z, z, uwp(sd, 0), uwp(sd, 1));
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        if (east) Sw[i][p0].y = t[i].y;
                        else Sw[i][p0].x = t[i].x;
                    }
                }
            }
            if (WALLS && wyl && rbL == 1) {
                // the S wall row's f* into the window slot of row 0
                f2 t[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) t[i] = Sw[i][p0];
                const f2 z = bc(0.f);
                nee2<INC, false>(t, rho0, bc(a.inv_rho0), z, z, z, uwp(FDLBM_WALL_S, 0),
                                 uwp(FDLBM_WALL_S, 1));
#pragma unroll
                for (int i = 0; i < 9; ++i) Sw[i][p1] = t[i];
            }
            ++rbL;
        }
        // ------------------------------------------------------------ C (row r-4)
        // f* rows r-6 .. r-2 sit in slots p4, p3, p2, p1, p0 of Sw.
        {
            const int qg = rq;
            rq = rq + 1 == a.ny ? 0 : rq + 1;
            const float ndy = -a.dt * myC;
            myC = __ldg(a.my + rq);
            // the y weights of the update, summing to zero exactly
            float ty[3], cyw;
            update_weights<GRID>(ndy, a.w, ty, cyw);
            const f2 by[3] = {bc(ty[0]), bc(ty[1]), bc(ty[2])};
            const f2 c_y = bc(cyw);
            const f2 c_d = add2(c_y, cxC);
            // element offsets fit 32 bits (9 planes < 2^32 elements, checked on
            // the host): one wide multiply-add per store address
            const unsigned roff = (unsigned)qg * (unsigned)a.pitch + (unsigned)xc;
            const unsigned plane32 = (unsigned)a.plane;
            const bool rowin = !wyl || (rcL >= 1 && rcL <= a.ny - 2);
            const bool st = store && k >= 8 && rowin;
            const bool gS = wyl && rcL == 1, gN = wyl && rcL == a.ny - 2;
            // (the lane at the east wall of an odd grid stores its second value
            // into the padding column nx, which nothing reads)
            auto put = [&](unsigned off, int i, f2 v) {
                *reinterpret_cast<f2 *>(a.gout + (off + (unsigned)i * plane32)) = v;
            };
            if (WALLS && gS) {
#pragma unroll
                for (int i = 0; i < 9; ++i)
                    if (cy(i) > 0) Sw[i][p4] = fma2(bc(3.f), sub2(Sw[i][p3], Sw[i][p2]), Sw[i][p1]);
            }
            if (WALLS && gN) {
#pragma unroll
                for (int i = 0; i < 9; ++i)
                    if (cy(i) < 0) Sw[i][p0] = fma2(bc(3.f), sub2(Sw[i][p1], Sw[i][p2]), Sw[i][p3]);
            }
            if (WALLS && winx) {
#pragma unroll
                for (int i = 0; i < 9; ++i)
                    if (cx(i) != 0) ghost_x(Sw[i][p2], gw, ge, go);
            }
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const f2 v0 = Sw[i][p2];
                f2 acc = sm.Q[p4][i][l];
                if (cx(i) != 0 && cy(i) != 0) acc = fma2(c_d, v0, acc);
                else if (cx(i) != 0) acc = fma2(cxC, v0, acc);
                else if (cy(i) != 0) acc = fma2(c_y, v0, acc);
                if (cx(i) != 0) acc = xtaps(axC, cx(i), v0, acc);
                if (cy(i) != 0) acc = ytaps(by, cy(i), Sw[i][p4], Sw[i][p3], Sw[i][p1], Sw[i][p0], acc);
                if (st) put(roff, i, acc);
            }
            if (WALLS && (winx || gS || gN) && k >= 8) {
                // Eq. 3.10 on the new f~ (force shift dt/2, the force of x_j),
                // from the values just stored: first the W (E) column from
                // column 1 (nx-2), then the S (N) row from row 1 (ny-2); the
                // corners take the value of the wall column at that row (its
                // diagonal x_j with the W/E velocity).  The condition is uniform
                // over the warp, so every lane reaches the warp barriers.
                __syncwarp();
                const f2 ir0 = bc(a.inv_rho0), hd = bc(a.hdt);
                if (st && (west || east || easto)) {
                    const int jx = west ? 1 : a.nx - 2, bx = west ? 0 : a.nx - 1;
                    const unsigned oj = (unsigned)qg * (unsigned)a.pitch + (unsigned)jx;
                    f2 t[9];
#pragma unroll
                    for (int i = 0; i < 9; ++i) t[i] = bc(a.gout[oj + (unsigned)i * plane32]);
                    f2 Fx = bc(0.f), Fy = bc(0.f);
                    if (FORCE) {
                        Fx = bc(__ldg(a.force + oj));
                        Fy = bc(__ldg(a.force + a.plane + oj));
                    }
                    const int sd = west ? FDLBM_WALL_W : FDLBM_WALL_E;
                    nee2<INC, FORCE>(t, rho0, ir0, hd, Fx, Fy, uwp(sd, 0), uwp(sd, 1));
                    const unsigned ob = (unsigned)qg * (unsigned)a.pitch + (unsigned)bx;
#pragma unroll
                    for (int i = 0; i < 9; ++i) a.gout[ob + (unsigned)i * plane32] = t[i].x;
                }
                if (gS || gN) __syncwarp();
                if ((gS || gN) && store) {
                    f2 t[9];
#pragma unroll
                    for (int i = 0; i < 9; ++i)
                        t[i] = *reinterpret_cast<const f2 *>(a.gout + (roff + (unsigned)i * plane32));
                    f2 Fx = bc(0.f), Fy = bc(0.f);
                    if (FORCE) {  // (the force field's padding column reads as any finite value)
                        Fx = __ldg(reinterpret_cast<const float2 *>(a.force + roff));
                        Fy = __ldg(reinterpret_cast<const float2 *>(a.force + a.plane + roff));
                    }
                    float corner[9];
#pragma unroll
                    for (int i = 0; i < 9; ++i) corner[i] = east ? t[i].y : t[i].x;
                    const int sd = gS ? FDLBM_WALL_S : FDLBM_WALL_N;
                    nee2<INC, FORCE>(t, rho0, ir0, hd, Fx, Fy, uwp(sd, 0), uwp(sd, 1));
                    const unsigned wrow = gS ? 0u : (unsigned)(a.ny - 1);
                    const unsigned woff = wrow * (unsigned)a.pitch + (unsigned)xc;
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        f2 v = t[i];
                        if (west || easto) v.x = corner[i];
                        if (east) v.y = corner[i];
                        put(woff, i, v);
                    }
                }
            }
            ++rcL;
        }
        // every lane has read the slot: refill it three rows ahead (force slot
        // (k + 3) mod 5, which stage B has just read).  The copy is issued at
        // the end of the row so that its memory ordering does not split stages
        // A and B, C into separately scheduled regions.
        __syncwarp();
        if (k + kStages < iters) issue(slot, (PH + 3) % 5);
        if (++slot == kStages) {
            slot = 0;
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
        // the last copy into slot s was issued at iteration s + 3 n < iters, in
        // phase n; wait (bounded) for it before the shared memory is released
        for (int s = 0; s < kStages && s < iters; ++s) {
            const int n = (iters - 1 - s) / kStages;
            (void)mbar_wait_bounded(&sm.bar[s], (uint32_t)(n & 1));
        }
        if (l == 0) atomicOr(a.err, 1);
    }
}

template <bool INC, bool GRID, bool FORCE, bool WALLS>
__global__ void __launch_bounds__(kLanes, FDLBM_WARP_MIN_BLOCKS)
    k_step_fused_warp(const __grid_constant__ ArgsW w)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    warp_tile<INC, GRID, FORCE, WALLS>(w.s, &w.tin, &w.tside, &w.tf, &w.tfside, blockIdx.x,
                                       blockIdx.y, smem_raw);
}

// Shared-memory offset of a batch case's scalars, after the rings.
template <bool FORCE>
constexpr size_t kArgsOff = (sizeof(WarpSmem<FORCE>) + 15) / 16 * 16;

// Batched: block blk_off + b is tile (b' - blk_start[c]) of case c = blk_case[b']
// (tiles_x[c] windows per row of tiles); the case's tensor maps are read from
// the table in global memory, its scalars from a copy in shared memory.
template <bool INC, bool GRID, bool FORCE, bool WALLS>
__global__ void __launch_bounds__(kLanes, FDLBM_WARP_MIN_BLOCKS)
    kb_step_fused_warp(const ArgsW *args, const int *blk_case, const int *blk_start,
                       const int *tiles_x, int blk_off)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int b = blk_off + blockIdx.x;
    const int c = blk_case[b];
    const ArgsW &w = args[c];
    ArgsS *sa = reinterpret_cast<ArgsS *>(smem_raw + kArgsOff<FORCE>);
    static_assert(sizeof(ArgsS) % 4 == 0, "scalars are copied as 32-bit words");
    {
        const int *src = reinterpret_cast<const int *>(&w.s);
        int *dst = reinterpret_cast<int *>(sa);
        for (int k = threadIdx.x; k < (int)(sizeof(ArgsS) / 4); k += kLanes) dst[k] = src[k];
    }
    __syncwarp();
    const int lb = b - blk_start[c], ns = tiles_x[c];
    warp_tile<INC, GRID, FORCE, WALLS>(*sa, &w.tin, &w.tside, &w.tf, &w.tfside, lb % ns, lb / ns,
                                       smem_raw);
}

// cuTensorMapEncodeTiled, looked up once through the runtime (no libcuda link).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

}  // namespace

bool fused_warp_ok(int nx, int ny, bool wall_x)
{
    // periodic x: every copy starts on a 16-byte boundary, a window crosses the
    // seam at most once and a lane's pair never straddles it (nx % 4 == 0);
    // walled x: any width (the lanes at the east wall handle either parity)
    const unsigned long long pitch = (nx + 31ull) / 32ull * 32ull;
    const bool cols = wall_x || nx % 4 == 0;
    return cols && nx >= kCols && ny >= 4 && 9ull * pitch * (unsigned long long)ny < (1ull << 32);
}

namespace {

// Tensor map of an FP32 field [depth][ny][pitch]: dims (nx, ny, depth), byte
// strides (4 pitch, 4 plane), box (box_x, 1, depth).  Columns outside [0, nx)
// read as zero (the kernel takes the wrapped ones from the side copies).
cudaError_t encode(unsigned char *map, const float *base, int nx, int ny, int pitch, size_t plane,
                   int depth, int box_x)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    CUtensorMap m;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)depth};
    const cuuint64_t strides[2] = {(cuuint64_t)pitch * sizeof(float), (cuuint64_t)plane * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)box_x, 1, (cuuint32_t)depth};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims,
                          strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    std::memcpy(map, &m, sizeof m);
    return cudaSuccess;
}

}  // namespace

static_assert(sizeof(CUtensorMap) == sizeof(WarpMaps::state[0]), "tensor map size");

// The tensor maps of both ping-pong buffers (and of the force field, if any).
cudaError_t fused_warp_encode(WarpMaps *m, const float *state0, const float *state1,
                              const float *force, int nx, int ny, int pitch, size_t plane)
{
    const float *st[2] = {state0, state1};
    for (int b = 0; b < 2; ++b) {
        cudaError_t e = encode(m->state[b], st[b], nx, ny, pitch, plane, 9, kCols);
        if (e == cudaSuccess && force) e = encode(m->side[b], st[b], nx, ny, pitch, plane, 9, kSide);
        if (e != cudaSuccess) return e;
    }
    m->has_force = force != nullptr;
    if (force) {
        cudaError_t e = encode(m->force, force, nx, ny, pitch, plane, 2, kCols);
        if (e == cudaSuccess) e = encode(m->force_side, force, nx, ny, pitch, plane, 2, kSide);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <bool INC, bool GRID, bool FORCE, bool WALLS>
cudaError_t launch_t(const ArgsW &a, dim3 grid, cudaStream_t stream)
{
    constexpr size_t smem = sizeof(WarpSmem<FORCE>);
    auto kern = k_step_fused_warp<INC, GRID, FORCE, WALLS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, kLanes, smem, stream>>>(a);
    return cudaGetLastError();
}

// Call f with the four instance flags of k as compile-time constants.
template <class F>
cudaError_t dispatch(const WarpKind &k, F &&f)
{
    using T = std::true_type;
    using N = std::false_type;
    auto w = [&](auto inc, auto gr, auto fo) {
        return k.walls ? f(inc, gr, fo, T{}) : f(inc, gr, fo, N{});
    };
    auto fo = [&](auto inc, auto gr) { return k.force ? w(inc, gr, T{}) : w(inc, gr, N{}); };
    auto gr = [&](auto inc) { return k.grid ? fo(inc, T{}) : fo(inc, N{}); };
    return k.inc ? gr(T{}) : gr(N{});
}

// The argument block of one grid at ping-pong parity `cur`.
ArgsW make_args(const StepArgs<float> &s, const WarpMaps &maps, int cur)
{
    ArgsW w;
    std::memset(&w, 0, sizeof w);
    const bool force = s.force != nullptr;
    std::memcpy(&w.tin, maps.state[cur], sizeof(CUtensorMap));
    if (force) {
        std::memcpy(&w.tside, maps.side[cur], sizeof(CUtensorMap));
        std::memcpy(&w.tf, maps.force, sizeof(CUtensorMap));
        std::memcpy(&w.tfside, maps.force_side, sizeof(CUtensorMap));
    }
    ArgsS &a = w.s;
    a.gout = s.gout;
    a.mx = s.mx;
    a.my = s.my;
    a.force = s.force;
    a.nx = s.nx;
    a.ny = s.ny;
    a.pitch = s.pitch;
    a.plane = s.plane;
    a.rows = s.rows;
    a.xoff = 0;
    a.xend = s.nx;
    a.yoff = 0;
    a.yend = s.ny;
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
    a.err = s.err;
    a.inv_rho0 = 1.0f / s.c.rho0;
    a.kstar = make_relax(s.c.b_star);
    a.hdt = s.c.half_dt;
    a.hh = s.c.half_h;
    a.k_bar = 3.0f * s.c.c_bar;
    a.k_til = 3.0f * s.c.c_til;
    a.k_star = 3.0f * s.c.c_star;
    a.wx = s.bc_x == FDLBM_WALL;
    a.wy = s.bc_y == FDLBM_WALL;
    for (int k = 0; k < 4; ++k) {
        a.uw[k][0] = s.wall_u[k][0];
        a.uw[k][1] = s.wall_u[k][1];
    }
    return w;
}

// Which instance a grid needs: the Sterbenz-ordered update weights need
// wm1 >= 0.55 |w1| (beta <= 0.16), else the weights go on their grid.
WarpKind warp_kind(const StepArgs<float> &s)
{
    WarpKind k;
    k.inc = s.c.incomp != 0;
    k.grid = !(s.st.wm1 >= 0.55f * std::fabs(s.st.w1));
    k.force = s.force != nullptr;
    k.walls = s.bc_x == FDLBM_WALL || s.bc_y == FDLBM_WALL;
    return k;
}

cudaError_t launch_fused_warp(const StepArgs<float> &s, const WarpMaps &maps, int cur,
                              cudaStream_t stream)
{
    if (s.force && !maps.has_force) return cudaErrorInvalidValue;
    const ArgsW a = make_args(s, maps, cur);
    const WarpKind k = warp_kind(s);
    const dim3 grid((s.nx + kW - 1) / kW, (s.ny + s.rows - 1) / s.rows);
    return dispatch(k, [&](auto inc, auto gr, auto fo, auto wa) {
        return launch_t<decltype(inc)::value, decltype(gr)::value, decltype(fo)::value,
                        decltype(wa)::value>(a, grid, stream);
    });
}

size_t fused_warp_args_bytes() { return sizeof(ArgsW); }

cudaError_t fused_warp_args(void *dst, const StepArgs<float> &s, const WarpMaps &maps, int cur)
{
    if (s.force && !maps.has_force) return cudaErrorInvalidValue;
    const ArgsW a = make_args(s, maps, cur);
    std::memcpy(dst, &a, sizeof a);
    return cudaSuccess;
}

// A batch's tiles [blk_off, blk_off + nblocks) of the table, all of kind k.
cudaError_t launch_batched_warp(const void *args, const int *blk_case, const int *blk_start,
                                const int *tiles_x, int blk_off, int nblocks, WarpKind k,
                                cudaStream_t stream)
{
    if (nblocks <= 0) return cudaSuccess;
    return dispatch(k, [&](auto inc, auto gr, auto fo, auto wa) {
        constexpr bool I = decltype(inc)::value, G = decltype(gr)::value, F = decltype(fo)::value,
                       W = decltype(wa)::value;
        constexpr size_t smem = kArgsOff<F> + sizeof(ArgsS);
        auto kern = kb_step_fused_warp<I, G, F, W>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<nblocks, kLanes, smem, stream>>>(static_cast<const ArgsW *>(args), blk_case, blk_start,
                                                tiles_x, blk_off);
        return cudaGetLastError();
    });
}

int fused_warp_tile_width() { return kW; }

int fused_warp_blocks_per_sm()
{
    int n = 0;
    constexpr size_t smem = sizeof(WarpSmem<false>);
    auto kern = k_step_fused_warp<false, false, false, false>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kLanes, smem) != cudaSuccess) return 0;
    return n;
}

}  // namespace fdlbm
