// Fused FP32-deviation T2S2-FDLBM step: one warp per tile, two adjacent
// columns per lane in packed FP32x2 arithmetic, no block-level barrier
// anywhere.  On a walled grid (Eq. 3.10) the same launch splits the nodes: the
// interior rectangle, at least 4 nodes from every wall, whose tiles load
// nothing from outside the grid, where the walled scheme and the periodic one
// compute the same values (the central differences next to a wall and the
// wall nodes' Eq. 3.10 reach 4 nodes in at most), runs the warp tile below;
// the frame around it runs the walls sweep (walls_sweep.cuh) in blocks of one
// warp.
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
// Requirements (checked by the host): nx >= 64 and, on a periodic x axis,
// nx % 4 == 0, so that every copy starts on a 16-byte boundary, a window
// crosses the seam at most once, and the two columns of a lane never straddle
// it (on a walled x axis the interior windows start at column 4 and end before
// nx); the state holds fewer than 2^32 values, so that element offsets fit 32
// bits.
#include <cstddef>
#include <cstdint>
#include <cmath>
#include <cstring>
#include <type_traits>

#include <cuda.h>

#include "internal.h"
#include "packed.cuh"
#include "tma.cuh"
#include "frame.cuh"
#include "walls_sweep.cuh"

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

// S2: T2S2-FDLBM2 (Eq. 5.23), whose sweep keeps f^n for the differences of
// L(f^n) in a per-warp shared ring (FN) and L(f^n) for the update two rows
// later (LN); the register window holds f~+ (in T2S2-FDLBM1, fbar^{+,h}, with
// f~+ in the Q ring).  Side rings of 4 columns where a force field or S2
// needs the room.
template <bool FORCE, bool S2 = false>
struct WarpSmem {
    static constexpr bool kSideRing = FORCE || S2;
    float ring[kStages][9][kCols];                // f~ rows of the window, [pop][window column]
    // the same rows at the other side of the seam: 64 columns, or the 4
    // columns next to the seam ([pop][4], one 256-byte slot per row)
    float wrap[kStages][kSideRing ? kSideSlot / 4 : 9 * kCols];
    float fring[FORCE ? kFRing : 1][2][kCols];    // force rows, [component][window column]
    float fwrap[FORCE ? kFRing : 1][kFSideSlot / 4];  // force columns next to the seam, [2][4]
    // (the members an instance does not use shrink to one element, so that
    // they cost no occupancy)
    f2 Q[S2 ? 1 : kQRing][S2 ? 1 : 9][S2 ? 1 : kLanes];  // f~+ of the lane's two columns
    f2 FN[S2 ? kQRing : 1][S2 ? 8 : 1][S2 ? kLanes : 1];  // S2: f^n of populations 1..8, rows r-4 .. r
    f2 LN[S2 ? 3 : 1][S2 ? 8 : 1][S2 ? kLanes : 1];       // S2: scaled L(f^n) of rows r-4 .. r-2
    uint64_t bar[kStages];
};
static_assert(sizeof(WarpSmem<false>) <= 26u * 1024u && sizeof(WarpSmem<true>) <= 23u * 1024u,
              "T2S2-FDLBM1 instances keep 8 warps per SM");
static_assert(offsetof(WarpSmem<false>, wrap) % 128 == 0, "tensor-copy destinations are 128-B aligned");
static_assert(offsetof(WarpSmem<true>, wrap) % 128 == 0, "tensor-copy destinations are 128-B aligned");
static_assert(offsetof(WarpSmem<true>, fring) % 128 == 0, "tensor-copy destinations are 128-B aligned");
static_assert(offsetof(WarpSmem<true>, fwrap) % 128 == 0, "tensor-copy destinations are 128-B aligned");
using WarpSmemS2 = WarpSmem<false, true>;
using WarpSmemS2F = WarpSmem<true, true>;
static_assert(offsetof(WarpSmemS2, wrap) % 128 == 0, "tensor-copy destinations are 128-B aligned");
static_assert(offsetof(WarpSmemS2F, fring) % 128 == 0, "tensor-copy destinations are 128-B aligned");
static_assert(offsetof(WarpSmemS2F, fwrap) % 128 == 0, "tensor-copy destinations are 128-B aligned");

// Scalars and pointers of one step of one grid.
struct ArgsS {
    float *gout;
    const float *mx, *my;
    const float *force;  // [2][ny][pitch]
    int nx, ny, pitch;
    size_t plane;
    int rows;
    // the interior rectangle, columns [xoff + 56 bx, ...) below xend and rows
    // [yoff + rows by, ...) below yend: the whole grid on a periodic one; on a
    // walled axis the nodes at least 4 from the walls whose windows (row
    // tiles) load no column (row) outside the grid, where the walled and the
    // periodic sweep compute the same values.  The frame around it (walled
    // axes) runs the walls sweep in tiles of kFrameW columns and erows rows.
    int xoff, xend, yoff, yend, erows;
    int nix, nframe;  // interior windows per row of tiles; frame tiles (0 on a periodic grid)
    float rho0, h, dt, b_bar, b_til, b_star;
    float w[4];  // wm1, w0, w1, w2
    int *err;
    float inv_rho0;  // incompressible equilibrium only
    RelaxK kstar;    // the relaxation of Eq. 2.52 (b = b_star) as packed weights
    // force field: shifts dt/2 and h/2 of the first moments (Eq. 3.3 and its
    // analogue for fbar), and 3 x the weights of the forcing term in fbar^{+,h}
    // (Eq. 2.34 after Eq. 2.19), f~+ (Eq. 2.20) and f* (Eq. 2.32)
    float hdt, hh, k_bar, k_til, k_star;
    // S2 (T2S2-FDLBM2): Eq. 2.52 at h = dt for f^n, and 3 x the weight of its
    // forcing term
    float b_phys, k_phys;
    int wx, wy;  // walled axes
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

// The same from the neighbouring lanes' pairs L (lane l - 1) and R (lane
// l + 1), read from shared memory instead of shuffled.
__device__ __forceinline__ f2 xtaps_lr(const f2 c[3], int sgn, f2 L, f2 v0, f2 R, f2 acc)
{
    if (sgn > 0) {
        acc = fma2(c[0], make_float2(v0.y, R.x), acc);
        acc = fma2(c[1], make_float2(L.y, v0.x), acc);
        return fma2(c[2], make_float2(L.x, L.y), acc);
    }
    acc = fma2(c[0], make_float2(L.y, v0.x), acc);
    acc = fma2(c[1], make_float2(v0.y, R.x), acc);
    return fma2(c[2], make_float2(R.x, R.y), acc);
}

// The same in y from the lane's own window (rows k-2 .. k+2 as vm2 .. vp2).
__device__ __forceinline__ f2 ytaps(const f2 c[3], int sgn, f2 vm2, f2 vm1, f2 vp1, f2 vp2, f2 acc)
{
    if (sgn > 0) return fma2(c[2], vm2, fma2(c[1], vm1, fma2(c[0], vp1, acc)));
    return fma2(c[2], vp2, fma2(c[1], vp1, fma2(c[0], vm1, acc)));
}

using frame::kFrameNT;
using frame::kFrameW;
using frame::Tile;
using frame::frame_tile;
static_assert(kFrameNT == kLanes && kFrameW == kFrameNT - 2 * walls_sweep::kHalo, "frame tiles");

// Tile (bx, by) of the interior rectangle.
__host__ __device__ inline Tile interior_tile(const ArgsS &a, int bx, int by)
{
    Tile t;
    t.x0 = a.xoff + bx * kW;
    t.xend = a.xend;
    t.y0 = a.yoff + by * a.rows;
    t.y1 = min(t.y0 + a.rows, a.yend);
    return t;
}

// INC: the incompressible equilibrium of He and Luo (velocity from rho0 u).
// GRID: how the update's weights are made to sum to zero (update_weights).
// FORCE: a body-acceleration field (Eqs. 3.3 and 3.12), whose rows arrive by
// tensor copy with the rows of f~ into a 5-row ring (stage B reads row r-2).
// S2: the second sequence of Sec. 2D (T2S2-FDLBM2, h = dt): stage A makes f^n
// (Eq. 2.52) and f~+ (Eq. 2.20); stage B makes fbar = f~+ - dt xi.grad f~+
// and f^{n+1} (Eq. 2.52) as stage B of T2S2-FDLBM1 does from fbar^{+,h}, and
// L(f^n) of its row; stage C adds dt/2 [L(f^n) + L(f^{n+1})] to f~+ (Eq.
// 5.23), both differences with the update weights of scale -dt/2 m.
template <bool INC, bool GRID, bool FORCE, bool S2 = false>
__device__ __forceinline__ void warp_tile(const ArgsS &a, const CUtensorMap *tin,
                                          const CUtensorMap *tside, const CUtensorMap *tf,
                                          const CUtensorMap *tfside, Tile tile,
                                          unsigned char *smem_raw)
{
    using Smem = WarpSmem<FORCE, S2>;
    constexpr bool SIDE = Smem::kSideRing;
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);

    const int l = threadIdx.x;
    const int x0 = tile.x0;  // first output column
    const int y0 = tile.y0, y1 = tile.y1;
    const int iters = (y1 - y0) + 2 * kHalo;
    const int xs = x0 - kHalo;             // window start before wrapping
    const int xc = xs + 2 * l;             // the lane's first column
    const int gx = wrap_index(xc, a.nx);   // even, and gx + 1 < nx
    const bool store = (l >= 2) && (l < kLanes - 2) && (xc < tile.xend);

    // ---- where the lane's pair lands: the main ring, or the side ring filled
    // from x = nx - 4 (first window) or x = 0 (last window)
    const bool wrap_lo = xs < 0, wrap_hi = xs + kCols > a.nx;
    const int wrap_x = wrap_lo ? a.nx - kHalo : 0;
    uint32_t rd = (uint32_t)offsetof(Smem, ring) + 8u * (uint32_t)l;
    uint32_t pstride = kCols * sizeof(float);  // bytes between populations
    uint32_t frd = (uint32_t)offsetof(Smem, fring) + 8u * (uint32_t)l;
    uint32_t fstride = kCols * sizeof(float);  // bytes between force components
    if (!SIDE) {
        if (xc < 0) rd = (uint32_t)offsetof(Smem, wrap) + 4u * (uint32_t)(xc + kHalo);
        if (xc >= a.nx) rd = (uint32_t)offsetof(Smem, wrap) + 4u * (uint32_t)(xc - a.nx);
    } else {
        // side rings of 4 columns; lanes further past the seam read the main
        // ring's zero fill (their values reach no output)
        const int side = xc < 0 ? xc + kHalo : (xc >= a.nx && xc < a.nx + kSide ? xc - a.nx : -1);
        if (side >= 0) {
            rd = (uint32_t)offsetof(Smem, wrap) + 4u * (uint32_t)side;
            pstride = kSide * sizeof(float);
            frd = (uint32_t)offsetof(Smem, fwrap) + 4u * (uint32_t)side;
            fstride = kSide * sizeof(float);
        }
    }
    const unsigned char *rd_base = smem_raw + rd;
    const unsigned char *frd_base = smem_raw + frd;

    // ---- constants: the x weights carry -h m_x (stage B) and -dt m_x (stage C)
    const f2 rho0 = bc(a.rho0);
    const f2 mx2 = make_float2(__ldg(a.mx + gx), __ldg(a.mx + (gx + 1 < a.nx ? gx + 1 : gx)));
    // (S2: the update's two differences at scale -dt/2)
    const f2 nhx = mul2(bc(-a.h), mx2), ndx = mul2(bc(S2 ? -a.hdt : -a.dt), mx2);
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
    const f2 bbar = bc(S2 ? a.b_phys : a.b_bar), btil = bc(a.b_til);

    const uint32_t bar0 = smem_addr(&sm.bar[0]);
    const uint32_t ring0 = smem_addr(&sm.ring[0][0][0]), wrap0 = smem_addr(&sm.wrap[0][0]);
    const uint32_t fring0 = smem_addr(&sm.fring[0][0][0]), fwrap0 = smem_addr(&sm.fwrap[0][0]);
    const bool seam = wrap_lo || wrap_hi;
    const uint32_t tx = SIDE ? kRowBytes + (seam ? 9u * kSide * 4u : 0u) +
                                   (FORCE ? kFRowBytes + (seam ? 2u * kSide * 4u : 0u) : 0u)
                             : (seam ? 2u * kRowBytes : kRowBytes);
    // next row to request
    int ld_row = wrap_index(y0 - kHalo, a.ny);
    // rows into f~ slot `slot` and (force field) force slot `fslot`
    auto issue = [&](int slot, int fslot) {
        if (l == 0) {
            fence_proxy_async();
            const uint32_t bar = bar0 + 8u * (uint32_t)slot;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(tx)
                         : "memory");
            tensor_copy_3d(ring0 + (uint32_t)slot * kRowBytes, tin, xs, ld_row, 0, bar);
            if (!SIDE) {
                if (seam)
                    tensor_copy_3d(wrap0 + (uint32_t)slot * kRowBytes, tin, wrap_x, ld_row, 0, bar);
            } else {
                if (FORCE) tensor_copy_3d(fring0 + (uint32_t)fslot * kFRowBytes, tf, xs, ld_row, 0, bar);
                if (seam) {
                    tensor_copy_3d(wrap0 + (uint32_t)slot * kSideSlot, tside, wrap_x, ld_row, 0, bar);
                    if (FORCE)
                        tensor_copy_3d(fwrap0 + (uint32_t)fslot * kFSideSlot, tfside, wrap_x, ld_row, 0,
                                       bar);
                }
            }
        }
        ld_row = ld_row + 1 == a.ny ? 0 : ld_row + 1;
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
    // rows of stage B (y0 - 6 + k) and C (y0 - 8 + k) at iteration k
    int rs = wrap_index(y0 - 6, a.ny), rq = wrap_index(y0 - 8, a.ny);
    float myB = __ldg(a.my + rs), myC = __ldg(a.my + rq);
    int slot = 0;          // iteration mod 3
    int lw = 0;            // S2: LN slot written at this iteration (mod 3); read: the next one
    uint32_t parity = 0;   // mbarrier phase parity of the current slot
    bool timed_out = false;
    // force of the lane's pair from force slot fs (components x, y)
    auto force_of = [&](int fs, f2 &Fx, f2 &Fy) {
        const unsigned char *src = frd_base + fs * kFRowBytes;
        if (SIDE && fstride != kCols * sizeof(float)) src = frd_base + fs * kFSideSlot;
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
                rd_base + slot * (SIDE && pstride != kCols * sizeof(float) ? kSideSlot : kRowBytes);
            f2 g[9];
#pragma unroll
            for (int i = 0; i < 9; ++i)
                g[i] = *reinterpret_cast<const f2 *>(src + i * (SIDE ? pstride : kCols * sizeof(float)));
            f2 geq[9];
            if (!FORCE) {
                equilibrium2_j(INC ? moments2_j_incomp(g, bc(a.inv_rho0)) : moments2_j(g, rho0), geq);
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const f2 neq = sub2(geq[i], g[i]);
                    if (!S2) {
                        Pw[i][p0] = fma2(bbar, neq, g[i]);
                        sm.Q[PH][i][l] = fma2(btil, neq, g[i]);
                    } else {
                        Pw[i][p0] = fma2(btil, neq, g[i]);                        // f~+
                        if (i > 0) sm.FN[PH][i - 1][l] = fma2(bbar, neq, g[i]);  // f^n
                    }
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
                force_add2(geq, INC ? sub2(rho0, m.drho) : rho0, Fx, Fy, uF, bc(S2 ? a.k_phys : a.k_bar),
                           bc(a.k_til), P, Qv);
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    if (!S2) {
                        Pw[i][p0] = P[i];
                        sm.Q[PH][i][l] = Qv[i];
                    } else {
                        Pw[i][p0] = Qv[i];
                        if (i > 0) sm.FN[PH][i - 1][l] = P[i];
                    }
                }
            }
        }
        // ------------------------------------------------------------ B (row r-2)
        {
            const float myb = myB;
            const float nhy = -a.h * myB;
            rs = rs + 1 == a.ny ? 0 : rs + 1;
            myB = __ldg(a.my + rs);
            const f2 ay[3] = {bc(nhy * a.w[0]), bc(nhy * a.w[2]), bc(nhy * a.w[3])};
            // centre coefficients: 1 + the centre weights of the differences taken
            const f2 c_y = bc(1.f + nhy * a.w[1]);
            const f2 c_d = add2(c_y, cxB);
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
#pragma unroll
            for (int i = 0; i < 9; ++i) Sw[i][p0] = fs[i];
            if (S2) {
                // -dt/2 (m_x D_x + m_y D_y) f^n of row r-2 (Eq. 5.23's L(f^n),
                // scaled as the update's other difference), from the f^n ring:
                // y from the lane's own column, x from the neighbouring lanes'
                // pairs; stored for stage C two rows on
                float tl[3], cl;
                update_weights<GRID>(-a.hdt * myb, a.w, tl, cl);
                const f2 byl[3] = {bc(tl[0]), bc(tl[1]), bc(tl[2])};
                const f2 c_yl = bc(cl), c_dl = add2(c_yl, cxC);
                const int lm = (l + kLanes - 1) & (kLanes - 1), lp = (l + 1) & (kLanes - 1);
#pragma unroll
                for (int i = 1; i < 9; ++i) {
                    const f2 v0 = sm.FN[p2][i - 1][l];
                    f2 acc;
                    if (cx(i) != 0 && cy(i) != 0) acc = mul2(c_dl, v0);
                    else if (cx(i) != 0) acc = mul2(cxC, v0);
                    else acc = mul2(c_yl, v0);
                    if (cx(i) != 0)
                        acc = xtaps_lr(axC, cx(i), sm.FN[p2][i - 1][lm], v0, sm.FN[p2][i - 1][lp], acc);
                    if (cy(i) != 0)
                        acc = ytaps(byl, cy(i), sm.FN[p4][i - 1][l], sm.FN[p3][i - 1][l],
                                    sm.FN[p1][i - 1][l], sm.FN[p0][i - 1][l], acc);
                    sm.LN[lw][i - 1][l] = acc;
                }
            }
        }
        // ------------------------------------------------------------ C (row r-4)
        // f* rows r-6 .. r-2 sit in slots p4, p3, p2, p1, p0 of Sw.
        {
            const int qg = rq;
            rq = rq + 1 == a.ny ? 0 : rq + 1;
            const float ndy = (S2 ? -a.hdt : -a.dt) * myC;
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
            const bool st = store && k >= 8;
            auto put = [&](unsigned off, int i, f2 v) {
                *reinterpret_cast<f2 *>(a.gout + (off + (unsigned)i * plane32)) = v;
            };
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const f2 v0 = Sw[i][p2];
                // T2S2-FDLBM1: f~+ from its ring; S2: f~+ of row r-4 from the
                // window and its L(f^n) term, stored two rows ago
                f2 acc;
                if (!S2) acc = sm.Q[p4][i][l];
                else acc = i == 0 ? Pw[0][p4] : add2(Pw[i][p4], sm.LN[lw == 2 ? 0 : lw + 1][i - 1][l]);
                if (cx(i) != 0 && cy(i) != 0) acc = fma2(c_d, v0, acc);
                else if (cx(i) != 0) acc = fma2(cxC, v0, acc);
                else if (cy(i) != 0) acc = fma2(c_y, v0, acc);
                if (cx(i) != 0) acc = xtaps(axC, cx(i), v0, acc);
                if (cy(i) != 0) acc = ytaps(by, cy(i), Sw[i][p4], Sw[i][p3], Sw[i][p1], Sw[i][p0], acc);
                if (st) put(roff, i, acc);
            }
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
        if (S2) lw = lw == 2 ? 0 : lw + 1;
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

// The interior: tile (blockIdx.x, blockIdx.y) of the rectangle.
template <bool INC, bool GRID, bool FORCE, bool S2>
__global__ void __launch_bounds__(kLanes, FDLBM_WARP_MIN_BLOCKS)
    k_step_fused_warp(const __grid_constant__ ArgsW w)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const Tile tile = interior_tile(w.s, blockIdx.x, blockIdx.y);
    if (tile.y0 >= tile.y1) return;  // uniform over the warp
    warp_tile<INC, GRID, FORCE, S2>(w.s, &w.tin, &w.tside, &w.tf, &w.tfside, tile, smem_raw);
}

// Shared-memory offset of a batch case's scalars, after the rings.
template <bool FORCE>
constexpr size_t kArgsOff = (sizeof(WarpSmem<FORCE>) + 15) / 16 * 16;

__device__ __forceinline__ void copy_words(void *dst, const void *src, int bytes)
{
    const int *s = static_cast<const int *>(src);
    int *d = static_cast<int *>(dst);
    for (int k = threadIdx.x; k < bytes / 4; k += kLanes) d[k] = s[k];
}

// Batched interiors: block blk_off + b is tile (b' - blk_start[c]) of case
// c = blk_case[b'] (nix tiles per row of tiles); the case's tensor maps are
// read from the table in global memory, its scalars from a copy in shared
// memory.
template <bool INC, bool GRID, bool FORCE>
__global__ void __launch_bounds__(kLanes, FDLBM_WARP_MIN_BLOCKS)
    kb_step_fused_warp(const ArgsW *args, const int *blk_case, const int *blk_start, int blk_off)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int b = blk_off + blockIdx.x;
    const int c = blk_case[b];
    const ArgsW &w = args[c];
    ArgsS *sa = reinterpret_cast<ArgsS *>(smem_raw + kArgsOff<FORCE>);
    static_assert(sizeof(ArgsS) % 4 == 0, "argument blocks are copied as 32-bit words");
    copy_words(sa, &w.s, sizeof(ArgsS));
    __syncwarp();
    const int u = b - blk_start[c];
    const Tile tile = interior_tile(*sa, u % sa->nix, u / sa->nix);
    if (tile.y0 >= tile.y1) return;  // uniform over the warp
    warp_tile<INC, GRID, FORCE>(*sa, &w.tin, &w.tside, &w.tf, &w.tfside, tile, smem_raw);
}

// The frame of a walled grid: the walls sweep (walls_sweep.cuh, Eq. 3.10
// inside it) on tiles of kFrameW columns in blocks of one warp, a launch of
// its own before the interior's.  Its rows are a chain of dependent work
// (about 1.6 us each for a lone warp), so the tiles are short -- 8 rows beside
// the interior, 4 in the frame rows of a walled y axis -- and the launch ends
// after about 16 rows of the sweep, all tiles in one wave.
using FrameSmem = walls_sweep::Smem<float, kFrameNT>;
constexpr int kFrameMinBlocks = 12;  // 168 registers, as the 128-column walls sweep
constexpr size_t kFrameArgsOff = (sizeof(FrameSmem) + 15) / 16 * 16;

template <bool FORCE>
__device__ __forceinline__ void frame_sweep(const StepArgs<float> &sa, const Tile &tile,
                                            unsigned char *smem_raw)
{
    auto &sm = *reinterpret_cast<FrameSmem *>(smem_raw);
    walls_sweep::sweep_tile<float, FORCE, kFrameNT, true>(sa, sm, tile.x0, tile.xend, tile.y0, tile.y1);
}

template <bool FORCE>
__global__ void __launch_bounds__(kFrameNT, kFrameMinBlocks)
    k_frame_sweep(const __grid_constant__ ArgsS a, const __grid_constant__ StepArgs<float> sa)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Tile tile;
    if (frame_tile(a, blockIdx.x, tile) >= 0) return;
    frame_sweep<FORCE>(sa, tile, smem_raw);
}

// Batched frames: block blk_off + b is frame tile (b' - frame_start[c]) of
// case c = blk_case[b']; the case's walls-sweep arguments are copied into
// shared memory after the rings.
template <bool FORCE>
__global__ void __launch_bounds__(kFrameNT, kFrameMinBlocks)
    kb_frame_sweep(const ArgsW *args, const StepArgs<float> *sargs, const int *blk_case,
                   const int *frame_start, int blk_off)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int b = blk_off + blockIdx.x;
    const int c = blk_case[b];
    Tile tile;
    if (frame_tile(args[c].s, b - frame_start[c], tile) >= 0) return;
    StepArgs<float> *ss = reinterpret_cast<StepArgs<float> *>(smem_raw + kFrameArgsOff);
    static_assert(sizeof(StepArgs<float>) % 4 == 0, "argument blocks are copied as 32-bit words");
    copy_words(ss, sargs + c, sizeof(StepArgs<float>));
    __syncwarp();
    frame_sweep<FORCE>(*ss, tile, smem_raw);
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
    // walled x: any width (interior windows from column 4, the rest is frame)
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
        if (e == cudaSuccess) e = encode(m->side[b], st[b], nx, ny, pitch, plane, 9, kSide);
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

template <bool INC, bool GRID, bool FORCE, bool S2>
cudaError_t launch_t(const ArgsW &a, dim3 grid, cudaStream_t stream)
{
    constexpr size_t smem = sizeof(WarpSmem<FORCE, S2>);
    auto kern = k_step_fused_warp<INC, GRID, FORCE, S2>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, kLanes, smem, stream>>>(a);
    return cudaGetLastError();
}

template <bool FORCE>
cudaError_t launch_frame_t(const ArgsS &a, const StepArgs<float> &sa, cudaStream_t stream)
{
    constexpr size_t smem = sizeof(FrameSmem);
    cudaError_t e = cudaFuncSetAttribute(k_frame_sweep<FORCE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_frame_sweep<FORCE><<<a.nframe, kFrameNT, smem, stream>>>(a, sa);
    return cudaGetLastError();
}

// Call f with the three instance flags of k as compile-time constants.
template <class F>
cudaError_t dispatch(const WarpKind &k, F &&f)
{
    using T = std::true_type;
    using N = std::false_type;
    auto fo = [&](auto inc, auto gr) { return k.force ? f(inc, gr, T{}) : f(inc, gr, N{}); };
    auto gr = [&](auto inc) { return k.grid ? fo(inc, T{}) : fo(inc, N{}); };
    return k.inc ? gr(T{}) : gr(N{});
}

// The interior rectangle of a grid and its tile counts.  A walled x axis:
// interior windows start at column 4 (loads from 0) and end while their loads
// stay below nx (the last one loads [x0 - 4, x0 + 60)), which leaves a frame
// of 4 columns at the W wall and 4 to 59 at the E wall.  A walled y axis:
// rows [4, ny-4).  Frame tiles beside the interior rows take the fewest rows
// of 4, 8, 16, ... (at most FDLBM_FRAME_MAX_ROWS) for which all frame tiles
// fit one wave of the frame launch: the launch lasts about (rows + 8) rows of
// the sweep.
#ifndef FDLBM_FRAME_MAX_ROWS
#define FDLBM_FRAME_MAX_ROWS 64
#endif
// One wave of the frame launch: 12 blocks per SM for the T2S2-FDLBM1 walls
// sweep (168 registers), fewer for the T2S2-FDLBM2 one.
static int frame_slots(bool s2)
{
    static const int sms = [] {
        int dev = 0, n = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
        return n;
    }();
    static const int per_sm_s2 = std::max(1, frame_s2_blocks_per_sm());
    return sms * (s2 ? per_sm_s2 : kFrameMinBlocks);
}

static void split(ArgsS &a, bool s2)
{
    a.xoff = 0;
    a.xend = a.nx;
    a.yoff = 0;
    a.yend = a.ny;
    a.erows = 4;
    if (a.wx) {
        const int n = a.nx >= kCols ? (a.nx - kCols) / kW + 1 : 0;
        a.xoff = kHalo;
        a.xend = kHalo + kW * n;
    }
    if (a.wy) {
        a.yoff = std::min(kHalo, a.ny);
        a.yend = std::max(a.yoff, a.ny - kHalo);
    }
    a.nix = a.xend > a.xoff ? (a.xend - a.xoff + kW - 1) / kW : 0;
    a.nframe = 0;
    if (a.wx || a.wy) {
        Tile unused;
        for (;;) {
            a.nframe = frame_tile(a, 1 << 30, unused);
            if (a.nframe <= frame_slots(s2) || 2 * a.erows > FDLBM_FRAME_MAX_ROWS) break;
            a.erows *= 2;
        }
    }
}

// Rows of interior tiles; interior tiles.
static int interior_rows(const ArgsS &a)
{
    return a.yend > a.yoff ? (a.yend - a.yoff + a.rows - 1) / a.rows : 0;
}

static int tile_count(const ArgsS &a)
{
    return a.nix > 0 ? a.nix * interior_rows(a) : 0;
}

// The argument block of one grid at ping-pong parity `cur`.
ArgsW make_args(const StepArgs<float> &s, const WarpMaps &maps, int cur)
{
    ArgsW w;
    std::memset(&w, 0, sizeof w);
    const bool force = s.force != nullptr;
    std::memcpy(&w.tin, maps.state[cur], sizeof(CUtensorMap));
    std::memcpy(&w.tside, maps.side[cur], sizeof(CUtensorMap));
    if (force) {
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
    a.b_phys = s.c.b_phys;
    a.k_phys = 3.0f * s.c.c_phys;
    a.wx = s.bc_x == FDLBM_WALL;
    a.wy = s.bc_y == FDLBM_WALL;
    split(a, s.scheme == FDLBM_SCHEME_T2S2_2);
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
    k.s2 = s.scheme == FDLBM_SCHEME_T2S2_2;
    return k;
}

cudaError_t launch_fused_warp(const StepArgs<float> &s, const WarpMaps &maps, int cur,
                              cudaStream_t stream)
{
    if (s.force && !maps.has_force) return cudaErrorInvalidValue;
    const ArgsW a = make_args(s, maps, cur);
    const WarpKind k = warp_kind(s);
    cudaError_t e = cudaSuccess;
    if (a.s.nframe > 0 && k.s2) {
        const FrameGeom g{a.s.nx, a.s.ny, a.s.wx, a.s.wy, a.s.xoff, a.s.xend, a.s.yoff, a.s.yend, a.s.erows,
                          a.s.nframe};
        e = launch_frame_s2(g, s, stream);
    } else if (a.s.nframe > 0) {
        e = s.force ? launch_frame_t<true>(a.s, s, stream) : launch_frame_t<false>(a.s, s, stream);
    }
    if (e != cudaSuccess || tile_count(a.s) <= 0) return e;
    const dim3 grid(a.s.nix, interior_rows(a.s));
    return dispatch(k, [&](auto inc, auto gr, auto fo) {
        constexpr bool I = decltype(inc)::value, G = decltype(gr)::value, F = decltype(fo)::value;
        return k.s2 ? launch_t<I, G, F, true>(a, grid, stream) : launch_t<I, G, F, false>(a, grid, stream);
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

void fused_warp_tiles(const StepArgs<float> &s, int *interior, int *frame)
{
    WarpMaps none;
    std::memset(&none, 0, sizeof none);
    none.has_force = s.force != nullptr;
    const ArgsS a = make_args(s, none, 0).s;
    *interior = tile_count(a);
    *frame = a.nframe;
}

// A batch's interior tiles [blk_off, blk_off + nblocks) of the table, all of
// kind k.
cudaError_t launch_batched_warp(const void *args, const int *blk_case, const int *blk_start,
                                int blk_off, int nblocks, WarpKind k, cudaStream_t stream)
{
    if (nblocks <= 0) return cudaSuccess;
    if (k.s2) return cudaErrorInvalidValue;  // batches run T2S2-FDLBM2 on the scalar sweep
    return dispatch(k, [&](auto inc, auto gr, auto fo) {
        constexpr bool I = decltype(inc)::value, G = decltype(gr)::value, F = decltype(fo)::value;
        constexpr size_t smem = kArgsOff<F> + sizeof(ArgsS);
        auto kern = kb_step_fused_warp<I, G, F>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<nblocks, kLanes, smem, stream>>>(static_cast<const ArgsW *>(args), blk_case, blk_start,
                                                blk_off);
        return cudaGetLastError();
    });
}

// A batch's frame tiles [blk_off, blk_off + nblocks) of the table (cases with
// a force field or all without); sargs: the cases' StepArgs<float>.
cudaError_t launch_batched_frame(const void *args, const void *sargs, const int *blk_case,
                                 const int *frame_start, int blk_off, int nblocks, bool force,
                                 cudaStream_t stream)
{
    if (nblocks <= 0) return cudaSuccess;
    constexpr size_t smem = kFrameArgsOff + sizeof(StepArgs<float>);
    auto kern = force ? kb_frame_sweep<true> : kb_frame_sweep<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<nblocks, kFrameNT, smem, stream>>>(static_cast<const ArgsW *>(args),
                                              static_cast<const StepArgs<float> *>(sargs), blk_case,
                                              frame_start, blk_off);
    return cudaGetLastError();
}

// The tiles of one grid's warp-tile step, host side only: interior windows
// (kind 0: x0, store end, y0, y1) in launch order, then frame tiles (kind 1).
int warp_tile_plan(int nx, int ny, bool wx, bool wy, int rows, bool s2, int *out, int cap)
{
    ArgsS a;
    std::memset(&a, 0, sizeof a);
    a.nx = nx;
    a.ny = ny;
    a.wx = wx;
    a.wy = wy;
    a.rows = std::max(1, std::min(rows, ny));
    split(a, s2);
    int n = 0;
    auto put = [&](int kind, const Tile &t) {
        if (n < cap && out) {
            int *o = out + 5 * n;
            o[0] = kind;
            o[1] = t.x0;
            o[2] = t.xend;
            o[3] = t.y0;
            o[4] = t.y1;
        }
        ++n;
    };
    for (int by = 0; by < interior_rows(a); ++by)
        for (int bx = 0; bx < a.nix; ++bx) {
            const Tile t = interior_tile(a, bx, by);
            if (t.y0 < t.y1) put(0, t);
        }
    for (int t = 0; t < a.nframe; ++t) {
        Tile tile;
        if (frame_tile(a, t, tile) < 0) put(1, tile);
    }
    return n;
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
