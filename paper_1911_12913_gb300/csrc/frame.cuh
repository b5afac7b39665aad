// Tiles of the frame of a walled grid (the nodes within 4 of a wall, or
// beside the interior rectangle that the warp-tile kernel covers), shared by
// the frame launches of both schemes.  G is any geometry with the fields nx,
// ny, wx, wy (walled axes), xoff, xend, yoff, yend (the interior rectangle)
// and erows (frame tile height beside the interior rows).
#pragma once

namespace fdlbm {
namespace frame {

// The frame runs the walls sweeps in blocks of one warp, one column per
// thread: 24 output columns per tile (32 less the 4-column halo on each side).
constexpr int kFrameNT = 32;
constexpr int kFrameW = kFrameNT - 8;

// One tile of a launch: its first output column x0, the end of the columns
// it stores, and its rows [y0, y1).
struct Tile {
    int x0, xend, y0, y1;
};

// Segment s of an axis of a walled grid: 0 the low frame, 1 the interior
// rectangle, 2 the high frame (on a periodic axis the interior is the whole
// axis and the frames are empty).
template <class G>
__host__ __device__ inline void x_segment(const G &a, int s, int &lo, int &hi)
{
    if (!a.wx) {
        lo = 0;
        hi = s == 1 ? a.nx : 0;
        return;
    }
    lo = s == 0 ? 0 : (s == 1 ? a.xoff : a.xend);
    hi = s == 0 ? min(a.xoff, a.xend) : (s == 1 ? a.xend : a.nx);
}

template <class G>
__host__ __device__ inline void y_segment(const G &a, int s, int &lo, int &hi)
{
    if (!a.wy) {
        lo = 0;
        hi = s == 1 ? a.ny : 0;
        return;
    }
    lo = s == 0 ? 0 : (s == 1 ? a.yoff : a.yend);
    hi = s == 0 ? a.yoff : (s == 1 ? a.yend : a.ny);
}

// Tile t of the frame (the segment pairs other than interior x interior, in
// tiles of kFrameW columns and, beside the interior rows, erows rows; the
// frame rows of a walled y axis are one tile of at most 4 rows).  Returns the
// number of frame tiles when t is past the last one (then `out` is unset),
// else -1.
template <class G>
__host__ __device__ inline int frame_tile(const G &a, int t, Tile &out)
{
    int n = 0;
    for (int sy = 0; sy < 3; ++sy) {
        int ylo, yhi;
        y_segment(a, sy, ylo, yhi);
        if (yhi <= ylo) continue;
        const int h = sy == 1 ? a.erows : yhi - ylo;
        const int nt = (yhi - ylo + h - 1) / h;
        for (int sx = 0; sx < 3; ++sx) {
            if (sx == 1 && sy == 1) continue;
            int xlo, xhi;
            x_segment(a, sx, xlo, xhi);
            if (xhi <= xlo) continue;
            const int nw = (xhi - xlo + kFrameW - 1) / kFrameW;
            if (t >= n && t < n + nw * nt) {
                const int u = t - n;
                out.x0 = xlo + (u % nw) * kFrameW;
                out.xend = xhi;
                out.y0 = ylo + (u / nw) * h;
                out.y1 = min(out.y0 + h, yhi);
                return -1;
            }
            n += nw * nt;
        }
    }
    return n;
}

}  // namespace frame
}  // namespace fdlbm
