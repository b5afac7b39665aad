"""The warp-tile kernel's split of a grid, read from the library itself
(fdlbm_tile_plan, no GPU): the interior windows and the frame tiles together
store every node exactly once; the interior windows load nothing outside the
grid on a walled axis and stay 4 nodes from every wall (there the walled and
the periodic scheme compute the same values: Eq. 3.10 and the central
differences next to a wall reach 4 nodes in); every interior window starts its
tensor copy on a 16-byte boundary."""
import ctypes

import numpy as np
import pytest

import inputs as I


@pytest.fixture(scope="module")
def B():
    from paper_1911_12913_gb300 import binding
    from paper_1911_12913_gb300 import build as b
    b.build()
    binding.load()
    return binding


def _axis(walled, n):
    return I.wall_axis(n - 1, 0.0, 1.0) if walled else I.periodic_axis(n, 0.0, 1.0)


def _plan(B, nx, ny, wx, wy, rows, scheme):
    """scheme 1 or 2: T2S2-FDLBM1 / T2S2-FDLBM2."""
    L = B.load()
    scheme = {1: B.SCHEME_T2S2_1, 2: B.SCHEME_T2S2_2}[scheme]
    grid, keep = B.make_grid(_axis(wx, nx), _axis(wy, ny))
    count = ctypes.c_int(0)
    st = L.fdlbm_tile_plan(ctypes.byref(grid), rows, scheme, None, 0, ctypes.byref(count))
    assert st == 0, st
    tiles = np.zeros((count.value, 5), dtype=np.int32)
    st = L.fdlbm_tile_plan(ctypes.byref(grid), rows, scheme, tiles.ctypes.data_as(ctypes.c_void_p),
                           count.value, ctypes.byref(count))
    assert st == 0 and count.value == len(tiles)
    return tiles


def _check(B, nx, ny, wx, wy, rows, scheme):
    tiles = _plan(B, nx, ny, wx, wy, rows, scheme)
    hits = np.zeros((ny, nx), dtype=np.int32)
    for kind, x0, xend, y0, y1 in tiles:
        assert 0 <= y0 < y1 <= ny
        width = 56 if kind == 0 else 24
        x1 = min(x0 + width, xend, nx) if wx else min(x0 + width, xend)
        assert x1 > x0
        if kind == 0:
            assert (x0 - 4) % 4 == 0                  # tensor copies on 16-byte boundaries
            if wx:
                assert x0 - 4 >= 0 and x0 + 60 <= nx  # loads inside the grid
                assert x0 >= 4 and x1 <= nx - 4       # 4 nodes from the walls
            if wy:
                assert y0 - 4 >= 0 and y1 + 4 <= ny
        cols = np.arange(x0, x1) % nx
        hits[y0:y1, cols] += 1
    assert hits.min() == 1 and hits.max() == 1, (nx, ny, wx, wy, rows, np.argwhere(hits != 1)[:5])
    return tiles


@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("wx,wy", [(True, True), (False, True), (True, False)])
def test_split_covers_every_node_once(B, wx, wy, scheme):
    """Widths 64..300 (odd and even, one window to several, with and without
    interior windows), heights down to 4 rows, tile heights 1 to 64."""
    for nx in list(range(64, 200, 3)) + [201, 224, 257, 281, 300]:
        if not wx and nx % 4:
            continue
        for ny, rows in ((4, 1), (5, 2), (7, 3), (8, 64), (9, 4), (21, 5), (40, 8), (97, 16)):
            _check(B, nx, ny, wx, wy, rows, scheme)


def test_split_full_size(B):
    """The 4097^2 cavity and the 4096 x 4097 channel at the automatic tile
    height of 257 rows: the interior is one window short of the periodic
    grid's 74 per row, and the frame tiles are short (8 rows beside the
    interior) so that they fit one wave."""
    tiles = _check(B, 4097, 4097, True, True, 257, 1)
    inner = tiles[tiles[:, 0] == 0]
    frame = tiles[tiles[:, 0] == 1]
    assert len(inner) == 73 * 16
    assert (frame[:, 4] - frame[:, 3]).max() <= 8
    tiles = _check(B, 4096, 4097, False, True, 257, 2)
    assert (tiles[tiles[:, 0] == 1][:, 4] - tiles[tiles[:, 0] == 1][:, 3]).max() <= 16


def test_plan_rejects(B):
    L = B.load()
    grid, keep = B.make_grid(I.periodic_axis(130, 0.0, 1.0), I.periodic_axis(64, 0.0, 1.0))
    count = ctypes.c_int(0)
    # 130 % 4 != 0 on a periodic axis: the warp-tile kernel does not apply
    assert L.fdlbm_tile_plan(ctypes.byref(grid), 8, B.SCHEME_T2S2_1, None, 0, ctypes.byref(count)) == -5
    grid2, keep2 = B.make_grid(I.periodic_axis(128, 0.0, 1.0), I.periodic_axis(64, 0.0, 1.0))
    assert L.fdlbm_tile_plan(ctypes.byref(grid2), 0, B.SCHEME_T2S2_1, None, 0, ctypes.byref(count)) == -1
    assert L.fdlbm_tile_plan(ctypes.byref(grid2), 8, 7, None, 0, ctypes.byref(count)) == -1
