"""Lid-driven cavity of Sec. 3C on the 257 x 257 tanh grid (Eq. 3.11, c = 1.5),
lid U = 0.1, Re = 1000 (nu = 1e-4), CFL 0.9, eta = 0.1, walls by Eq. 3.10:
(a) element-wise parity with the oracle over the first 1000 steps, through the
replayed CUDA graph; (b) the march to E(u) < 1e-8 in FP64 and the vortex
centres against the paper's table of vortex locations; (c) FP32-deviation
storage on the same march, its residual floor and its distance from FP64."""
import json
import math
import pathlib

import numpy as np
import pytest

import inputs as I
import oracle as O
from conftest import assert_parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1911_12913_gb300.analysis import march_to_steady, stream_function, vortex_centre  # noqa: E402
from paper_1911_12913_gb300.solver import FDLBM  # noqa: E402

N_CELLS, C, U, RE, CFL, ETA = 256, 1.5, 0.1, 1000.0, 0.9, 0.1
NU = U * 1.0 / RE
LID = [(0, 0), (0, 0), (0, 0), (U, 0.0)]
GOLD = json.loads((pathlib.Path(__file__).parent / "golden" / "paper_table5_cavity.json").read_text())
# the three vortices: search box (x0, x1, y0, y1) and sign of the psi extremum
BOXES = {"primary": ((0.3, 0.7, 0.3, 0.8), -1), "left_lower": ((0.0, 0.25, 0.0, 0.25), 1),
         "right_lower": ((0.7, 1.0, 0.0, 0.3), 1)}


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _solver(precision, graph_steps=100):
    ax = I.tanh_axis(N_CELLS, C)
    s = FDLBM(ax, ax, nu=NU, cfl=CFL, blend=ETA, precision=precision, wall_u=LID,
              graph_steps=graph_steps)
    one = np.ones((ax.n, ax.n))
    s.init_fields(one, 0 * one, 0 * one)
    return ax, s


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-7)])
def test_cavity_257_matches_oracle_through_graph_replay(precision, tol):
    from conftest import oracle_threads
    ax, s = _solver(precision)
    assert "graph_steps=100" in s.describe
    o = O.Oracle(ax, ax, nu=NU, dt=s.dt, beta=ETA, wall_u=LID, nthreads=oracle_threads())
    one = np.ones((ax.n, ax.n))
    o.init_fields(one, 0 * one, 0 * one)
    # 1 direct, then a realignment step, 3 graph replays and a direct remainder
    for n in (1, 537, 462):
        s.step(n)
        o.step(n)
    s.sync()
    assert_parity(s.get_state(), o.f, l2=tol, dev=1e-11 if precision == "fp64" else 5e-6,
                  label=f"cavity 257^2 {precision} after 1000 steps")


def _centres(ax, s):
    _, ux, _ = s.moments()
    psi = stream_function(ax.coords, ux)
    return {k: vortex_centre(ax.coords, ax.coords, psi, box, sign) for k, (box, sign) in BOXES.items()}


@pytest.mark.slow
def test_cavity_re1000_steady_state_fp64_and_fp32():
    ax, s64 = _solver("fp64")
    steps, res, _ = march_to_steady(s64, 1e-8, max_steps=900_000)
    assert res < 1e-8, (steps, res)
    c64 = _centres(ax, s64)
    print(f"FP64: E(u) {res:.2e} after {steps} steps (t = {steps * s64.dt:.1f})")
    for k, (x, y, p) in c64.items():
        px, py = GOLD["T2S2_FDLBM1"][k]
        gx, gy = GOLD["Ghia"][k]
        print(f"  {k}: ({x:.4f}, {y:.4f}) psi {p:+.3e}; paper ({px}, {py}), Ghia ({gx}, {gy})")
        # the paper's own 64^2 run and Ghia's 129^2 differ by up to 0.0045; a
        # 257^2 run lands within a cell of the paper's coarse grid of both
        tolc = 0.01 if k == "primary" else 0.015
        assert math.hypot(x - px, y - py) <= tolc and math.hypot(x - gx, y - gy) <= tolc, k
    _, u64x, u64y = s64.moments()

    # FP32-deviation storage on the same march: the residual stalls at its
    # round-off floor (~5e-8 per step).  The slowest mode decays by only
    # ~1.4e-5 per step, so a rounding bias d per step would shift the state by
    # about d / 1.4e-5 (a momentum bias of 3e-8 gave 3.3e-3); with the
    # equilibrium's first moment and the difference weights exact the FP32
    # state settles 2.8e-4 (relative L2 of u) from the FP64 one, the centre
    # unchanged
    ax, s32 = _solver("fp32")
    steps32, res32, _ = march_to_steady(s32, 1e-8, max_steps=steps)
    _, u32x, u32y = s32.moments()
    du = math.sqrt(rel(u32x, u64x) ** 2 + rel(u32y, u64y) ** 2)
    c32 = _centres(ax, s32)
    print(f"FP32: E(u) {res32:.2e} after {steps32} steps; rel L2 of u vs FP64 {du:.2e}; "
          f"primary ({c32['primary'][0]:.4f}, {c32['primary'][1]:.4f})")
    assert res32 < 2e-7
    assert du < 1e-3
    assert math.hypot(c32["primary"][0] - c64["primary"][0], c32["primary"][1] - c64["primary"][1]) < 1e-3
