"""C ABI checks that need no GPU: the library loads, exports every entry point
that include/fdlbm.h declares, and its host-only logic (Eq. 3.1 time step,
workspace sizing, argument validation) behaves as documented."""
import ctypes
import json
import math
import re
from pathlib import Path

import numpy as np
import pytest

import inputs as I
import oracle as O

ROOT = Path(__file__).resolve().parents[1]
GOLDEN = Path(__file__).resolve().parent / "golden"


@pytest.fixture(scope="module")
def B():
    from paper_1911_12913_gb300 import binding
    from paper_1911_12913_gb300 import build as b
    b.build()
    binding.load()
    return binding


def _declared_functions():
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        text = re.sub(r"/\*.*?\*/", "", h.read_text(), flags=re.S)
        names |= set(re.findall(r"\b(fdlbm_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(B):
    names = _declared_functions()
    assert len(names) >= 20
    lib = ctypes.CDLL(str(B.lib_path()))
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    bound = {n for n, _, _ in B.SIGNATURES}
    assert set(names) == bound, set(names) ^ bound


def test_struct_layouts_match_header(B, tmp_path):
    """The ctypes mirrors have the size and field offsets the C compiler gives
    the structs of include/fdlbm.h (a C program compiled against the header)."""
    import subprocess
    fields = {"fdlbm_grid": B.Grid, "fdlbm_metrics": B.Metrics, "fdlbm_opts": B.Opts}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "fdlbm.h"', "int main(void){"]
    for cname, py in fields.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", f"-I{ROOT / 'include'}", str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in fields.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
    o = B.Opts()
    B.load().fdlbm_default_opts(ctypes.byref(o))
    assert (o.A, o.rho0, o.precision, o.path, o.variant, o.workspace) == \
        (0.5, 1.0, B.FP64, B.PATH_AUTO, B.VARIANT_AUTO, None)


def test_time_step_matches_paper_tables(B):
    """Host-only Eq. 3.1 of the library reproduces the iteration counts of Tables 4 and 8."""
    L = B.load()
    g = json.loads((GOLDEN / "paper_time_steps.json").read_text())
    tg = g["taylor"]
    xa = I.periodic_axis(tg["grid"][0], *tg["domain"])
    ya = I.periodic_axis(tg["grid"][1], *tg["domain"])
    grid, keep = B.make_grid(xa, ya)
    tc = math.log(2) / (tg["nu"] * (tg["k"][0] ** 2 + tg["k"][1] ** 2))
    for run in tg["runs"]:
        dt = L.fdlbm_time_step(ctypes.byref(grid), run["cfl"])
        assert int(2 * tc / dt) == run["steps"]
        assert dt == pytest.approx(O.time_step(run["cfl"], xa, ya), rel=1e-15)
    p = g["poiseuille"]
    xa = I.periodic_axis(p["grid"][0], 0.0, 1.0)
    ya = I.tanh_axis(p["grid"][1], p["c"])
    grid, keep = B.make_grid(xa, ya)
    for run in p["runs"]:
        dt = L.fdlbm_time_step(ctypes.byref(grid), run["cfl"])
        assert int(p["t_end"] / dt) == run["steps"]


def test_workspace_and_validation_without_gpu(B):
    L = B.load()
    xa = I.periodic_axis(64, 0.0, 1.0)
    grid, keep = B.make_grid(xa, xa)
    o = B.Opts()
    L.fdlbm_default_opts(ctypes.byref(o))
    n64 = L.fdlbm_workspace_bytes(ctypes.byref(grid), ctypes.byref(o))
    o.precision = B.FP32_DEV
    n32 = L.fdlbm_workspace_bytes(ctypes.byref(grid), ctypes.byref(o))
    assert n64 > n32 >= 2 * 9 * 64 * 64 * 4
    o.path = B.PATH_STAGED
    assert L.fdlbm_workspace_bytes(ctypes.byref(grid), ctypes.byref(o)) > n32
    # walled grids take the fused path (Eq. 3.10 inside the sweep), for both
    # schemes; the warp-tile kernel is FP32 only
    wa = I.wall_axis(20, 0.0, 1.0)
    wgrid, keep2 = B.make_grid(xa, wa)
    o.path = B.PATH_FUSED
    assert L.fdlbm_workspace_bytes(ctypes.byref(wgrid), ctypes.byref(o)) > 0
    o.scheme = B.SCHEME_T2S2_2
    assert L.fdlbm_workspace_bytes(ctypes.byref(wgrid), ctypes.byref(o)) > 0
    h = ctypes.c_void_p()
    o.variant = B.VARIANT_WARP
    o.precision = B.FP64
    assert L.fdlbm_create(ctypes.byref(wgrid), None, 0.01, 0.5, 0.1, ctypes.byref(o),
                          ctypes.byref(h)) == -5
    o.precision = B.FP32_DEV
    o.variant = B.VARIANT_AUTO
    # invalid arguments are rejected before any device work
    L.fdlbm_default_opts(ctypes.byref(o))
    for nu, cfl, blend in ((0.0, 0.5, 0.1), (0.01, -1.0, 0.1), (0.01, 0.5, 1.5)):
        assert L.fdlbm_create(ctypes.byref(grid), None, nu, cfl, blend, ctypes.byref(o),
                              ctypes.byref(h)) == -1
    bad = np.array([0.0, 0.2, 0.1, 0.3])
    bgrid, keep3 = B.make_grid(I.Axis(bad, np.ones(4), False, 0.0), xa)
    assert L.fdlbm_time_step(ctypes.byref(bgrid), 0.5) < 0
    assert L.fdlbm_create(ctypes.byref(bgrid), None, 0.01, 0.5, 0.1, None, ctypes.byref(h)) == -1
    mneg = B.Metrics()
    neg = -np.ones(64)
    mneg.dzeta_dx = B._dptr(neg)
    assert L.fdlbm_create(ctypes.byref(grid), ctypes.byref(mneg), 0.01, 0.5, 0.1, None,
                          ctypes.byref(h)) == -1
    # the equilibrium option: unknown values are invalid; the incompressible
    # equilibrium has no adjoint step
    L.fdlbm_default_opts(ctypes.byref(o))
    o.equilibrium = 2
    assert L.fdlbm_create(ctypes.byref(grid), None, 0.01, 0.5, 0.1, ctypes.byref(o),
                          ctypes.byref(h)) == -1
    L.fdlbm_default_opts(ctypes.byref(o))
    o.equilibrium = B.EQ_INCOMPRESSIBLE
    o.precision = B.FP32_DEV
    o.adjoint = 1
    assert L.fdlbm_create(ctypes.byref(grid), None, 0.01, 0.5, 0.1, ctypes.byref(o),
                          ctypes.byref(h)) == -5
    # variant values that name no kernel are invalid
    for value in (2, 3, 4, 6, -1):
        L.fdlbm_default_opts(ctypes.byref(o))
        o.variant = value
        assert L.fdlbm_create(ctypes.byref(grid), None, 0.01, 0.5, 0.1, ctypes.byref(o),
                              ctypes.byref(h)) == -1, value
    assert L.fdlbm_status_string(-4) == b"non-finite result"
    assert L.fdlbm_last_error(None) == b"NULL handle"
    L.fdlbm_destroy(None)
