"""GPU parity of the incompressible equilibrium of He and Luo (cited in Sec. 2
as usable with both T2S2 schemes) against the CPU FP64 oracle: every kernel
that accepts it (scalar and warp-tile fused sweeps, the walls sweep, the staged
kernels, T2S2-FDLBM2, the batch modes), on states whose density varies so that
rho0 u and rho u differ.  Tolerances as in test_gpu_parity.py."""
import math

import numpy as np
import pytest

import inputs as I
import oracle as O
from conftest import assert_parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1911_12913_gb300.solver import FDLBM, FDLBMBatch  # noqa: E402

FP64_TOL = 1e-12
# FP32 bounds, about 10x the largest errors measured on GB300 over these tests
# (relative L2 of f~ up to 1.5e-8 after 12-25 steps from random states, 3e-8
# after 400 cavity steps; L-infinity of the error relative to the largest
# deviation f~ - w_i rho0 up to 1.9e-6).  The deviations are O(u) ~ 1e-2 and
# each step rounds them to 2^-24 relative, so a few steps leave errors of a
# few 1e-8 of the deviation at most nodes and the largest of about 1e-6.
# FP64: the L2 bound the benchmark spec fixes, and 1e-11 on the deviation
# (measured up to 4.7e-13).
FP32_L2 = 1e-7
FP32_DEV = 2e-5
FP64_DEV = 1e-11


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _pair(xa, ya, *, nu, cfl, beta, precision="fp64", force=None, wall_u=None, path="auto",
          rows=0, variant="auto", scheme=1):
    s = FDLBM(xa, ya, nu=nu, cfl=cfl, blend=beta, precision=precision,
              has_force=force is not None, wall_u=wall_u, path=path, rows_per_cta=rows,
              variant=variant, scheme=scheme, equilibrium="incompressible")
    assert s.describe.endswith("incompressible"), s.describe
    o = O.Oracle(xa, ya, nu=nu, dt=s.dt, beta=beta, force=force, wall_u=wall_u, scheme=scheme,
                 incomp=True)
    if force is not None:
        s.set_force(force)
    return s, o


def _init_both(s, o, fields):
    g = [fields["dudx"], fields["dudy"], fields["dvdx"], fields["dvdy"]]
    s.init_fields(fields["rho"], fields["ux"], fields["uy"], g)
    o.init_fields(fields["rho"], fields["ux"], fields["uy"], g)


@pytest.mark.parametrize("path,rows", [("fused", 0), ("fused", 3), ("staged", 0)])
@pytest.mark.parametrize("nx,ny", [(133, 37), (6, 9)])
def test_incomp_periodic_force_stretched_fp64(path, rows, nx, ny):
    """Random state with 5 % density variation, a force field and random
    metrics, ragged strips and segments: 25 steps, and the moments."""
    xa = I.periodic_axis(nx, 0.0, 1.0)
    ya = I.periodic_axis(ny, 0.0, 0.7)
    xa.metric = I.random_metric(nx, 31, base=nx, spread=0.4)
    ya.metric = I.random_metric(ny, 32, base=ny / 0.7, spread=0.4)
    force = 1e-3 * np.random.default_rng(7).uniform(-1, 1, size=(2, ny, nx))
    s, o = _pair(xa, ya, nu=0.02, cfl=0.4, beta=0.2, force=force, path=path, rows=rows)
    _init_both(s, o, I.random_fields(nx, ny, 17, drho=0.05))
    s.step(25)
    o.step(25)
    assert rel(s.get_state(), o.f) <= FP64_TOL
    r, ux, uy = s.moments()
    orr, oux, ouy = o.moments()
    assert rel(r, orr) <= FP64_TOL
    assert O.gre(ux, uy, oux, ouy) <= 1e-10


@pytest.mark.parametrize("variant", ["warp", "scalar"])
@pytest.mark.parametrize("nx,ny,rows", [(256, 21, 0), (68, 13, 2), (500, 37, 0)])
def test_incomp_fp32_fused(variant, nx, ny, rows):
    """FP32 deviations on the warp-tile and scalar fused kernels: 25 steps
    against the FP64 oracle."""
    xa = I.periodic_axis(nx, 0.0, 1.0)
    ya = I.periodic_axis(ny, 0.0, 0.7)
    xa.metric = I.random_metric(nx, 41, base=nx, spread=0.3)
    ya.metric = I.random_metric(ny, 42, base=ny / 0.7, spread=0.3)
    s, o = _pair(xa, ya, nu=0.02, cfl=0.4, beta=0.2, precision="fp32", rows=rows,
                 variant=variant)
    assert s.describe.split()[0] == {"warp": "fused-warp", "scalar": "fused"}[variant]
    _init_both(s, o, I.random_fields(nx, ny, 23, drho=0.05))
    s.step(25)
    o.step(25)
    s.sync()
    assert_parity(s.get_state(), o.f, l2=FP32_L2, dev=FP32_DEV, label=f"{s.describe} {nx}x{ny}")


@pytest.mark.parametrize("nx", [130, 128])
def test_incomp_fp32_with_force(nx):
    """The incompressible equilibrium with a body-force field on the scalar
    sweep (nx = 130) and the warp-tile kernel (nx = 128)."""
    ny = 20
    xa = I.periodic_axis(nx, 0.0, 1.0)
    ya = I.periodic_axis(ny, 0.0, 0.5)
    force = 1e-3 * np.random.default_rng(3).uniform(-1, 1, size=(2, ny, nx))
    s, o = _pair(xa, ya, nu=0.02, cfl=0.4, beta=0.2, precision="fp32", force=force)
    _init_both(s, o, I.random_fields(nx, ny, 29, drho=0.05))
    s.step(25)
    o.step(25)
    assert_parity(s.get_state(), o.f, l2=FP32_L2, dev=FP32_DEV, label=f"{s.describe} forced")


_WALLS = [("wall", "wall", 40, 33, 3), ("periodic", "wall", 96, 24, 0), ("wall", "periodic", 33, 40, 4)]


def _axis(kind, n, seed, length):
    if kind == "periodic":
        ax = I.periodic_axis(n, 0.0, length)
        ax.metric = I.random_metric(n, seed, base=n / length, spread=0.3)
        return ax
    return I.tanh_axis(n - 1, 1.5)


@pytest.mark.parametrize("precision,tol,path", [("fp64", FP64_TOL, "fused"),
                                                ("fp64", FP64_TOL, "staged"),
                                                ("fp32", FP32_L2, "fused")])
@pytest.mark.parametrize("bcx,bcy,nx,ny,rows", _WALLS)
def test_incomp_walls(precision, tol, path, bcx, bcy, nx, ny, rows):
    """Eq. 3.10 under the incompressible equilibrium (the fused walls sweep and
    the staged kernels), moving walls, a force field: 12 steps."""
    xa = _axis(bcx, nx, 81, 1.0)
    ya = _axis(bcy, ny, 82, 0.8)
    rng = np.random.default_rng(nx * 1000 + ny)
    force = 1e-3 * rng.uniform(-1, 1, size=(2, ny, nx))
    wall_u = [tuple(0.05 * rng.uniform(-1, 1, size=2)) for _ in range(4)]
    s, o = _pair(xa, ya, nu=0.02, cfl=0.4, beta=0.2, precision=precision, force=force,
                 wall_u=wall_u, rows=rows, path=path)
    _init_both(s, o, I.random_fields(nx, ny, 90 + nx, drho=0.05))
    for n in (1, 11):
        s.step(n)
        o.step(n)
    s.sync()
    assert_parity(s.get_state(), o.f, l2=tol, dev=FP64_DEV if precision == "fp64" else FP32_DEV,
                  label=f"{s.describe} {bcx}/{bcy} {nx}x{ny}")


@pytest.mark.parametrize("walls,precision,tol,nx", [(True, "fp64", FP64_TOL, 24), (False, "fp64", FP64_TOL, 24),
                                                    (True, "fp32", FP32_L2, 24), (False, "fp32", FP32_L2, 128)])
def test_incomp_scheme2(walls, precision, tol, nx):
    """T2S2-FDLBM2 with the incompressible equilibrium: the staged kernels on an
    FP64 channel, the fused sweeps on an FP32 channel and a periodic grid, and
    the warp-tile kernel on a periodic FP32 grid of 128 columns."""
    ny = 20
    xa = I.periodic_axis(nx, 0.0, 1.0)
    ya = I.tanh_axis(ny - 1, 1.5) if walls else I.periodic_axis(ny, 0.0, 0.8)
    force = 1e-3 * np.random.default_rng(4).uniform(-1, 1, size=(2, ny, nx))
    s, o = _pair(xa, ya, nu=0.02, cfl=0.3, beta=0.2, force=force, scheme=2, precision=precision,
                 wall_u=[(0, 0), (0, 0), (0, 0), (0.05, 0.0)] if walls else None)
    staged = walls and precision == "fp64"
    warp = not walls and precision == "fp32" and nx >= 64
    assert s.describe.startswith("staged-scheme2" if staged else
                                 "fused-warp-scheme2" if warp else "fused-scheme2"), s.describe
    _init_both(s, o, I.random_fields(nx, ny, 5, drho=0.05))
    s.step(15)
    o.step(15)
    assert_parity(s.get_state(), o.f, l2=tol, dev=FP64_DEV if precision == "fp64" else FP32_DEV,
                  label=f"{s.describe} scheme2")


@pytest.mark.parametrize("precision,tol,mode", [("fp64", FP64_TOL, "staged"), ("fp32", FP32_L2, "fused"),
                                                ("fp32", FP32_L2, "persistent")])
def test_incomp_batch(precision, tol, mode):
    """A batch of a cavity, a forced channel and a periodic case, all with the
    incompressible equilibrium, in three batch modes."""
    cav = I.tanh_axis(16, 1.5)
    lid = [(0, 0), (0, 0), (0, 0), (0.1, 0.0)]
    per = I.periodic_axis(33, 0.0, 1.0)
    per.metric = I.random_metric(33, 5, base=33)
    cases = [
        dict(xa=cav, ya=cav, nu=0.001, cfl=0.5, blend=0.1, wall_u=lid),
        dict(xa=I.periodic_axis(10, 0.0, 1.0), ya=I.tanh_axis(20, 1.5), nu=0.011, cfl=0.5,
             blend=0.1, has_force=True),
        dict(xa=per, ya=I.periodic_axis(29, 0.0, 0.8), nu=0.02, cfl=0.4, blend=0.2),
    ]
    for cs in cases:
        cs["equilibrium"] = "incompressible"
    batch = FDLBMBatch(cases, precision=precision, graph_steps=4, autotune=False, mode=mode)
    oracles = []
    for c, cs in enumerate(cases):
        view = batch.case(c)
        xa, ya = cs["xa"], cs["ya"]
        force = None
        if cs.get("has_force"):
            force = np.zeros((2, ya.n, xa.n))
            force[0] = 0.01
            view.set_force(force)
        o = O.Oracle(xa, ya, nu=cs["nu"], dt=view.dt, beta=cs["blend"], force=force,
                     wall_u=cs.get("wall_u"), incomp=True)
        fld = I.random_fields(xa.n, ya.n, 100 + c, drho=0.05)
        g = [fld["dudx"], fld["dudy"], fld["dvdx"], fld["dvdy"]]
        view.init_fields(fld["rho"], fld["ux"], fld["uy"], g)
        o.init_fields(fld["rho"], fld["ux"], fld["uy"], g)
        oracles.append(o)
    for n in (11, 1, 5):
        batch.step(n)
        for o in oracles:
            o.step(n)
    batch.sync()
    for c, o in enumerate(oracles):
        assert_parity(batch.case(c).get_state(), o.f, l2=tol,
                      dev=FP64_DEV if precision == "fp64" else FP32_DEV,
                      label=f"{batch.describe} case {c}")


def test_incomp_differs_from_standard():
    """The option changes the result: on a state with density variation the
    two equilibria give different states after a few steps (the parity above
    would otherwise be vacuous)."""
    nx, ny = 64, 16
    xa = I.periodic_axis(nx, 0.0, 1.0)
    ya = I.periodic_axis(ny, 0.0, 0.25)
    fld = I.random_fields(nx, ny, 8, drho=0.05)
    out = []
    for eq in ("standard", "incompressible"):
        s = FDLBM(xa, ya, nu=0.02, cfl=0.4, blend=0.2, equilibrium=eq)
        s.init_fields(fld["rho"], fld["ux"], fld["uy"], None)
        s.step(5)
        out.append(s.get_state())
    assert rel(out[1], out[0]) > 1e-6
