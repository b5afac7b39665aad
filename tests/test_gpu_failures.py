"""Failure detection without a GPU fault: faults are made on the host (a
non-finite value in the state, invalid arguments) and must come back as a
status, with the context still usable afterwards.  The bounded-wait timeout of
the persistent batch mode is covered in test_gpu_batch.py."""
import math

import numpy as np
import pytest

import inputs as I
import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1911_12913_gb300 import binding as B  # noqa: E402
from paper_1911_12913_gb300.solver import FDLBM, FDLBMBatch  # noqa: E402


@pytest.mark.parametrize("precision,variant", [("fp32", "warp"), ("fp32", "scalar"), ("fp64", "auto")])
def test_nonfinite_state_is_reported(precision, variant):
    """A NaN planted in the state on the host spreads through the steps, and
    fdlbm_reduce returns ENONFINITE; a clean state loaded afterwards steps and
    reduces normally (the context is unharmed)."""
    n = 64
    xa = I.periodic_axis(n, 0.0, 2 * math.pi)
    s = FDLBM(xa, xa, nu=0.01, cfl=0.5, blend=0.1, precision=precision, variant=variant)
    f = I.taylor_green(xa, xa, u0=0.01)
    s.init_fields(f["rho"], f["ux"], f["uy"], None)
    clean = s.get_state()
    bad = clean.copy()
    bad[5, 17, 40] = np.nan
    s.set_state(bad)
    s.step(4)
    with pytest.raises(B.FdlbmError, match="ENONFINITE"):
        s.reduce()
    s.set_state(clean)
    s.step(4)
    mass, _ = s.reduce()
    assert math.isfinite(mass)


def test_nonfinite_case_in_batch_is_reported():
    """The same inside a batch: the poisoned case reports ENONFINITE through
    its own reduce, the other cases stay finite."""
    cav = I.tanh_axis(16, 1.5)
    lid = [(0, 0), (0, 0), (0, 0), (0.1, 0.0)]
    cases = [dict(xa=cav, ya=cav, nu=0.001, cfl=0.5, blend=0.1, wall_u=lid),
             dict(xa=I.periodic_axis(32, 0.0, 1.0), ya=I.periodic_axis(24, 0.0, 1.0), nu=0.02,
                  cfl=0.4, blend=0.2)]
    batch = FDLBMBatch(cases, precision="fp32", graph_steps=0, autotune=False)
    for c, cs in enumerate(cases):
        one = np.ones((cs["ya"].n, cs["xa"].n))
        batch.case(c).init_fields(one, 0 * one, 0 * one)
    st = batch.case(1).get_state()
    st[0, 3, 3] = np.inf
    batch.case(1).set_state(st)
    batch.step(3)
    batch.sync()
    assert math.isfinite(batch.case(0).reduce()[0])
    with pytest.raises(B.FdlbmError, match="ENONFINITE"):
        batch.case(1).reduce()


def test_invalid_arguments_are_rejected():
    """Host-side argument faults: non-positive metrics, a negative viscosity
    and an unknown equilibrium are refused at create with EINVAL, and a step
    with a negative count with EINVAL, before any device work."""
    xa = I.periodic_axis(16, 0.0, 1.0)
    bad = I.periodic_axis(16, 0.0, 1.0)
    bad.metric = -np.ones(16)
    with pytest.raises(B.FdlbmError, match="EINVAL"):
        FDLBM(bad, xa, nu=0.01, cfl=0.5, blend=0.1)
    with pytest.raises(B.FdlbmError, match="EINVAL"):
        FDLBM(xa, xa, nu=-0.01, cfl=0.5, blend=0.1)
    s = FDLBM(xa, xa, nu=0.01, cfl=0.5, blend=0.1)
    L = B.load()
    assert L.fdlbm_step(s._h, -1) == -1
    s.step(2)
    s.sync()
