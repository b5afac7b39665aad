"""The allocation-free reduction (fdlbm_reduce_noalloc) against fdlbm_reduce.

fdlbm_reduce_noalloc serves callers that cannot allocate device memory: it
reads only buffers the caller passes and keeps its scratch in a fixed device
array.  Here the caller's buffers come from torch (the caller's side may
allocate).  Two calls in a row must each match the handle's own reduction,
which also shows that the shared scratch left by the first call does not leak
into the second.  This file is named to be collected last.
"""
import ctypes
import math

import numpy as np
import pytest

import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1911_12913_gb300 import binding as B  # noqa: E402
from paper_1911_12913_gb300.solver import FDLBM  # noqa: E402


def test_noalloc_reduce_matches_handle_reduce_twice():
    nx, ny = 150, 97
    xa = I.periodic_axis(nx, 0.0, 1.0)
    ya = I.periodic_axis(ny, 0.0, 0.8)
    xa.metric = I.random_metric(nx, 3, base=nx)
    ya.metric = I.random_metric(ny, 4, base=ny / 0.8)
    s = FDLBM(xa, ya, nu=0.02, cfl=0.4, blend=0.1)
    r = I.random_fields(nx, ny, 61)
    s.init_fields(r["rho"], r["ux"], r["uy"], [r["dudx"], r["dudy"], r["dvdx"], r["dvdy"]])
    L = B.load()
    dev = s.device
    mx = torch.tensor(xa.metric, dtype=torch.float64, device=dev)
    my = torch.tensor(ya.metric, dtype=torch.float64, device=dev)
    out = torch.full((3,), float("nan"), dtype=torch.float64, device=dev)
    stream = s.stream.cuda_stream

    s.reduce()                                   # handle snapshot of u(t0)
    for call in range(2):
        _, ux, uy = s.moments(device=True)       # u before the step
        uprev = torch.stack([ux, uy]).contiguous()
        s.step(1)
        mass, resid = s.reduce()
        f = s.get_state(device=True)
        rc = L.fdlbm_reduce_noalloc(f.data_ptr(), nx, ny, mx.data_ptr(), my.data_ptr(),
                                    uprev.data_ptr(), out.data_ptr(), stream)
        assert rc == 0, B.STATUS.get(rc, rc)
        s.stream.synchronize()
        got = out.cpu().numpy()
        assert got[0] == pytest.approx(mass, rel=1e-13), call
        assert got[1] == pytest.approx(resid, rel=1e-9), call
        _, ux1, uy1 = s.moments()
        assert got[2] == pytest.approx(float(np.sum(ux1 ** 2 + uy1 ** 2)), rel=1e-12), call

    # without a previous velocity the residual is reported as -1
    rc = L.fdlbm_reduce_noalloc(f.data_ptr(), nx, ny, mx.data_ptr(), my.data_ptr(), None,
                                out.data_ptr(), stream)
    assert rc == 0
    s.stream.synchronize()
    assert out[1].item() == -1.0 and out[0].item() == pytest.approx(mass, rel=1e-13)

    # sizes beyond the fixed scratch are rejected before any launch
    big = L.fdlbm_reduce_noalloc_max_rows() + 1
    assert L.fdlbm_reduce_noalloc(f.data_ptr(), 1, big, mx.data_ptr(), my.data_ptr(), None,
                                  out.data_ptr(), stream) == -6
