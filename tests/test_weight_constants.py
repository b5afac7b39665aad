"""Exact sums of the weight constants of the CUDA path (host-side, no GPU).

On a periodic uniform grid the scheme conserves mass and momentum because the
weights of the difference of Eq. 2.36 sum to zero and the node maps keep the
moments of Eq. 3.3.  In floating point these identities survive only if they
hold for the rounded constants themselves; a residual of 1e-8 is a damping of
1e-8 per step.  A small host program built from the CUDA sources prints the
constants as hex floats, and the sums are taken here in rational arithmetic."""
import os
import shutil
import subprocess
from fractions import Fraction as Fr
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
CSRC = ROOT / "paper_1911_12913_gb300" / "csrc"


@pytest.fixture(scope="module")
def constants(tmp_path_factory):
    nvcc = shutil.which("nvcc") or (os.path.exists("/usr/local/cuda/bin/nvcc") and "/usr/local/cuda/bin/nvcc")
    if not nvcc:
        pytest.skip("nvcc not available")
    exe = tmp_path_factory.mktemp("wc") / "weight_constants"
    # the packed FP32x2 intrinsics of packed.cuh exist for sm_100-family
    # targets only; no device code runs
    subprocess.run([nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", str(CSRC), "-I", str(ROOT / "include"),
                    "-o", str(exe), str(ROOT / "tests" / "native" / "weight_constants.cu")],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe), "101"], check=True, capture_output=True, text=True).stdout
    return [line.split() for line in out.splitlines()]


def _x(h):
    return Fr(float.fromhex(h))


def test_stencil_weights_sum_to_zero_exactly(constants):
    rows = [r for r in constants if r[0] == "stencil"]
    assert len(rows) == 101
    for r in rows:
        beta = Fr(float(r[1]))
        exact = [(1 - beta) / 2, 3 * beta / 2, -(1 - beta) / 2 - 2 * beta, beta / 2]
        # half the grid spacing (2^-22 in FP32, 2^-51 in FP64), plus the FP64
        # rounding of the expressions in beta before they go on the grid
        for tag, vals, tol in (("f", r[3:7], Fr(1, 2 ** 23) + Fr(1, 2 ** 50)),
                               ("d", r[8:12], Fr(1, 2 ** 52) + Fr(4, 2 ** 53))):
            w = [_x(v) for v in vals]
            assert sum(w) == 0, (tag, r[1])
            assert max(abs(a - b) for a, b in zip(w, exact)) <= tol, (tag, r[1])


def test_linear_coefficients_carry_the_momentum_exactly(constants):
    (r,) = [r for r in constants if r[0] == "linear"]
    for c1, c2, ulp in ((r[2], r[3], Fr(1, 2 ** 24)), (r[5], r[6], Fr(1, 2 ** 53))):
        c1, c2 = _x(c1), _x(c2)
        assert 2 * c1 + 4 * c2 == 1
        assert abs(c1 - Fr(1, 3)) <= ulp and abs(c2 - Fr(1, 12)) <= 2 * ulp


def test_folded_relaxation_conserves_exactly(constants):
    rows = [r for r in constants if r[0] == "relax"]
    assert len(rows) == 100
    for r in rows:
        b, bw0, bw1, bw2, bc1, bc2, nbc1, nbc2, omb = (_x(v) for v in r[1:])
        bp = 1 - omb
        # (1 - b') + b' = 1 with b' within 3e-8 of b
        assert abs(bp - b) <= Fr(1, 2 ** 25)
        # the linear weights carry b' j exactly, so the first moment is j
        assert 2 * bc1 + 4 * bc2 == bp
        assert nbc1 == -bc1 and nbc2 == -bc2
        # the density weights sum to b' within FP32 rounding of each term
        assert abs(bw0 + 4 * bw1 + 4 * bw2 - bp) <= 6 * bp / 2 ** 24
