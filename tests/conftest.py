import os
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU oracle runs")


def oracle_threads() -> int:
    return max(1, min(8, os.cpu_count() or 1))


# Lattice weights of D2Q9 (Sec. 3), used only to form the deviation f~ - w_i rho0
# of a state in the parity checks below.
_W = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4


def parity_errors(got, want, rho0: float = 1.0):
    """Errors of a state ``got`` ([9, ny, nx] f~) against the oracle's ``want``:
    the relative L2 norm over f~, and the L-infinity norm of the difference
    relative to the largest deviation |f~_i - w_i rho0| of the oracle's state.
    The first is dominated by the O(1) rest populations w_i rho0; the second
    sees a defect confined to a few nodes or one population at the size of the
    O(u) signal that the FP32 storage keeps."""
    import numpy as np
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    w = np.asarray(_W).reshape(9, *([1] * (want.ndim - 1)))
    l2 = float(np.linalg.norm(got - want) / np.linalg.norm(want))
    dev = float(np.abs(got - want).max() / np.abs(want - w * rho0).max())
    return l2, dev


def assert_parity(got, want, *, l2: float, dev: float, label: str = "", rho0: float = 1.0):
    e_l2, e_dev = parity_errors(got, want, rho0)
    print(f"{label}: rel L2(f~) = {e_l2:.3e}, rel Linf(deviation) = {e_dev:.3e}")
    assert e_l2 <= l2, (label, e_l2, l2)
    assert e_dev <= dev, (label, e_dev, dev)
