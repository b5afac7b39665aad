"""Python handle on the CPU FP64 oracle of the T2S2-FDLBM step.

TEST INFRASTRUCTURE ONLY: the CUDA library never imports, links or calls this
package.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
legs of ``bench.py`` use it.  The arithmetic lives in ``fdlbm_oracle.c``
(plain C, FP64, whole-field passes in the order of Sec. 2D of the paper); this
module compiles it with gcc, marshals numpy arrays and adds the host-side
conventions of Sec. 3:

* time step from the CFL number, Eq. 3.1, with xi = 1 (the lattice speed) and
  the smallest node spacing over both axes;
* relaxation time tau = nu / cs^2 (the paper does not print the relation; this is
  the continuous BGK relation, the f~ change of variables already makes the
  collision second order);
* the global relative error of Eq. 3.6 and the successive-step residual of the
  cavity section.

Parity status of each function is listed in the repository's design notes;
every function here is pinned by a ``-m "not gpu"`` test except where a
docstring says "parity unpinned".
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "fdlbm_oracle.c"
_LIB = _HERE / "_build" / "liboracle.so"
_LIB_C = _HERE / "_build" / "liboracle_complex.so"
CS2 = 1.0 / 3.0

_dp = ctypes.POINTER(ctypes.c_double)


class _Cfg(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("periodic_x", ctypes.c_int), ("periodic_y", ctypes.c_int),
        ("mx", _dp), ("my", _dp),
        ("tau", ctypes.c_double), ("dt", ctypes.c_double),
        ("A", ctypes.c_double), ("beta", ctypes.c_double),
        ("beta_is_central", ctypes.c_int), ("scheme", ctypes.c_int),
        ("force", ctypes.c_void_p),
        ("wall_u", (ctypes.c_double * 2) * 4),
        ("nthreads", ctypes.c_int),
        ("incomp", ctypes.c_int),
        ("rho0", ctypes.c_double),
    ]


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (FP64, no fast-math, no FMA contraction), once
    with real values and once with complex values (complex-step derivatives)."""
    _LIB.parent.mkdir(exist_ok=True)
    for lib_path, extra in ((_LIB, []), (_LIB_C, ["-DORACLE_COMPLEX"])):
        if force or not lib_path.exists() or lib_path.stat().st_mtime < _SRC.stat().st_mtime:
            tmp = lib_path.with_suffix(f".{os.getpid()}.tmp")
            cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                   "-std=c11", *extra, str(_SRC), "-o", str(tmp), "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, lib_path)
    return _LIB


_lib = None
_lib_c = None


def lib_complex():
    """The complex-valued build (pointer arguments only)."""
    global _lib_c
    if _lib_c is None:
        build()
        L = ctypes.CDLL(str(_LIB_C))
        P = ctypes.POINTER(_Cfg)
        vp = ctypes.c_void_p
        L.oracle_step.argtypes = [P, vp, ctypes.c_int]
        L.oracle_step.restype = ctypes.c_int
        L.oracle_moments.argtypes = [P, vp, vp, vp, vp]
        _lib_c = L
    return _lib_c


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(str(_LIB))
        P = ctypes.POINTER(_Cfg)
        L.oracle_step.argtypes = [P, _dp, ctypes.c_int]
        L.oracle_step.restype = ctypes.c_int
        L.oracle_step_t1s2.argtypes = [P, _dp, ctypes.c_int]
        L.oracle_step_t1s2.restype = ctypes.c_int
        L.oracle_moments.argtypes = [P, _dp, _dp, _dp, _dp]
        L.oracle_init.argtypes = [P, _dp, _dp, _dp, _dp, ctypes.c_double, _dp]
        L.oracle_feq.argtypes = [ctypes.c_double] * 3 + [_dp]
        L.oracle_feq_incomp.argtypes = [ctypes.c_double] * 4 + [_dp]
        L.oracle_force_term.argtypes = [_dp] + [ctypes.c_double] * 4 + [_dp]
        L.oracle_derivative.argtypes = [P, _dp, ctypes.c_int, ctypes.c_int, _dp]
        L.oracle_stages.argtypes = [P, _dp] + [_dp] * 5
        L.oracle_stages.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


# ---------------------------------------------------------------- host conventions
def time_step(cfl: float, *axes) -> float:
    """Eq. 3.1: dt = CFL * dx_min / xi with xi = 1 and dx_min over all axes."""
    best = math.inf
    for ax in axes:
        d = np.diff(ax.coords)
        if ax.periodic:
            d = np.append(d, ax.coords[0] + ax.length - ax.coords[-1])
        best = min(best, float(d.min()))
    return cfl * best / 1.0


def tau_from_nu(nu: float) -> float:
    """tau = nu / cs^2 (reading of the paper's unstated relation)."""
    return nu / CS2


def gre(u, v, ua, va) -> float:
    """Eq. 3.6 on the velocity vector: ||u - u'|| / ||u'|| over all nodes."""
    num = np.sum((u - ua) ** 2 + (v - va) ** 2)
    den = np.sum(ua ** 2 + va ** 2)
    return float(math.sqrt(num / den))


def gre_component(u, ua) -> float:
    """Eq. 3.6 on one velocity component (Tables 1-2 report E(u) and E(v))."""
    return float(math.sqrt(np.sum((u - ua) ** 2) / np.sum(ua ** 2)))


def feq(rho: float, ux: float, uy: float) -> np.ndarray:
    """Eq. 3.2 at one node."""
    out = np.zeros(9)
    lib().oracle_feq(rho, ux, uy, _ptr(out))
    return out


def feq_incomp(rho: float, rho0: float, ux: float, uy: float) -> np.ndarray:
    """The incompressible equilibrium of He and Luo at one node (the paper cites
    it in Sec. 2 as usable with both schemes but does not print it):
    Eq. 3.2 with rho0 in place of rho in the velocity terms."""
    out = np.zeros(9)
    lib().oracle_feq_incomp(rho, rho0, ux, uy, _ptr(out))
    return out


def force_term(fe: np.ndarray, ux: float, uy: float, Fx: float, Fy: float) -> np.ndarray:
    """Eq. 3.12 at one node."""
    fe = np.ascontiguousarray(fe, dtype=np.float64)
    out = np.zeros(9)
    lib().oracle_force_term(_ptr(fe), ux, uy, Fx, Fy, _ptr(out))
    return out


class Oracle:
    """One grid + parameter set, holding f~ as float64 ``[9, ny, nx]``.

    ``A``: the intermediate time fraction (0.5: T2S2-FDLBM1, 0: T1S2-FDLBM).
    ``beta``: upwind weight of the mixed difference.  ``scheme=2`` selects
    T2S2-FDLBM2 (Eq. 5.23; pinned by the grid-convergence table of Sec. 3A,
    its time order and invariants; parity with the paper's large-CFL FDLBM2
    errors unpinned).  Walled axes use Eq. 3.10
    (parity with the paper's Poiseuille error magnitudes unpinned).  ``incomp=True`` selects the incompressible
    equilibrium of He and Luo with reference density ``rho0`` (velocity from
    rho0 u = sum xi f, forcing term at rho0).
    """

    def __init__(self, xa, ya, *, nu: float, dt: float, beta: float, A: float = 0.5,
                 scheme: int = 1, force=None, wall_u=None, beta_is_central: bool = False,
                 nthreads: int = 1, tau: float | None = None, incomp: bool = False,
                 rho0: float = 1.0):
        self.xa, self.ya = xa, ya
        self.nx, self.ny = xa.n, ya.n
        self.mx = np.ascontiguousarray(xa.metric, dtype=np.float64)
        self.my = np.ascontiguousarray(ya.metric, dtype=np.float64)
        self.tau = tau_from_nu(nu) if tau is None else tau
        self.dt = dt
        self.force = None if force is None else np.ascontiguousarray(force, dtype=np.float64)
        if self.force is not None:
            assert self.force.shape == (2, self.ny, self.nx)
        c = _Cfg()
        c.nx, c.ny = self.nx, self.ny
        c.periodic_x, c.periodic_y = int(xa.periodic), int(ya.periodic)
        c.mx, c.my = _ptr(self.mx), _ptr(self.my)
        c.tau, c.dt, c.A, c.beta = self.tau, dt, A, beta
        c.beta_is_central = int(beta_is_central)
        c.scheme = scheme
        c.force = self.force.ctypes.data if self.force is not None else None
        wu = wall_u if wall_u is not None else [(0.0, 0.0)] * 4
        for s in range(4):
            c.wall_u[s][0], c.wall_u[s][1] = float(wu[s][0]), float(wu[s][1])
        c.nthreads = nthreads
        c.incomp = int(incomp)
        c.rho0 = rho0
        self.rho0 = rho0
        self._cfg = c
        self.f = np.zeros((9, self.ny, self.nx))

    @property
    def cfg(self):
        return ctypes.byref(self._cfg)

    def set_threads(self, n: int):
        self._cfg.nthreads = n

    def init_fields(self, rho, ux, uy, grad=None, rho0: float | None = None):
        """Eq. 3.2 (or the incompressible equilibrium), plus the gradient term
        of Eq. 3.5 when the velocity gradient is given."""
        rho0 = self.rho0 if rho0 is None else rho0
        a = [np.ascontiguousarray(v, dtype=np.float64) for v in (rho, ux, uy)]
        g = None
        if grad is not None:
            g = np.ascontiguousarray(np.stack(grad), dtype=np.float64)
        lib().oracle_init(self.cfg, *(_ptr(v) for v in a),
                          _ptr(g) if g is not None else ctypes.cast(None, _dp), rho0,
                          _ptr(self.f))
        return self

    def step(self, n: int = 1):
        rc = lib().oracle_step(self.cfg, _ptr(self.f), n)
        if rc != 0:
            raise MemoryError("oracle_step failed")
        return self

    def step_t1s2(self, n: int = 1):
        rc = lib().oracle_step_t1s2(self.cfg, _ptr(self.f), n)
        if rc != 0:
            raise MemoryError("oracle_step_t1s2 failed")
        return self

    def moments(self):
        r = np.zeros((self.ny, self.nx)); ux = np.zeros_like(r); uy = np.zeros_like(r)
        lib().oracle_moments(self.cfg, _ptr(self.f), _ptr(r), _ptr(ux), _ptr(uy))
        return r, ux, uy

    def derivative(self, fld, axis: int, sign: int):
        fld = np.ascontiguousarray(fld, dtype=np.float64)
        out = np.zeros_like(fld)
        lib().oracle_derivative(self.cfg, _ptr(fld), axis, sign, _ptr(out))
        return out

    def stages(self):
        outs = [np.zeros_like(self.f) for _ in range(5)]
        rc = lib().oracle_stages(self.cfg, _ptr(self.f), *(_ptr(o) for o in outs))
        if rc != 0:
            raise MemoryError("oracle_stages failed")
        return dict(zip(["fbar_plus", "fbar_star", "fstar", "ftil_plus", "L"], outs))

    def mass(self):
        """Jacobian-weighted mass sum_{x,y} rho / (m_x m_y) (exact invariant on periodic grids)."""
        r, _, _ = self.moments()
        return float(np.sum(r / np.outer(self.my, self.mx)))


# ------------------------------------------------------------------ complex step
def step_complex(xa, ya, *, nu: float, dt: float, beta: float, f, force=None, A: float = 0.5,
                 nsteps: int = 1, wall_u=None, scheme: int = 1):
    """Advance a complex-valued state (and complex force field, if given) with
    the complex build of the oracle: the same arithmetic as ``Oracle.step``."""
    o = Oracle(xa, ya, nu=nu, dt=dt, beta=beta, A=A, wall_u=wall_u, scheme=scheme)
    fc = np.ascontiguousarray(f, dtype=np.complex128).copy()
    keep = None
    if force is not None:
        keep = np.ascontiguousarray(force, dtype=np.complex128)
        o._cfg.force = keep.ctypes.data
    rc = lib_complex().oracle_step(o.cfg, fc.ctypes.data, nsteps)
    if rc != 0:
        raise MemoryError("oracle_step (complex) failed")
    del keep
    return fc


def step_vjp(xa, ya, *, nu: float, dt: float, beta: float, f0, lam, force=None, A: float = 0.5,
             eps: float = 1e-20):
    """Reference reverse mode of one step on a tiny periodic grid, by brute
    force: every column of the step's Jacobian (with respect to the state and to
    the force field) comes from one complex-step evaluation,
    J e_k = Im(step(x + i eps e_k)) / eps, exact to rounding.  Returns
    (J_f^T lam, J_F^T lam), shaped like f0 and like the force field."""
    f0 = np.asarray(f0, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    F = np.zeros((2,) + f0.shape[1:]) if force is None else np.asarray(force, dtype=np.float64)
    kw = dict(nu=nu, dt=dt, beta=beta, A=A)
    out_f = np.zeros(f0.size)
    for k in range(f0.size):
        x = f0.astype(np.complex128).ravel()
        x[k] += 1j * eps
        y = step_complex(xa, ya, f=x.reshape(f0.shape), force=F, **kw)
        out_f[k] = float(np.sum(y.imag / eps * lam))
    out_F = np.zeros(F.size)
    for k in range(F.size):
        Fc = F.astype(np.complex128).ravel()
        Fc[k] += 1j * eps
        y = step_complex(xa, ya, f=f0, force=Fc.reshape(F.shape), **kw)
        out_F[k] = float(np.sum(y.imag / eps * lam))
    return out_f.reshape(f0.shape), out_F.reshape(F.shape)
