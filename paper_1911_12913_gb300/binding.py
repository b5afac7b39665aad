"""Thin ctypes binding of the C ABI in include/fdlbm.h.

Argument marshalling only: every step of the method runs in the CUDA kernels
of libfdlbm.so.  PyTorch supplies device memory (the handle's workspace and
any device-side field) and the CUDA stream.  There is no CPU fallback: if the
compiled library is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

import numpy as np

_LIB_PATH = Path(__file__).resolve().parent / "_lib" / "libfdlbm.so"

PERIODIC, WALL = 0, 1
FP64, FP32_DEV = 0, 1
PATH_AUTO, PATH_FUSED, PATH_STAGED = 0, 1, 2
MEM_HOST, MEM_DEVICE = 0, 1
SCHEME_T2S2_1, SCHEME_T2S2_2 = 0, 1
EQ_STANDARD, EQ_INCOMPRESSIBLE = 0, 1
BATCH_FUSED, BATCH_STAGED, BATCH_PERSISTENT = 0, 1, 2
VARIANT_AUTO, VARIANT_SCALAR, VARIANT_WARP = 0, 1, 5
STATUS = {0: "ok", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ENONFINITE", -5: "EUNSUPPORTED",
          -6: "ETOOBIG"}

_dp = ctypes.POINTER(ctypes.c_double)


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("x", _dp), ("y", _dp), ("lx", ctypes.c_double), ("ly", ctypes.c_double),
                ("bc_x", ctypes.c_int), ("bc_y", ctypes.c_int),
                ("wall_u", (ctypes.c_double * 2) * 4)]


class Metrics(ctypes.Structure):
    _fields_ = [("dzeta_dx", _dp), ("dmu_dy", _dp)]


class Opts(ctypes.Structure):
    _fields_ = [("A", ctypes.c_double), ("rho0", ctypes.c_double),
                ("precision", ctypes.c_int), ("has_force", ctypes.c_int),
                ("path", ctypes.c_int), ("rows_per_cta", ctypes.c_int), ("variant", ctypes.c_int),
                ("scheme", ctypes.c_int), ("adjoint", ctypes.c_int),
                ("graph_steps", ctypes.c_int), ("equilibrium", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("workspace", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_size_t)]


# (name, restype, argtypes) of every entry point declared in include/fdlbm.h
_H = ctypes.c_void_p
SIGNATURES = [
    ("fdlbm_default_opts", None, [ctypes.POINTER(Opts)]),
    ("fdlbm_time_step", ctypes.c_double, [ctypes.POINTER(Grid), ctypes.c_double]),
    ("fdlbm_workspace_bytes", ctypes.c_size_t, [ctypes.POINTER(Grid), ctypes.POINTER(Opts)]),
    ("fdlbm_create", ctypes.c_int, [ctypes.POINTER(Grid), ctypes.POINTER(Metrics), ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double, ctypes.POINTER(Opts),
                                    ctypes.POINTER(_H)]),
    ("fdlbm_destroy", None, [_H]),
    ("fdlbm_init_fields", ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_int]),
    ("fdlbm_init_fields_f32", ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_int]),
    ("fdlbm_set_state", ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_int]),
    ("fdlbm_get_state", ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_int]),
    ("fdlbm_set_force", ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_int]),
    ("fdlbm_step", ctypes.c_int, [_H, ctypes.c_int]),
    ("fdlbm_moments", ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_int]),
    ("fdlbm_moments_f32", ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_int]),
    ("fdlbm_reduce", ctypes.c_int, [_H, _dp, _dp]),
    ("fdlbm_set_stream", ctypes.c_int, [_H, ctypes.c_void_p]),
    ("fdlbm_sync", ctypes.c_int, [_H]),
    ("fdlbm_dt", ctypes.c_double, [_H]),
    ("fdlbm_tau", ctypes.c_double, [_H]),
    ("fdlbm_steps_done", ctypes.c_longlong, [_H]),
    ("fdlbm_path", ctypes.c_int, [_H]),
    ("fdlbm_kernels_per_step", ctypes.c_int, [_H]),
    ("fdlbm_tile_plan", ctypes.c_int, [ctypes.POINTER(Grid), ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    ("fdlbm_last_error", ctypes.c_char_p, [_H]),
    ("fdlbm_describe", ctypes.c_char_p, [_H]),
    ("fdlbm_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("fdlbm_state_bytes", ctypes.c_size_t, [_H]),
    ("fdlbm_copy_state", ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_int]),
    ("fdlbm_state_layout", ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    ("fdlbm_adjoint_step", ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p]),
    ("fdlbm_moments_vjp", ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p]),
    ("fdlbm_batch_workspace_bytes", ctypes.c_size_t, [ctypes.c_int, ctypes.POINTER(Grid),
                                                      ctypes.POINTER(Opts)]),
    ("fdlbm_batch_create", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(Grid), ctypes.POINTER(Metrics),
                                          _dp, _dp, _dp, ctypes.POINTER(Opts), ctypes.c_int,
                                          ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t,
                                          ctypes.POINTER(_H)]),
    ("fdlbm_batch_case", _H, [_H, ctypes.c_int]),
    ("fdlbm_batch_size", ctypes.c_int, [_H]),
    ("fdlbm_batch_cells", ctypes.c_longlong, [_H]),
    ("fdlbm_batch_step", ctypes.c_int, [_H, ctypes.c_int]),
    ("fdlbm_batch_set_mode", ctypes.c_int, [_H, ctypes.c_int]),
    ("fdlbm_batch_mode", ctypes.c_int, [_H]),
    ("fdlbm_batch_sync", ctypes.c_int, [_H]),
    ("fdlbm_init_vjp", ctypes.c_int, [_H] + [ctypes.c_void_p] * 8),
    ("fdlbm_batch_set_spin_limit", ctypes.c_int, [_H, ctypes.c_uint]),
    ("fdlbm_batch_stream", ctypes.c_void_p, [_H]),
    ("fdlbm_batch_describe", ctypes.c_char_p, [_H]),
    ("fdlbm_batch_last_error", ctypes.c_char_p, [_H]),
    ("fdlbm_batch_destroy", None, [_H]),
    ("fdlbm_reduce_noalloc", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p]),
    ("fdlbm_reduce_noalloc_max_rows", ctypes.c_int, []),
    ("fdlbm_probe_fp64_fma", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p]),
]

_lib = None


def lib_path() -> Path:
    return _LIB_PATH


def load():
    """Load libfdlbm.so (built by ``paper_1911_12913_gb300.build``); raise if absent."""
    global _lib
    if _lib is None:
        if not _LIB_PATH.exists():
            raise ImportError(f"{_LIB_PATH} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(str(_LIB_PATH))
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class FdlbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def make_grid(xa, ya, wall_u=None) -> tuple:
    """A ``Grid`` struct from two axes (``inputs.Axis``-like: coords, periodic,
    length); returns the struct and the arrays it points into (keep alive)."""
    x = np.ascontiguousarray(xa.coords, dtype=np.float64)
    y = np.ascontiguousarray(ya.coords, dtype=np.float64)
    g = Grid()
    g.nx, g.ny = x.size, y.size
    g.x, g.y = _dptr(x), _dptr(y)
    g.lx = float(xa.length) if xa.periodic else 0.0
    g.ly = float(ya.length) if ya.periodic else 0.0
    g.bc_x = PERIODIC if xa.periodic else WALL
    g.bc_y = PERIODIC if ya.periodic else WALL
    wu = wall_u if wall_u is not None else [(0.0, 0.0)] * 4
    for s in range(4):
        g.wall_u[s][0], g.wall_u[s][1] = float(wu[s][0]), float(wu[s][1])
    return g, (x, y)
