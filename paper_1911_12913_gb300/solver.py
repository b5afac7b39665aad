"""Python handle on one libfdlbm solver (the same calls as the C ABI).

Device memory for the handle's workspace comes from PyTorch; the handle uses
torch's current CUDA stream unless another stream is given.  Fields can be
passed as numpy arrays (host, copied through the library's staging area) or as
CUDA torch tensors (read in place on the stream).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import binding as B


def _check(L, h, rc, what):
    if rc != 0:
        msg = L.fdlbm_last_error(h).decode() if h else ""
        raise B.FdlbmError(rc, f"{what}: {msg}")


class FDLBM:
    """One grid, one parameter set, one distribution state on the GPU.

    ``xa, ya``: axes with ``coords``, ``metric`` (d zeta/dx), ``periodic`` and
    ``length`` (see ``inputs.Axis``).  ``blend``: upwind weight of the mixed
    difference.  ``precision``: ``"fp64"`` or ``"fp32"`` (FP32 deviation storage).
    ``scheme``: 1 = T2S2-FDLBM1 (Eq. 2.23, A = 0 gives T1S2), 2 = T2S2-FDLBM2 (Eq. 5.23).
    ``graph_steps``: > 0 replays a CUDA graph of that many steps inside ``step``
    (small grids, where launch latency dominates).  ``equilibrium``:
    ``"standard"`` (Eq. 3.2) or ``"incompressible"`` (the equilibrium of He and
    Luo that Sec. 2 cites; velocity from rho0 u = sum xi f).
    """

    def __init__(self, xa, ya, *, nu: float, cfl: float, blend: float, A: float = 0.5,
                 precision: str = "fp64", rho0: float = 1.0, has_force: bool = False,
                 wall_u=None, path: str = "auto", rows_per_cta: int = 0, variant: str = "auto",
                 scheme: int = 1, adjoint: bool = False, graph_steps: int = 0, stream=None,
                 device=None, equilibrium: str = "standard"):
        self._L = L = B.load()
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.nx, self.ny = xa.n, ya.n
        self._grid, self._keep = B.make_grid(xa, ya, wall_u)
        self._mx = np.ascontiguousarray(xa.metric, dtype=np.float64)
        self._my = np.ascontiguousarray(ya.metric, dtype=np.float64)
        m = B.Metrics()
        m.dzeta_dx, m.dmu_dy = B._dptr(self._mx), B._dptr(self._my)
        o = B.Opts()
        L.fdlbm_default_opts(ctypes.byref(o))
        o.A, o.rho0 = A, rho0
        o.precision = {"fp64": B.FP64, "fp32": B.FP32_DEV}[precision]
        o.has_force = int(has_force)
        o.path = {"auto": B.PATH_AUTO, "fused": B.PATH_FUSED, "staged": B.PATH_STAGED}[path]
        o.rows_per_cta = rows_per_cta
        o.scheme = {1: B.SCHEME_T2S2_1, 2: B.SCHEME_T2S2_2}[scheme]
        o.adjoint = int(adjoint)
        o.graph_steps = graph_steps
        o.equilibrium = {"standard": B.EQ_STANDARD, "incompressible": B.EQ_INCOMPRESSIBLE}[equilibrium]
        o.variant = {"auto": B.VARIANT_AUTO, "scalar": B.VARIANT_SCALAR,
                     "warp": B.VARIANT_WARP}[variant]
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        o.stream = self.stream.cuda_stream
        nbytes = L.fdlbm_workspace_bytes(ctypes.byref(self._grid), ctypes.byref(o))
        if nbytes == 0:
            raise B.FdlbmError(-1, "invalid grid/options (workspace size 0)")
        # torch allocations are 512-byte aligned
        self._ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        o.workspace, o.workspace_bytes = self._ws.data_ptr(), nbytes
        h = ctypes.c_void_p()
        rc = L.fdlbm_create(ctypes.byref(self._grid), ctypes.byref(m), nu, cfl, blend,
                            ctypes.byref(o), ctypes.byref(h))
        _check(L, None, rc, "fdlbm_create")
        self._h = h
        self.precision = precision

    @classmethod
    def _case_view(cls, L, handle, xa, ya, stream, device, precision, batch):
        """A non-owning view of case handle `handle` of a batch."""
        self = cls.__new__(cls)
        self._L = L
        self._h = handle
        self._owned = False
        self._batch = batch  # keeps the batch (and its memory) alive
        self.nx, self.ny = xa.n, ya.n
        self.stream = stream
        self.device = device
        self.precision = precision
        return self

    # ----------------------------------------------------------- lifetime
    def close(self):
        if getattr(self, "_h", None) and getattr(self, "_owned", True):
            self._L.fdlbm_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ----------------------------------------------------------- properties
    @property
    def dt(self) -> float:
        return self._L.fdlbm_dt(self._h)

    @property
    def tau(self) -> float:
        return self._L.fdlbm_tau(self._h)

    @property
    def path(self) -> str:
        return {B.PATH_FUSED: "fused", B.PATH_STAGED: "staged"}[self._L.fdlbm_path(self._h)]

    @property
    def describe(self) -> str:
        return self._L.fdlbm_describe(self._h).decode()

    @property
    def kernels_per_step(self) -> int:
        return self._L.fdlbm_kernels_per_step(self._h)

    @property
    def steps_done(self) -> int:
        return self._L.fdlbm_steps_done(self._h)

    # ----------------------------------------------------------- marshalling
    def _arg(self, a, shape):
        """(pointer, where, keepalive) for a numpy array or CUDA tensor of FP64."""
        if a is None:
            return None, B.MEM_HOST, None
        if isinstance(a, torch.Tensor):
            if a.is_cuda:
                t = a.detach().to(torch.float64).contiguous()
                assert tuple(t.shape) == shape, (t.shape, shape)
                return t.data_ptr(), B.MEM_DEVICE, t
            a = a.detach().cpu().numpy()
        arr = np.ascontiguousarray(a, dtype=np.float64)
        assert arr.shape == shape, (arr.shape, shape)
        return arr.ctypes.data, B.MEM_HOST, arr

    def init_fields(self, rho, ux, uy, grad=None):
        """Eq. 3.2 (or Eq. 3.5 with the velocity gradient [dudx, dudy, dvdx, dvdy])."""
        sh = (self.ny, self.nx)
        args = [self._arg(v, sh) for v in (rho, ux, uy)]
        g = None
        if grad is not None:
            gs = torch.stack([torch.as_tensor(v) for v in grad]) if isinstance(grad[0], torch.Tensor) \
                else np.stack(grad)
            g = self._arg(gs, (4,) + sh)
        wheres = {w for _, w, _ in args} | ({g[1]} if g else set())
        if len(wheres) != 1:
            raise ValueError("all fields must live on the same side (host or device)")
        rc = self._L.fdlbm_init_fields(self._h, args[0][0], args[1][0], args[2][0],
                                       g[0] if g else None, wheres.pop())
        _check(self._L, self._h, rc, "init_fields")
        return self

    def init_fields_f32(self, drho, ux, uy, grad=None):
        """As init_fields, from FP32 fields with the density given as rho - rho0
        (numpy arrays or CUDA tensors, all on one side)."""
        sh = (self.ny, self.nx)
        # grad: a list of 4 fields, or one [4, ny, nx] array (kept as it is, so
        # that a pinned one is read in place)
        whole = grad is not None and not isinstance(grad, (list, tuple))
        fields = [drho, ux, uy] + (list(grad) if grad is not None and not whole else [])
        dev = isinstance(fields[0], torch.Tensor) and fields[0].is_cuda
        if dev:
            keep = [torch.as_tensor(v).detach().to(torch.float32).contiguous() for v in fields]
            ptrs = [t.data_ptr() for t in keep[:3]]
            g = None
            if grad is not None:
                g = grad.detach().to(torch.float32).contiguous() if whole else torch.stack(keep[3:])
        else:
            def host(v):
                return np.ascontiguousarray(np.asarray(v.cpu() if isinstance(v, torch.Tensor) else v),
                                            dtype=np.float32)
            keep = [host(v) for v in fields]
            ptrs = [a.ctypes.data for a in keep[:3]]
            g = None
            if grad is not None:
                g = host(grad) if whole else np.ascontiguousarray(np.stack(keep[3:]))
        if g is not None:
            assert tuple(g.shape) == (4,) + sh, (g.shape, sh)
        for a in keep[:3]:
            assert tuple(a.shape) == sh, (a.shape, sh)
        gp = None if g is None else (g.data_ptr() if dev else g.ctypes.data)
        rc = self._L.fdlbm_init_fields_f32(self._h, *ptrs, gp, B.MEM_DEVICE if dev else B.MEM_HOST)
        _check(self._L, self._h, rc, "init_fields_f32")
        return self

    def moments_f32(self, device: bool = False):
        """(rho - rho0, ux, uy) as FP32 arrays (CUDA tensors with device=True)."""
        sh = (self.ny, self.nx)
        if device:
            outs = [torch.empty(sh, dtype=torch.float32, device=self.device) for _ in range(3)]
            rc = self._L.fdlbm_moments_f32(self._h, *(o.data_ptr() for o in outs), B.MEM_DEVICE)
        else:
            outs = [np.empty(sh, dtype=np.float32) for _ in range(3)]
            rc = self._L.fdlbm_moments_f32(self._h, *(o.ctypes.data for o in outs), B.MEM_HOST)
        _check(self._L, self._h, rc, "moments_f32")
        return tuple(outs)

    def set_state(self, f):
        p, where, keep = self._arg(f, (9, self.ny, self.nx))
        _check(self._L, self._h, self._L.fdlbm_set_state(self._h, p, where), "set_state")
        if where == B.MEM_DEVICE:
            self.stream.synchronize()
        return self

    def get_state(self, device: bool = False):
        if device:
            out = torch.empty((9, self.ny, self.nx), dtype=torch.float64, device=self.device)
            _check(self._L, self._h, self._L.fdlbm_get_state(self._h, out.data_ptr(), B.MEM_DEVICE),
                   "get_state")
            return out
        out = np.empty((9, self.ny, self.nx))
        _check(self._L, self._h, self._L.fdlbm_get_state(self._h, out.ctypes.data, B.MEM_HOST),
               "get_state")
        return out

    def set_force(self, force):
        p, where, keep = self._arg(force, (2, self.ny, self.nx))
        _check(self._L, self._h, self._L.fdlbm_set_force(self._h, p, where), "set_force")
        if where == B.MEM_DEVICE:
            self.stream.synchronize()
        return self

    def step(self, n: int = 1):
        _check(self._L, self._h, self._L.fdlbm_step(self._h, int(n)), "step")
        return self

    def moments(self, device: bool = False):
        sh = (self.ny, self.nx)
        if device:
            outs = [torch.empty(sh, dtype=torch.float64, device=self.device) for _ in range(3)]
            rc = self._L.fdlbm_moments(self._h, *(o.data_ptr() for o in outs), B.MEM_DEVICE)
        else:
            outs = [np.empty(sh) for _ in range(3)]
            rc = self._L.fdlbm_moments(self._h, *(o.ctypes.data for o in outs), B.MEM_HOST)
        _check(self._L, self._h, rc, "moments")
        return tuple(outs)

    def reduce(self):
        """(Jacobian-weighted mass, successive-state residual or -1)."""
        m, r = ctypes.c_double(), ctypes.c_double()
        rc = self._L.fdlbm_reduce(self._h, ctypes.byref(m), ctypes.byref(r))
        _check(self._L, self._h, rc, "reduce")
        return m.value, r.value

    def sync(self):
        _check(self._L, self._h, self._L.fdlbm_sync(self._h), "sync")

    # ----------------------------------------------------------- reverse mode
    def layout(self):
        """(pitch, dtype) of the storage layout of states and cotangents."""
        p, e = ctypes.c_int(), ctypes.c_int()
        _check(self._L, self._h, self._L.fdlbm_state_layout(self._h, ctypes.byref(p), ctypes.byref(e)),
               "state_layout")
        return p.value, (torch.float32 if e.value == 4 else torch.float64)

    def new_buffer(self):
        """A zeroed device buffer in the storage layout, shaped [9, ny, pitch]."""
        pitch, dt = self.layout()
        return torch.zeros((9, self.ny, pitch), dtype=dt, device=self.device)

    def save_state(self, buf):
        _check(self._L, self._h, self._L.fdlbm_copy_state(self._h, buf.data_ptr(), 0), "copy_state")
        return buf

    def load_state(self, buf):
        _check(self._L, self._h, self._L.fdlbm_copy_state(self._h, buf.data_ptr(), 1), "copy_state")
        return self

    def adjoint_step(self, state_n, lam_next, lam_prev, dforce=None):
        rc = self._L.fdlbm_adjoint_step(self._h, state_n.data_ptr(), lam_next.data_ptr(),
                                        lam_prev.data_ptr(),
                                        dforce.data_ptr() if dforce is not None else None)
        _check(self._L, self._h, rc, "adjoint_step")

    def init_vjp(self, rho, ux, uy, lam, drho, dux, duy, dforce=None):
        """Add the cotangents of the fields of an equilibrium initialisation to
        drho (may be None), dux, duy, and that of the force field through the
        initial state to dforce (may be None), given the cotangent ``lam``
        (storage layout) of the state they produced (all CUDA tensors)."""
        def ptr(t):
            return None if t is None else t.data_ptr()
        for t in (rho, ux, uy, drho, dux, duy, dforce):
            assert t is None or (t.dtype == torch.float64 and t.is_contiguous() and t.is_cuda)
        rc = self._L.fdlbm_init_vjp(self._h, ptr(rho), ptr(ux), ptr(uy), ptr(lam), ptr(drho),
                                    ptr(dux), ptr(duy), ptr(dforce))
        _check(self._L, self._h, rc, "init_vjp")
        return self

    def moments_vjp(self, state, du, lam, dforce=None):
        du = du.detach().to(torch.float64).contiguous()
        rc = self._L.fdlbm_moments_vjp(self._h, state.data_ptr(), du.data_ptr(), lam.data_ptr(),
                                       dforce.data_ptr() if dforce is not None else None)
        _check(self._L, self._h, rc, "moments_vjp")
        return du


class FDLBMBatch:
    """Many independent cases stepped together (batched staged kernels, CUDA
    graph replay, autotuned block shape).  ``cases``: list of dicts with keys
    ``xa, ya, nu, cfl, blend`` and optional ``wall_u, has_force, A, scheme,
    equilibrium``.
    ``batch.case(c)`` returns an ``FDLBM`` view of case c for initialisation and
    read-back; ``batch.step(n)`` advances every case."""

    def __init__(self, cases, *, precision: str = "fp32", graph_steps: int = 50,
                 autotune: bool = True, mode: str = "auto", device=None):
        self._L = L = B.load()
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        n = len(cases)
        grids = (B.Grid * n)()
        mets = (B.Metrics * n)()
        opts = (B.Opts * n)()
        self._keep = []
        for c, cs in enumerate(cases):
            g, keep = B.make_grid(cs["xa"], cs["ya"], cs.get("wall_u"))
            grids[c] = g
            mx = np.ascontiguousarray(cs["xa"].metric, dtype=np.float64)
            my = np.ascontiguousarray(cs["ya"].metric, dtype=np.float64)
            mets[c].dzeta_dx, mets[c].dmu_dy = B._dptr(mx), B._dptr(my)
            self._keep += [keep, mx, my]
            L.fdlbm_default_opts(ctypes.byref(opts[c]))
            opts[c].precision = {"fp64": B.FP64, "fp32": B.FP32_DEV}[precision]
            opts[c].has_force = int(cs.get("has_force", False))
            opts[c].A = cs.get("A", 0.5)
            opts[c].scheme = {1: B.SCHEME_T2S2_1, 2: B.SCHEME_T2S2_2}[cs.get("scheme", 1)]
            opts[c].variant = {"auto": B.VARIANT_AUTO, "scalar": B.VARIANT_SCALAR,
                               "warp": B.VARIANT_WARP}[cs.get("variant", "auto")]
            opts[c].equilibrium = {"standard": B.EQ_STANDARD,
                                   "incompressible": B.EQ_INCOMPRESSIBLE}[cs.get("equilibrium", "standard")]
        nu = np.ascontiguousarray([cs["nu"] for cs in cases], dtype=np.float64)
        cfl = np.ascontiguousarray([cs["cfl"] for cs in cases], dtype=np.float64)
        blend = np.ascontiguousarray([cs["blend"] for cs in cases], dtype=np.float64)
        nbytes = L.fdlbm_batch_workspace_bytes(n, grids, opts)
        if nbytes == 0:
            raise B.FdlbmError(-1, "invalid batch (workspace size 0)")
        self._ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        h = ctypes.c_void_p()
        rc = L.fdlbm_batch_create(n, grids, mets, B._dptr(nu), B._dptr(cfl), B._dptr(blend), opts,
                                  graph_steps, int(autotune), self._ws.data_ptr(), nbytes,
                                  ctypes.byref(h))
        if rc != 0:
            raise B.FdlbmError(rc, "fdlbm_batch_create")
        if mode != "auto":
            rc = L.fdlbm_batch_set_mode(h, {"fused": B.BATCH_FUSED, "staged": B.BATCH_STAGED,
                                            "persistent": B.BATCH_PERSISTENT}[mode])
            if rc != 0:
                raise B.FdlbmError(rc, "fdlbm_batch_set_mode")
        self._h = h
        self.stream = torch.cuda.ExternalStream(L.fdlbm_batch_stream(h), device=self.device)
        self._cases = [FDLBM._case_view(L, L.fdlbm_batch_case(h, c), cs["xa"], cs["ya"], self.stream,
                                        self.device, precision, self)
                       for c, cs in enumerate(cases)]

    def case(self, c: int) -> FDLBM:
        return self._cases[c]

    def __len__(self):
        return len(self._cases)

    @property
    def cells(self) -> int:
        return self._L.fdlbm_batch_cells(self._h)

    @property
    def describe(self) -> str:
        return self._L.fdlbm_batch_describe(self._h).decode()

    def step(self, n: int = 1):
        rc = self._L.fdlbm_batch_step(self._h, int(n))
        if rc != 0:
            raise B.FdlbmError(rc, self._L.fdlbm_batch_last_error(self._h).decode())
        return self

    def sync(self):
        rc = self._L.fdlbm_batch_sync(self._h)
        if rc != 0:
            raise B.FdlbmError(rc, self._L.fdlbm_batch_last_error(self._h).decode())

    def set_spin_limit(self, polls: int):
        """Polls before a block of the persistent mode gives up at a grid
        barrier (0 exercises the timeout path; the default is 2**24)."""
        rc = self._L.fdlbm_batch_set_spin_limit(self._h, int(polls))
        if rc != 0:
            raise B.FdlbmError(rc, self._L.fdlbm_batch_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            for cv in self._cases:
                cv._h = None
            self._L.fdlbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
