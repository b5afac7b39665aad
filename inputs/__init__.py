"""Seeded synthetic inputs shared by the CPU oracle tests and the CUDA path.

This module only builds the *problem data* of the paper's test cases: node
coordinates and 1-D grid metrics of tensor-product grids (Sec. 3, Eqs. 3.9 and
3.11), closed-form flow fields (Taylor vortex Eq. 3.4, Poiseuille Eq. 3.7) and
seeded random fields.  It holds none of the lattice Boltzmann arithmetic: no
lattice velocities or weights, no equilibrium, no collision, no stencils.  Each
side (the oracle and the CUDA library) turns these fields into distributions
with its own code.

Array conventions: fields are float64 numpy arrays shaped ``[ny, nx]`` (row
index = y, column index = x).  A grid axis is a pair ``(coords, metric)`` where
``metric[k] = d(zeta)/dx`` at node ``k`` for the computational coordinate
``zeta`` = node index (unit spacing).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Axis", "periodic_axis", "wall_axis", "tanh_axis", "min_spacing",
    "taylor_green", "taylor_green_velocity", "poiseuille_velocity",
    "random_fields", "random_metric", "spectral_vorticity_velocity",
    "batched_cases", "batched_problem",
]


@dataclass
class Axis:
    """Node coordinates and metric of one grid axis.

    ``periodic``: node ``n`` coincides with node 0 (not stored).  Otherwise the
    first and last stored nodes are walls.
    """
    coords: np.ndarray
    metric: np.ndarray
    periodic: bool
    length: float = 0.0

    @property
    def n(self) -> int:
        return int(self.coords.shape[0])


def periodic_axis(n: int, lo: float, hi: float) -> Axis:
    """Uniform periodic axis with ``n`` unique nodes on ``[lo, hi)``."""
    dx = (hi - lo) / n
    x = lo + dx * np.arange(n, dtype=np.float64)
    return Axis(x, np.full(n, 1.0 / dx), True, hi - lo)


def wall_axis(n_cells: int, lo: float, hi: float) -> Axis:
    """Uniform axis with walls at both ends: ``n_cells + 1`` nodes, ends included."""
    dx = (hi - lo) / n_cells
    x = lo + dx * np.arange(n_cells + 1, dtype=np.float64)
    return Axis(x, np.full(n_cells + 1, 1.0 / dx), False, hi - lo)


def tanh_axis(n_cells: int, c: float) -> Axis:
    """Wall-clustered axis on [0, 1] from the tanh map of Eq. 3.9 (and 3.11).

    ``y = (a + tanh(c*mu)) / (2a)``, ``a = tanh(c)``, ``mu_j = (2j - N)/N`` for
    ``j = 0..N``; the metric is the analytic ``d(j)/dy``.  Eq. 3.11 prints
    ``zeta_i = i/N`` for the cavity, which maps only onto [1/2, 1]; the cavity
    uses this same symmetric parameterisation so that both walls are refined.
    """
    a = math.tanh(c)
    j = np.arange(n_cells + 1, dtype=np.float64)
    mu = (2.0 * j - n_cells) / n_cells
    y = (a + np.tanh(c * mu)) / (2.0 * a)
    dy_dmu = c / (2.0 * a) / np.cosh(c * mu) ** 2
    dy_dj = dy_dmu * (2.0 / n_cells)
    # The end nodes of the map are exactly 0 and 1.
    y[0], y[-1] = 0.0, 1.0
    return Axis(y, 1.0 / dy_dj, False, 1.0)


def min_spacing(*axes: Axis) -> float:
    """Smallest distance between neighbouring nodes over all axes."""
    best = math.inf
    for ax in axes:
        d = np.diff(ax.coords)
        if ax.periodic and ax.n > 0:
            d = np.append(d, ax.coords[0] + ax.length - ax.coords[-1])
        best = min(best, float(d.min()))
    return best


def _mesh(xa: Axis, ya: Axis):
    return np.meshgrid(xa.coords, ya.coords, indexing="xy")


def taylor_green(xa: Axis, ya: Axis, *, u0: float, k1: float = 1.0,
                 k2: float = 1.0, rho0: float = 1.0, cs2: float = 1.0 / 3.0,
                 phase=(0.0, 0.0)) -> dict:
    """Initial Taylor-vortex fields of Eq. 3.4 at t = 0 (optionally phase shifted).

    Returns ``rho, ux, uy`` and the velocity gradient ``dudx, dudy, dvdx, dvdy``.
    The density is ``rho0 + (p - p0)/cs2`` as the text of Sec. 3A states; the
    sound speed squared of the isothermal lattice gas is a problem parameter
    passed in by the caller.
    """
    X, Y = _mesh(xa, ya)
    ax = k1 * X + phase[0]
    ay = k2 * Y + phase[1]
    r = k1 / k2
    ux = -u0 * np.cos(ax) * np.sin(ay)
    uy = u0 * r * np.sin(ax) * np.cos(ay)
    dp = -0.25 * u0 * u0 * (np.cos(2 * ax) + r * r * np.cos(2 * ay))
    return dict(
        rho=rho0 + dp / cs2, ux=ux, uy=uy,
        dudx=u0 * k1 * np.sin(ax) * np.sin(ay),
        dudy=-u0 * k2 * np.cos(ax) * np.cos(ay),
        dvdx=u0 * r * k1 * np.cos(ax) * np.cos(ay),
        dvdy=-u0 * r * k2 * np.sin(ax) * np.sin(ay),
    )


def taylor_green_velocity(xa: Axis, ya: Axis, t: float, *, u0: float, nu: float,
                          k1: float = 1.0, k2: float = 1.0, phase=(0.0, 0.0)):
    """Closed-form Taylor-vortex velocity of Eq. 3.4 at time ``t``."""
    X, Y = _mesh(xa, ya)
    ax = k1 * X + phase[0]
    ay = k2 * Y + phase[1]
    decay = math.exp(-nu * (k1 * k1 + k2 * k2) * t)
    ux = -u0 * np.cos(ax) * np.sin(ay) * decay
    uy = u0 * (k1 / k2) * np.sin(ax) * np.cos(ay) * decay
    return ux, uy


def poiseuille_velocity(y: np.ndarray, *, H: float, u0: float) -> np.ndarray:
    """Steady channel profile of Eq. 3.7, ``4 u0 (y/H)(1 - y/H)``.

    Eq. 3.7 prints ``y/h`` in the first factor; ``h`` there is the channel
    height ``H`` (the profile must vanish at both walls and peak at ``u0``).
    """
    return 4.0 * u0 * (y / H) * (1.0 - y / H)


def random_fields(nx: int, ny: int, seed: int, *, du: float = 0.02,
                  drho: float = 0.01, dgrad: float = 0.01, smooth: bool = False) -> dict:
    """Seeded random ``rho, ux, uy`` and gradient-like fields.

    Used to build generic non-equilibrium states: each side feeds the
    "gradient" fields through its own non-equilibrium initialisation.
    With ``smooth`` the fields are sums of a few low Fourier modes.
    """
    rng = np.random.default_rng(seed)
    if smooth:
        X, Y = np.meshgrid(2 * np.pi * np.arange(nx) / nx,
                           2 * np.pi * np.arange(ny) / ny, indexing="xy")

        def fld(scale):
            out = np.zeros((ny, nx))
            for _ in range(4):
                kx, ky = rng.integers(0, 3, size=2)
                ph = rng.uniform(0, 2 * np.pi)
                out += rng.uniform(-1, 1) * np.cos(kx * X + ky * Y + ph)
            return scale * out / 4.0
    else:
        def fld(scale):
            return scale * rng.uniform(-1.0, 1.0, size=(ny, nx))
    out = dict(rho=1.0 + fld(drho), ux=fld(du), uy=fld(du))
    for k in ("dudx", "dudy", "dvdx", "dvdy"):
        out[k] = fld(dgrad)
    return out


def random_metric(n: int, seed: int, *, base: float = 1.0, spread: float = 0.5) -> np.ndarray:
    """Seeded positive metric array (used for invariants on arbitrary stretched grids)."""
    rng = np.random.default_rng(seed)
    return base * (1.0 + spread * rng.uniform(-1.0, 1.0, size=n))


def spectral_vorticity_velocity(n: int, seed: int, *, kmax: int = 8,
                                umax: float = 0.01):
    """Seeded smooth periodic velocity on the uniform ``n x n`` grid of [0, 2pi)^2.

    Vorticity ``w = sum_{1<=|k|<=kmax} A_k cos(k.x + phi_k)`` with
    ``|A_k|^2 ~ |k|^-2`` so the shell energy spectrum is ``E(k) ~ k^-3``;
    the velocity is ``u = (d psi/dy, -d psi/dx)`` with ``lap(psi) = -w``,
    rescaled so that ``max|u| = umax``.  Returns ``ux, uy`` and the exact
    gradient fields (computed spectrally).
    """
    rng = np.random.default_rng(seed)
    x = 2 * np.pi * np.arange(n) / n
    X, Y = np.meshgrid(x, x, indexing="xy")
    ux = np.zeros((n, n)); uy = np.zeros((n, n))
    g = {k: np.zeros((n, n)) for k in ("dudx", "dudy", "dvdx", "dvdy")}
    for kx in range(-kmax, kmax + 1):
        for ky in range(0, kmax + 1):
            if ky == 0 and kx <= 0:
                continue
            k2 = kx * kx + ky * ky
            if k2 < 1 or k2 > kmax * kmax:
                continue
            amp = rng.normal() / math.sqrt(k2)
            ph = rng.uniform(0, 2 * np.pi)
            th = kx * X + ky * Y + ph
            # psi = amp/k2 cos(th);  u = dpsi/dy, v = -dpsi/dx
            c, s = np.cos(th), np.sin(th)
            ux += -amp / k2 * ky * s
            uy += amp / k2 * kx * s
            g["dudx"] += -amp / k2 * ky * kx * c
            g["dudy"] += -amp / k2 * ky * ky * c
            g["dvdx"] += amp / k2 * kx * kx * c
            g["dvdy"] += amp / k2 * kx * ky * c
    scale = umax / max(np.abs(ux).max(), np.abs(uy).max())
    out = dict(ux=ux * scale, uy=uy * scale)
    out.update({k: v * scale for k, v in g.items()})
    return out


@dataclass
class Case:
    """One case of a batched sweep (sizes, kind, Reynolds number, stretching)."""
    kind: str          # "cavity" or "poiseuille"
    n: int             # cells per axis
    re: float
    stretched: bool
    extra: dict = field(default_factory=dict)


def batched_problem(case: "Case", *, U: float = 0.1, c: float = 1.5) -> dict:
    """Problem data of one batched case: axes, viscosity from the Reynolds
    number, wall velocities, and the uniform driving acceleration of a channel.

    cavity: unit square, walls on all sides, lid (north wall) speed U,
    nu = U / Re; tanh-clustered at the walls when ``stretched`` (Eq. 3.11 with
    the symmetric parameterisation), else uniform.
    channel: unit-height channel, periodic x with n nodes over the same length,
    walls in y (tanh map of Eq. 3.9 when ``stretched``), centre-line speed U,
    nu = U / Re, acceleration F = 8 nu U / H^2 (from Eq. 3.7).
    """
    n = case.n
    if case.kind == "cavity":
        ax = tanh_axis(n, c) if case.stretched else wall_axis(n, 0.0, 1.0)
        return dict(xa=ax, ya=ax, nu=U / case.re, wall_u=[(0.0, 0.0)] * 3 + [(U, 0.0)],
                    force=None)
    xa = periodic_axis(n, 0.0, 1.0)
    ya = tanh_axis(n, c) if case.stretched else wall_axis(n, 0.0, 1.0)
    nu = U / case.re
    force = np.zeros((2, ya.n, xa.n))
    force[0] = 8.0 * nu * U
    return dict(xa=xa, ya=ya, nu=nu, wall_u=None, force=force)


def batched_cases(count: int, seed: int, *, nmin: int = 33, nmax: int = 513,
                  re_min: float = 10.0, re_max: float = 2000.0) -> list:
    """Seeded mix of cavity and channel cases with uneven sizes and Reynolds numbers."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(nmin, nmax + 1))
        re = float(math.exp(rng.uniform(math.log(re_min), math.log(re_max))))
        kind = "cavity" if rng.uniform() < 0.5 else "poiseuille"
        out.append(Case(kind=kind, n=n, re=re, stretched=(i % 2 == 0)))
    return out
