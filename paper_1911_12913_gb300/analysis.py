"""Post-processing for the lid-driven cavity of Sec. 3C: marching to a steady
state under the successive-step residual of the cavity section, and locating
vortex centres from the stream function.  Host-side numpy on fields read back
through ``FDLBM.moments``; nothing here steps the scheme."""
import math

import numpy as np


def march_to_steady(solver, tol: float, *, check_every: int = 100, max_steps: int = 10**6):
    """Step until E(u) = |u^n - u^{n-1}| / |u^n| (one step apart, FP64 reduction
    on the GPU) drops below ``tol``, testing every ``check_every`` steps.

    Returns (steps, residual, history) with history = [(steps, residual), ...]
    every 100 checks; residual is the last one measured."""
    steps, res, hist = 0, math.inf, []
    while steps < max_steps:
        solver.step(check_every - 1)
        solver.reduce()
        solver.step(1)
        _, res = solver.reduce()
        steps += check_every
        if (steps // check_every) % 100 == 0:
            hist.append((steps, res))
        if res < tol:
            break
    return steps, res, hist


def stream_function(ya_coords, ux):
    """psi(x, y) = integral of u dy from the bottom wall (trapezoid rule on the
    node coordinates); [ny][nx]."""
    dy = np.diff(np.asarray(ya_coords, dtype=np.float64))
    psi = np.zeros_like(ux, dtype=np.float64)
    psi[1:] = np.cumsum(0.5 * (ux[1:] + ux[:-1]) * dy[:, None], axis=0)
    return psi


def _vertex(c, v):
    """Abscissa of the extremum of the parabola through three (c, v) points."""
    (x0, x1, x2), (f0, f1, f2) = c, v
    d01, d12 = (f1 - f0) / (x1 - x0), (f2 - f1) / (x2 - x1)
    a = (d12 - d01) / (x2 - x0)
    if a == 0:
        return x1
    # Newton form p = f0 + d01 (x - x0) + a (x - x0)(x - x1); p' = 0
    return 0.5 * (x0 + x1) - d01 / (2 * a)


def vortex_centre(xa_coords, ya_coords, psi, box, sign):
    """Centre of the vortex whose stream function has its extremum (minimum for
    sign < 0, maximum for sign > 0) inside box = (x0, x1, y0, y1): the extremal
    node refined by a parabola through it and its two neighbours along each axis.
    Returns (x, y, psi at the node)."""
    x = np.asarray(xa_coords, dtype=np.float64)
    y = np.asarray(ya_coords, dtype=np.float64)
    x0, x1, y0, y1 = box
    ix = np.where((x >= x0) & (x <= x1))[0]
    iy = np.where((y >= y0) & (y <= y1))[0]
    sub = sign * psi[np.ix_(iy, ix)]
    j, i = np.unravel_index(np.argmax(sub), sub.shape)
    J, I = iy[j], ix[i]
    xc, yc = x[I], y[J]
    if 0 < I < len(x) - 1:
        xc = _vertex(x[I - 1:I + 2], sign * psi[J, I - 1:I + 2])
    if 0 < J < len(y) - 1:
        yc = _vertex(y[J - 1:J + 2], sign * psi[J - 1:J + 2, I])
    return float(xc), float(yc), float(psi[J, I])
