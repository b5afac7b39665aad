"""Numerical von Neumann check (Sec. 2C): the spectral radius of the step
linearised about a uniform flow on a small periodic grid.

The Jacobian of the oracle's step is assembled column by column from exact
complex-step derivatives (complex build of the same oracle); its eigenvalues
are the amplification factors of every Fourier mode the 8 x 8 grid carries.
With unit spacing, CFL = dt and omega = dt / tau."""
import numpy as np
import pytest

import inputs as I
import oracle as O


def spectral_radius(cfl, omega, *, u=(0.01, 0.01), beta=0.1, A=0.5, n=8, scheme=1):
    xa = I.periodic_axis(n, 0.0, float(n))
    ya = I.periodic_axis(n, 0.0, float(n))
    dt = cfl
    nu = dt / omega / 3.0
    o = O.Oracle(xa, ya, nu=nu, dt=dt, beta=beta, A=A, scheme=scheme)
    one = np.ones((n, n))
    o.init_fields(one, u[0] * one, u[1] * one)
    f0 = o.f.copy()
    J = np.empty((f0.size, f0.size))
    for k in range(f0.size):
        x = f0.astype(np.complex128).ravel()
        x[k] += 1e-20j
        y = O.step_complex(xa, ya, nu=nu, dt=dt, beta=beta, A=A, f=x.reshape(f0.shape),
                           scheme=scheme)
        J[:, k] = (y.imag / 1e-20).ravel()
    return float(np.abs(np.linalg.eigvals(J)).max())


@pytest.mark.parametrize("cfl", [0.5, 0.8, 0.9])
def test_t2s2_stable_to_cfl_09_in_the_taylor_vortex_regime(cfl):
    """Sec. 3A / Table 3: T2S2-FDLBM1 (A = 1/2, eta = 0.1) works up to CFL 0.9
    (Taylor-vortex regime: |u| ~ 0.01, dt/tau ~ 15)."""
    assert spectral_radius(cfl, 15.0) <= 1.0 + 1e-10


def test_t2s2_unstable_beyond_cfl_1():
    assert spectral_radius(1.0, 15.0) > 1.005


def test_t1s2_growth_rates():
    """Table 3 reports T1S2 unstable from CFL 0.3.  Its amplification exceeds 1
    already at CFL 0.1 but only by ~7e-4 per step (a factor ~1e5 over the
    16612 steps of Table 4, invisible from round-off); at CFL 0.3 it is 1.2 %
    per step (a factor ~1e28 over its 5537 steps)."""
    r1 = spectral_radius(0.1, 15.0, A=0.0)
    r3 = spectral_radius(0.3, 15.0, A=0.0)
    assert 1.0 < r1 < 1.002
    assert r3 > 1.01
    assert 5537 * np.log(r3) > 20 * np.log(10)   # round-off grows past O(1)
    assert 16612 * np.log(r1) < 14 * np.log(10)


def test_nearly_collisionless_regime_is_unstable():
    """The reading used for the throughput workload: at CFL 0.5 the step is
    stable for dt/tau >= 0.1 but unstable at dt/tau = 0.026 (nu = 0.01 on a
    4096^2 grid of [0, 2pi)^2), so that workload uses nu = 0.001."""
    assert spectral_radius(0.5, 1.0, u=(0.2, 0.2)) <= 1.0 + 1e-10
    assert spectral_radius(0.5, 0.1, u=(0.2, 0.2)) <= 1.0 + 1e-10
    assert spectral_radius(0.5, 0.026, u=(0.2, 0.2)) > 1.01


# omega = dt / tau of the Taylor vortex of Sec. 3A at a given CFL: dt = CFL *
# 2 pi / 128 and tau = 3 nu = 0.003
TV_OMEGA_PER_CFL = 2 * np.pi / 128 / 0.003


@pytest.mark.parametrize("cfl", [0.6, 0.7, 0.8])
def test_fdlbm2_stable_to_cfl_08(cfl):
    """T2S2-FDLBM2 (Eq. 5.23) at eta = 0.1 with the Taylor vortex's dt / tau is
    stable up to CFL 0.8 ..."""
    assert spectral_radius(cfl, TV_OMEGA_PER_CFL * cfl, scheme=2) <= 1.0 + 1e-10


def test_fdlbm2_unstable_at_cfl_09_where_fdlbm1_is_stable():
    """... and unstable at CFL 0.9 (the worst mode of the 8 x 8 grid grows by
    about 8 % per step), where T2S2-FDLBM1 is still stable.  The Taylor-vortex
    CFL table of Sec. 3A shows the same split: T2S2-FDLBM2 fails at CFL 0.9
    (GRE 1.01) while T2S2-FDLBM1 keeps a small error there."""
    om = TV_OMEGA_PER_CFL * 0.9
    assert spectral_radius(0.9, om, scheme=2) > 1.05
    assert spectral_radius(0.9, om, scheme=1) <= 1.0 + 1e-10
