"""Reverse mode: the hand-written adjoint step and the checkpointed rollout
gradient, against (a) the transposed Jacobian of the oracle's step assembled
column by column from exact complex-step derivatives, (b) finite differences
of the GPU forward step, (c) central finite differences of the full rollout."""
import math

import numpy as np
import pytest

import inputs as I
import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1911_12913_gb300.adjoint import rollout_velocity, rollout_velocity_from_fields  # noqa: E402
from paper_1911_12913_gb300.solver import FDLBM  # noqa: E402

NU, CFL, BETA = 0.02, 0.4, 0.2


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _problem(nx, ny, seed, precision="fp64", metrics=True):
    xa = I.periodic_axis(nx, 0.0, 1.0)
    ya = I.periodic_axis(ny, 0.0, 0.9)
    if metrics:
        xa.metric = I.random_metric(nx, seed + 1, base=nx, spread=0.3)
        ya.metric = I.random_metric(ny, seed + 2, base=ny / 0.9, spread=0.3)
    s = FDLBM(xa, ya, nu=NU, cfl=CFL, blend=BETA, has_force=True, adjoint=True,
              precision=precision)
    o = O.Oracle(xa, ya, nu=NU, dt=s.dt, beta=BETA)
    r = I.random_fields(nx, ny, seed)
    o.init_fields(r["rho"], r["ux"], r["uy"], grad=[r["dudx"], r["dudy"], r["dvdx"], r["dvdy"]])
    rng = np.random.default_rng(seed + 3)
    force = 2e-3 * rng.uniform(-1, 1, size=(2, ny, nx))
    return xa, ya, s, o.f.copy(), force, rng


def _to_buffer(s, arr):
    buf = s.new_buffer()
    buf[:, :, : s.nx] = torch.as_tensor(arr, dtype=buf.dtype, device=buf.device)
    return buf


@pytest.mark.parametrize("nx,ny", [(6, 5), (9, 7)])
def test_adjoint_step_equals_oracle_transposed_jacobian(nx, ny):
    xa, ya, s, f0, force, rng = _problem(nx, ny, seed=10 * nx + ny)
    lam = rng.normal(size=f0.shape)
    s.set_state(f0)
    s.set_force(force)
    state = s.save_state(s.new_buffer())
    out = s.new_buffer()
    dF = torch.zeros((2, ny, nx), dtype=torch.float64, device=s.device)
    s.adjoint_step(state, _to_buffer(s, lam), out, dF)
    s.sync()
    ref_f, ref_F = O.step_vjp(xa, ya, nu=NU, dt=s.dt, beta=BETA, f0=f0, lam=lam, force=force)
    got_f = out[:, :, :nx].cpu().numpy()
    assert rel(got_f, ref_f) <= 1e-12
    assert rel(dF.cpu().numpy(), ref_F) <= 1e-12


def test_adjoint_dot_product_against_forward_differences():
    """<J v, w> from central differences of the GPU forward step equals
    <v, J^T w> from the adjoint step (16 x 16, FP64)."""
    nx = ny = 16
    xa, ya, s, f0, force, rng = _problem(nx, ny, seed=5)
    s.set_state(f0)
    s.set_force(force)
    g = s.save_state(s.new_buffer())
    v = _to_buffer(s, rng.normal(size=f0.shape))
    w = _to_buffer(s, rng.normal(size=f0.shape))
    eps = 1e-6

    def step_of(buf):
        s.load_state(buf)
        s.step(1)
        return s.save_state(s.new_buffer())

    jv = (step_of(g + eps * v) - step_of(g - eps * v)) / (2 * eps)
    jtw = s.new_buffer()
    s.adjoint_step(g, w, jtw, None)
    s.sync()
    lhs = float((jv[:, :, :nx] * w[:, :, :nx]).sum())
    rhs = float((v[:, :, :nx] * jtw[:, :, :nx]).sum())
    assert abs(lhs - rhs) <= 1e-8 * abs(rhs)


def _loss_and_grad(s, f0buf, force, target, nsteps):
    F = torch.tensor(force, dtype=torch.float64, device=s.device, requires_grad=True)
    u = rollout_velocity(s, F, f0buf, nsteps)
    loss = 0.5 * ((u - target) ** 2).sum()
    loss.backward()
    return float(loss.detach()), F.grad.detach().cpu().numpy()


def _loss(s, f0buf, force, target, nsteps):
    F = torch.tensor(force, dtype=torch.float64, device=s.device)
    with torch.no_grad():
        u = rollout_velocity(s, F, f0buf, nsteps)
    return float(0.5 * ((u - target) ** 2).sum())


def test_rollout_gradient_matches_central_differences():
    """dJ/dF of J = 1/2 |u_N(F) - u*|^2 over a 30-step rollout (checkpoints every
    6 steps) against central differences along random directions (16 x 16, FP64)."""
    nx = ny = 16
    nsteps = 30
    xa, ya, s, f0, force, rng = _problem(nx, ny, seed=8)
    s.set_state(f0)
    f0buf = s.save_state(s.new_buffer())
    target = torch.zeros((2, ny, nx), dtype=torch.float64, device=s.device)
    hidden = force + 1e-3 * rng.uniform(-1, 1, size=force.shape)
    with torch.no_grad():
        target = rollout_velocity(s, torch.tensor(hidden, device=s.device), f0buf, nsteps).clone()
    J, grad = _loss_and_grad(s, f0buf, force, target, nsteps)
    assert J > 0
    def central(V, eps):
        return (_loss(s, f0buf, force + eps * V, target, nsteps) -
                _loss(s, f0buf, force - eps * V, target, nsteps)) / (2 * eps)

    for k in range(3):
        V = rng.normal(size=force.shape)
        # Richardson-extrapolated central difference: truncation O(eps^4)
        eps = 2e-4
        fd = (4.0 * central(V, eps / 2) - central(V, eps)) / 3.0
        ad = float(np.sum(grad * V))
        assert abs(fd - ad) <= 1e-6 * abs(fd), (k, fd, ad)


@pytest.mark.parametrize("eq,precision,forced,tol", [
    ("standard", "fp64", False, 1e-9), ("incompressible", "fp64", False, 1e-9),
    ("standard", "fp32", False, 1e-4), ("standard", "fp64", True, 1e-9),
    ("incompressible", "fp64", True, 1e-9), ("standard", "fp32", True, 1e-4)])
def test_init_vjp_dot_product(eq, precision, forced, tol):
    """fdlbm_init_vjp is the transpose of the initialisation f~ = f^eq -
    (dt/2) F_i (Eqs. 3.2, 2.19, 3.12): <J v, lam> = <v, J^T lam> with J v from
    central differences of fdlbm_set_force + fdlbm_init_fields along random
    directions of the density, the velocity and (forced cases) the force field
    (16 x 12, random fields)."""
    nx, ny = 16, 12
    xa = I.periodic_axis(nx, 0.0, 1.0)
    ya = I.periodic_axis(ny, 0.0, 0.8)
    s = FDLBM(xa, ya, nu=NU, cfl=CFL, blend=BETA, equilibrium=eq, precision=precision,
              has_force=forced)
    rng = np.random.default_rng(3)
    dev = s.device
    f = [torch.tensor(v, dtype=torch.float64, device=dev) for v in
         (1.0 + 0.05 * rng.uniform(-1, 1, (ny, nx)), 0.05 * rng.uniform(-1, 1, (ny, nx)),
          0.05 * rng.uniform(-1, 1, (ny, nx)))]
    v = [torch.tensor(rng.normal(size=(ny, nx)), dtype=torch.float64, device=dev) for _ in range(3)]
    # a force of 0.5 per unit time: (dt/2) F_i is then a few per cent of f^eq
    F = torch.tensor(0.5 * rng.uniform(-1, 1, (2, ny, nx)), dtype=torch.float64, device=dev)
    vF = torch.tensor(rng.normal(size=(2, ny, nx)), dtype=torch.float64, device=dev)
    lam = s.new_buffer()
    lam[:, :, :nx] = torch.tensor(rng.normal(size=(9, ny, nx)), dtype=lam.dtype, device=dev)

    def state_of(fields, force):
        if forced:
            s.set_force(force)
        s.init_fields(*fields)
        return s.save_state(s.new_buffer()).to(torch.float64)

    # the state is cubic in (rho, u) jointly, so central differences carry an
    # O(eps^2) error; FP32 rounding of the deviations (~1e-9) over eps = 1e-3
    # stays well below the tolerance
    eps = 1e-5 if precision == "fp64" else 1e-3
    jv = (state_of([a + eps * b for a, b in zip(f, v)], F + eps * vF) -
          state_of([a - eps * b for a, b in zip(f, v)], F - eps * vF)) / (2 * eps)
    g = [torch.zeros_like(a) for a in f]
    gF = torch.zeros_like(F)
    if forced:
        s.set_force(F)
    s.init_vjp(*f, lam, *g, gF if forced else None)
    s.sync()
    lhs = float((jv[:, :, :nx] * lam[:, :, :nx].to(torch.float64)).sum())
    rhs = float(sum((a * b).sum() for a, b in zip(v, g)))
    if forced:
        rhs += float((vF * gF).sum())
        assert float(gF.abs().max()) > 0
    assert abs(lhs - rhs) <= tol * abs(rhs), (lhs, rhs)


def test_rollout_gradient_wrt_initial_velocity():
    """dJ/d(u0, v0, rho0) of J = 1/2 |u_N - u*|^2 over a 30-step rollout from the
    equilibrium of the fields (checkpoints every 6 steps) against central
    differences along random directions (16 x 16, FP64, with a force field)."""
    nx = ny = 16
    nsteps = 30
    xa, ya, s, _, force, rng = _problem(nx, ny, seed=12)
    dev = s.device
    F = torch.tensor(force, dtype=torch.float64, device=dev)
    r = I.random_fields(nx, ny, 31, du=0.03, drho=0.02)
    base = [torch.tensor(r[k], dtype=torch.float64, device=dev) for k in ("rho", "ux", "uy")]
    with torch.no_grad():
        tgt = rollout_velocity_from_fields(s, F, base[0], base[1] + 0.01, base[2], nsteps).clone()

    def loss(fields, grad=False):
        fs = [t.clone().requires_grad_(grad) for t in fields]
        u = rollout_velocity_from_fields(s, F, *fs, nsteps)
        J = 0.5 * ((u - tgt) ** 2).sum()
        if grad:
            J.backward()
            return float(J.detach()), [t.grad.detach() for t in fs]
        return float(J.detach())

    J, grads = loss(base, grad=True)
    assert J > 0 and all(float(g.abs().max()) > 0 for g in grads)

    def central(V, eps):
        up = [a + eps * b for a, b in zip(base, V)]
        dn = [a - eps * b for a, b in zip(base, V)]
        with torch.no_grad():
            return (loss(up) - loss(dn)) / (2 * eps)

    for k in range(3):
        V = [torch.tensor(rng.normal(size=(ny, nx)), dtype=torch.float64, device=dev) for _ in range(3)]
        eps = 2e-4
        fd = (4.0 * central(V, eps / 2) - central(V, eps)) / 3.0
        ad = float(sum((g * b).sum() for g, b in zip(grads, V)))
        assert abs(fd - ad) <= 1e-6 * abs(fd), (k, fd, ad)

    # d/d force of the same rollout: through the steps and through the initial
    # state, which carries -(dt/2) F_i (Eq. 2.19)
    Fg = F.clone().requires_grad_(True)
    u = rollout_velocity_from_fields(s, Fg, *base, nsteps)
    (0.5 * ((u - tgt) ** 2).sum()).backward()
    VF = torch.tensor(rng.normal(size=(2, ny, nx)), dtype=torch.float64, device=dev)

    def central_F(eps):
        with torch.no_grad():
            jp = 0.5 * float(((rollout_velocity_from_fields(s, F + eps * VF, *base, nsteps) - tgt) ** 2).sum())
            jm = 0.5 * float(((rollout_velocity_from_fields(s, F - eps * VF, *base, nsteps) - tgt) ** 2).sum())
        return (jp - jm) / (2 * eps)

    eps = 1e-4
    fd = (4.0 * central_F(eps / 2) - central_F(eps)) / 3.0
    ad = float((Fg.grad * VF).sum())
    assert abs(fd - ad) <= 1e-6 * abs(fd), (fd, ad)


def test_recover_initial_velocity_by_gradient_descent():
    """The inverse problem on the initial state: from the rest state, recover a
    hidden smooth initial velocity (k <= 2, max 5e-3) on a 32 x 32 periodic grid
    from the velocity after 60 steps, by steepest descent with the gradient of
    rollout_velocity_from_fields and an exact line search on the (nearly
    linear) misfit.  Six iterations cut the misfit at least 100-fold."""
    n, nsteps = 32, 60
    ax = I.periodic_axis(n, 0.0, 2 * math.pi)
    s = FDLBM(ax, ax, nu=0.01, cfl=0.5, blend=0.1, has_force=True, adjoint=True)
    dev = s.device
    F = torch.zeros((2, n, n), dtype=torch.float64, device=dev)
    h = I.spectral_vorticity_velocity(n, 5, kmax=2, umax=5e-3)
    hidden = [torch.tensor(h[k], dtype=torch.float64, device=dev) for k in ("ux", "uy")]
    rho = torch.ones((n, n), dtype=torch.float64, device=dev)
    with torch.no_grad():
        tgt = rollout_velocity_from_fields(s, F, rho, *hidden, nsteps).clone()

    def misfit(u0):
        with torch.no_grad():
            return rollout_velocity_from_fields(s, F, rho, *u0, nsteps) - tgt

    x = [torch.zeros_like(hidden[0]), torch.zeros_like(hidden[1])]
    J0 = 0.5 * float((misfit(x) ** 2).sum())
    for _ in range(6):
        xs = [t.clone().requires_grad_(True) for t in x]
        u = rollout_velocity_from_fields(s, F, rho, *xs, nsteps)
        (0.5 * ((u - tgt) ** 2).sum()).backward()
        g = [t.grad.detach() for t in xs]
        r0 = misfit(x)
        eps = 1e-3 / float(max(t.abs().max() for t in g))
        Ag = (misfit([a + eps * b for a, b in zip(x, g)]) - r0) / eps
        alpha = float(sum((b * b).sum() for b in g)) / float((Ag * Ag).sum())
        x = [a - alpha * b for a, b in zip(x, g)]
    J = 0.5 * float((misfit(x) ** 2).sum())
    err = math.sqrt(sum(float(((a - b) ** 2).sum()) for a, b in zip(x, hidden)) /
                    sum(float((b ** 2).sum()) for b in hidden))
    print(f"initial-velocity recovery: misfit {J0:.3e} -> {J:.3e}, rel error of u0 {err:.3e}")
    assert J <= 1e-2 * J0


def test_fp32_adjoint_close_to_fp64():
    nx, ny = 40, 33
    res = {}
    for prec in ("fp64", "fp32"):
        xa, ya, s, f0, force, rng = _problem(nx, ny, seed=21, precision=prec)
        lam = np.random.default_rng(99).normal(size=f0.shape)
        s.set_state(f0)
        s.set_force(force)
        state = s.save_state(s.new_buffer())
        out = s.new_buffer()
        dF = torch.zeros((2, ny, nx), dtype=torch.float64, device=s.device)
        s.adjoint_step(state, _to_buffer(s, lam), out, dF)
        s.sync()
        res[prec] = (out[:, :, :nx].double().cpu().numpy(), dF.cpu().numpy())
    e_lam = rel(res["fp32"][0], res["fp64"][0])
    e_F = rel(res["fp32"][1], res["fp64"][1])
    print(f"FP32 adjoint vs FP64: rel lam {e_lam:.2e}, rel dF {e_F:.2e}")
    assert e_lam <= 1e-5 and e_F <= 1e-4


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 1e-5)])
def test_adjoint_256_against_oracle_directional_derivative(precision, tol):
    """The adjoint step on the inverse problem's grid (256^2 periodic, initial
    velocity from a k^-3 vorticity spectrum up to k = 8, smooth force field):
    <J v, w>, with J v the oracle's complex-step directional derivative of one
    step along a random state and force direction (exact to rounding), equals
    <v, J^T w> from the GPU adjoint step."""
    n = 256
    ax = I.periodic_axis(n, 0.0, 2 * math.pi)
    s = FDLBM(ax, ax, nu=0.01, cfl=0.5, blend=0.1, precision=precision, has_force=True,
              adjoint=True)
    v = I.spectral_vorticity_velocity(n, 11, kmax=8, umax=0.01)
    o = O.Oracle(ax, ax, nu=0.01, dt=s.dt, beta=0.1)
    one = np.ones((n, n))
    o.init_fields(one, v["ux"], v["uy"], [v["dudx"], v["dudy"], v["dvdx"], v["dvdy"]])
    f0 = o.f.copy()
    h = I.spectral_vorticity_velocity(n, 12, kmax=8, umax=1e-5)
    F = np.stack([h["ux"], h["uy"]])
    rng = np.random.default_rng(256)
    dv, dF, w = rng.normal(size=f0.shape), rng.normal(size=F.shape), rng.normal(size=f0.shape)
    eps = 1e-20
    y = O.step_complex(ax, ax, nu=0.01, dt=s.dt, beta=0.1, f=f0 + 1j * eps * dv,
                       force=F + 1j * eps * dF)
    lhs = float(np.sum(y.imag / eps * w))
    s.set_state(f0)
    s.set_force(F)
    state = s.save_state(s.new_buffer())
    out = s.new_buffer()
    dFg = torch.zeros((2, n, n), dtype=torch.float64, device=s.device)
    s.adjoint_step(state, _to_buffer(s, w), out, dFg)
    s.sync()
    rhs = float(np.sum(dv * out[:, :, :n].double().cpu().numpy()) + np.sum(dF * dFg.cpu().numpy()))
    print(f"{precision} 256^2: <Jv, w> = {lhs:.12e}, <v, J^T w> = {rhs:.12e}, rel {abs(lhs - rhs) / abs(lhs):.2e}")
    assert abs(lhs - rhs) <= tol * abs(lhs)


def test_adjoint_rejects_walls_and_missing_scratch():
    xa = I.periodic_axis(16, 0.0, 1.0)
    s = FDLBM(xa, xa, nu=NU, cfl=CFL, blend=BETA)        # no adjoint scratch
    b = s.new_buffer()
    with pytest.raises(Exception, match="EUNSUPPORTED"):
        s.adjoint_step(b, b.clone(), s.new_buffer())
    wa = I.wall_axis(15, 0.0, 1.0)
    w = FDLBM(xa, wa, nu=NU, cfl=CFL, blend=BETA, adjoint=True)
    bw = w.new_buffer()
    with pytest.raises(Exception, match="EUNSUPPORTED"):
        w.adjoint_step(bw, bw.clone(), w.new_buffer())
