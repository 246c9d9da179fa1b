"""Pins of the oracle's lattice Boltzmann core (Sec. 2.1, Eqs. 5-11) and of
its boundary rules.

Each pin is a fact fixed by the mathematics rather than a re-typed formula:
lattice moments of the equilibrium and of the Guo term, the exact momentum
budget of forced BGK (Eqs. 5, 7, 11), ballistic transport under streaming,
exact invariance of uniform flow under every boundary rule, the defining
property of non-equilibrium extrapolation, the Poiseuille closed form and the
Taylor-Green decay rate (Eqs. 40-41, second order, Sec. 5.1).
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


def test_equilibrium_moments():
    rng = np.random.default_rng(0)
    for _ in range(50):
        rho = 1.0 + 0.1 * rng.standard_normal()
        ux, uy = 0.1 * rng.standard_normal(2)
        f = O.feq(rho, ux, uy)
        assert abs(f.sum() - rho) < 1e-14
        assert abs((EX * f).sum() - rho * ux) < 1e-15
        assert abs((EY * f).sum() - rho * uy) < 1e-15
        # second moments: rho cs^2 delta_ij + rho u_i u_j, cs^2 = 1/3
        assert abs((EX * EX * f).sum() - (rho / 3 + rho * ux * ux)) < 1e-14
        assert abs((EY * EY * f).sum() - (rho / 3 + rho * uy * uy)) < 1e-14
        assert abs((EX * EY * f).sum() - rho * ux * uy) < 1e-15


def test_guo_term_moments():
    rng = np.random.default_rng(1)
    for _ in range(50):
        tau = 0.5 + rng.uniform(0.01, 2.0)
        ux, uy, fx, fy = 0.1 * rng.standard_normal(4)
        F = O.guo(tau, ux, uy, fx, fy)
        c = 1.0 - 1.0 / (2.0 * tau)
        assert abs(F.sum()) < 1e-15
        assert abs((EX * F).sum() - c * fx) < 1e-15
        assert abs((EY * F).sum() - c * fy) < 1e-15
        assert abs((EX * EX * F).sum() - c * 2 * ux * fx) < 1e-15
        assert abs((EY * EY * F).sum() - c * 2 * uy * fy) < 1e-15
        assert abs((EX * EY * F).sum() - c * (ux * fy + uy * fx)) < 1e-15


def _periodic_with_body(nf=1, g=(1e-5, -2e-5)):
    c = W.periodic_box(24, 20, 0.7, seed=3, u=0.03, noise=1e-3)
    s = O.Sim(c.nx, c.ny, c.tau, 0.0, W.BCX_PERIODIC, W.BCY_PERIODIC, g[0], g[1], 3, nf)
    s.init_fields(*c.initial_fields())
    b = W.circle_markers(12.3, 9.7, 6.0, 19)
    s.add_body(b.X, b.Y, b.ds)
    return s, g


@pytest.mark.parametrize("nf", [1, 3])
def test_exact_momentum_budget(nf):
    """Forced BGK adds exactly f + g of momentum per node per step and keeps
    mass: sum(e f') = rho u* + f (Eqs. 5, 7, 11)."""
    s, g = _periodic_with_body(nf)
    for _ in range(5):
        r0, ux0, uy0 = s.moments()
        s.step()
        r1, ux1, uy1 = s.moments()
        fx, fy = s.force_field()
        assert abs(r1.sum() - r0.sum()) < 1e-11
        dpx = (r1 * ux1).sum() - (r0 * ux0).sum()
        dpy = (r1 * uy1).sum() - (r0 * uy0).sum()
        assert abs(dpx - (fx.sum() + g[0] * r0.size)) < 1e-12
        assert abs(dpy - (fy.sum() + g[1] * r0.size)) < 1e-12
        assert np.abs(fx).max() > 1e-4  # the body really forces the fluid


def test_body_force_is_minus_fluid_force():
    """Eq. 27: both sides agree, and the body receives minus what the fluid gets."""
    s, _ = _periodic_with_body(1, g=(0.0, 0.0))
    s.step(3)
    fx, fy = s.force_field()
    Fx, Fy = s.history(0)
    assert abs(Fx[-1] + fx.sum()) < 1e-13
    assert abs(Fy[-1] + fy.sum()) < 1e-13


def _uniform_case(bc_x, bc_y, u=(0.04, 0.0), steps=50):
    nx, ny = 20, 12
    s = O.Sim(nx, ny, 0.63, u[0], bc_x, bc_y, 0.0, 0.0, 3, 1)
    s.init_fields(np.ones((ny, nx)), np.full((ny, nx), u[0]), np.full((ny, nx), u[1]))
    s.step(steps)
    return s.moments()


@pytest.mark.parametrize("bcx,bcy,u", [
    (W.BCX_PERIODIC, W.BCY_PERIODIC, (0.04, 0.013)),
    (W.BCX_PERIODIC, W.BCY_FREESLIP, (0.04, 0.0)),
    (W.BCX_INOUT, W.BCY_FREESLIP, (0.04, 0.0)),
    (W.BCX_INOUT, W.BCY_PERIODIC, (0.04, 0.0)),
    (W.BCX_CONVECTIVE, W.BCY_FREESLIP, (0.04, 0.0)),
    (W.BCX_CONVECTIVE, W.BCY_PERIODIC, (0.04, 0.0)),
    (W.BCX_PERIODIC, W.BCY_NOSLIP, (0.0, 0.0)),
])
def test_uniform_flow_is_exact_steady_state(bcx, bcy, u):
    r, ux, uy = _uniform_case(bcx, bcy, u)
    assert np.abs(r - 1).max() < 1e-14
    assert np.abs(ux - u[0]).max() < 1e-14
    assert np.abs(uy - u[1]).max() < 1e-14


def _ballistic(bc_y, a0, x0, y0, steps, nx=16, ny=6):
    """A small excess on one population travels without collision (tau huge)."""
    s = O.Sim(nx, ny, 1e15, 0.0, W.BCX_PERIODIC, bc_y, 0.0, 0.0, 3, 1)
    s.init_fields(np.ones((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx)))
    base = s.pops()
    f = base.copy()
    f[y0, x0, a0] += 1e-3
    s.set_pops(f)
    s.step(steps)
    d = s.pops() - base
    idx = np.argwhere(np.abs(d) > 5e-4)
    assert len(idx) == 1, idx
    return tuple(idx[0])


def _expected_track(bc_y, a0, x0, y0, steps, nx=16, ny=6):
    vx, vy = EX[a0], EY[a0]
    x, y = x0, y0
    for _ in range(steps):
        ny_ = y + vy
        if 0 <= ny_ < ny:
            x, y = (x + vx) % nx, ny_
        else:  # half-way wall: reflect the normal component (free-slip keeps
            # the tangential one and advances by it, bounce-back reverses it)
            vy = -vy
            if bc_y == W.BCY_NOSLIP:
                vx = -vx
            else:
                x = (x + vx) % nx
    a = int(np.where((EX == vx) & (EY == vy))[0][0])
    return (y, x, a)


@pytest.mark.parametrize("bcy", [W.BCY_FREESLIP, W.BCY_NOSLIP])
@pytest.mark.parametrize("a0", [2, 4, 5, 6, 7, 8])
def test_ballistic_transport_with_walls(bcy, a0):
    for steps in (1, 3, 7, 11):
        got = _ballistic(bcy, a0, 5, 2, steps)
        assert got == _expected_track(bcy, a0, 5, 2, steps), (steps, got)


def test_periodic_streaming_is_a_shift():
    nx, ny = 9, 7
    s = O.Sim(nx, ny, 1e15, 0.0, 0, 0, 0.0, 0.0, 3, 1)
    rng = np.random.default_rng(5)
    s.init_fields(1 + 0.01 * rng.standard_normal((ny, nx)), 0.01 * rng.standard_normal((ny, nx)),
                  0.01 * rng.standard_normal((ny, nx)))
    f0 = s.pops()
    s.step()
    f1 = s.pops()
    for a in range(9):
        expect = np.roll(np.roll(f0[:, :, a], EX[a], axis=1), EY[a], axis=0)
        assert np.abs(f1[:, :, a] - expect).max() < 1e-14


def test_inlet_extrapolation_imposes_velocity():
    """Non-equilibrium extrapolation: column 0 gets column 1's density and
    exactly the inlet velocity; the outlet column copies its neighbour."""
    c = W.small_cylinder(delta=3)
    s = O.Sim.from_case(c)
    s.step(20)
    r, ux, uy = s.moments()
    assert np.abs(ux[:, 0] - c.u_in).max() < 1e-14
    assert np.abs(uy[:, 0]).max() < 1e-14
    assert np.abs(r[:, 0] - r[:, 1]).max() < 1e-14
    f = s.pops()
    assert np.abs(f[:, -1, :] - f[:, -2, :]).max() == 0.0


def test_convective_outlet_holds_its_column_without_inflow():
    """With U = 0 the convective condition d f / dt + U d f / dx = 0 reads
    d f / dt = 0: the outlet column keeps its initial populations exactly,
    whatever the flow next to it does."""
    nx, ny = 24, 10
    rng = np.random.default_rng(3)
    s = O.Sim(nx, ny, 0.7, 0.0, W.BCX_CONVECTIVE, W.BCY_FREESLIP, 0.0, 0.0, 3, 1)
    s.init_fields(1.0 + 1e-3 * rng.standard_normal((ny, nx)), 0.02 * rng.standard_normal((ny, nx)),
                  0.02 * rng.standard_normal((ny, nx)))
    f0 = s.pops()
    s.step(30)
    f = s.pops()
    assert np.array_equal(f[:, -1, :], f0[:, -1, :])
    assert not np.array_equal(f[:, -2, :], f0[:, -2, :])


def test_convective_outlet_relaxes_towards_its_neighbour():
    """Each step moves the outlet column a fraction U / (1 + U) of the way
    from its previous value to the new neighbouring column (implicit upwind),
    so it always lies between the two; with U > 0 an outlet column that
    starts away from the neighbour's state converges to it."""
    c = W.small_cylinder(delta=3)
    c.bc_x = W.BCX_CONVECTIVE
    s = O.Sim.from_case(c)
    s.step(50)
    old = s.pops()[:, -1, :]
    s.step(1)
    f = s.pops()
    lo = np.minimum(old, f[:, -2, :]) - 1e-15
    hi = np.maximum(old, f[:, -2, :]) + 1e-15
    assert np.all(f[:, -1, :] >= lo) and np.all(f[:, -1, :] <= hi)
    z = O.Sim.from_case(W.small_cylinder(delta=3))
    z.step(51)
    assert not np.array_equal(f[:, -1, :], z.pops()[:, -1, :])   # not the zero-gradient copy


def _tg_box_error(N, T=0.5):
    tg = W.TaylorGreenBox(N)
    s = O.Sim(tg.n, tg.n, tg.tau, 0.0, W.BCX_BOX, 0, 0.0, 0.0, 3, 1)
    s.init_fields(*tg.fields(0.0))
    K = tg.steps_to(T)
    for k in range(1, K + 1):
        s.set_boundary_velocity(*tg.boundary(k))   # the boundary at the time the step reaches
        s.step(1)
    _, ux, uy = s.moments()
    X, Y = tg.coords()
    ax, ay = tg.velocity(X, Y, K)
    return math.sqrt((((ux - ax) ** 2 + (uy - ay) ** 2).sum()) / ((ax ** 2 + ay ** 2).sum()))


def test_taylor_green_box_second_order():
    """Sec. 5.1 without the circle: the decaying vortex (Eqs. 40-42) in the
    box [-L, L]^2 whose outer nodes carry the exact velocity by
    non-equilibrium extrapolation converges at second order (Eq. 43 error
    ratio ~4 per halving of dh)."""
    e = [_tg_box_error(N) for N in (8, 16, 32)]
    r1, r2 = e[0] / e[1], e[1] / e[2]
    assert 3.3 < r1 < 4.6 and 3.3 < r2 < 4.6, (e, r1, r2)


def test_box_keeps_a_uniform_flow():
    """A uniform flow whose velocity is also prescribed on the box stays
    exactly uniform."""
    n, u = 12, (0.03, -0.02)
    s = O.Sim(n, n, 0.7, 0.0, W.BCX_BOX, 0, 0.0, 0.0, 3, 1)
    s.init_fields(np.ones((n, n)), np.full((n, n), u[0]), np.full((n, n), u[1]))
    px, _ = W.perimeter_nodes(n, n)
    s.set_boundary_velocity(np.full(len(px), u[0]), np.full(len(px), u[1]))
    s.step(40)
    r, ux, uy = s.moments()
    assert np.abs(r - 1).max() < 1e-14
    assert np.abs(ux - u[0]).max() < 1e-14 and np.abs(uy - u[1]).max() < 1e-14


def _poiseuille(tau, ny=16, g=1e-6, steps=None):
    nu = (tau - 0.5) / 3.0
    if steps is None:
        steps = int(40.0 * ny * ny / (nu * math.pi ** 2))
    s = O.Sim(4, ny, tau, 0.0, W.BCX_PERIODIC, W.BCY_NOSLIP, g, 0.0, 3, 1)
    s.init_fields(np.ones((ny, 4)), np.zeros((ny, 4)), np.zeros((ny, 4)))
    s.step(steps)
    r, ux, uy = s.moments()
    u = ux[:, 0] + g / (2.0 * r[:, 0])   # Eq. 11 with the uniform force
    return u, nu, g


@pytest.mark.parametrize("tau", [0.6, 0.8, 1.2])
def test_poiseuille_curvature(tau):
    u, nu, g = _poiseuille(tau)
    curv = u[2:] - 2 * u[1:-1] + u[:-2]
    assert np.abs(curv + g / nu).max() < 1e-6 * g / nu


def test_poiseuille_exact_at_magic_tau():
    """BGK with half-way bounce-back has no wall slip when (tau - 1/2)^2 = 3/16."""
    tau = 0.5 + math.sqrt(3.0 / 16.0)
    ny = 16
    u, nu, g = _poiseuille(tau, ny)
    y = np.arange(ny)
    exact = g / (2 * nu) * (y + 0.5) * (ny - 0.5 - y)
    assert np.abs(u - exact).max() < 1e-8 * exact.max()


def _tg_rate(n, tau=0.8, u0=1e-3):
    rho, ux, uy = W.taylor_green_fields(n, u0)
    s = O.Sim(n, n, tau, 0.0, 0, 0, 0.0, 0.0, 3, 1)
    s.init_fields(rho, ux, uy)
    nu = (tau - 0.5) / 3.0
    L = n / 2.0
    t_decay = L * L / (2 * math.pi ** 2 * nu)
    t1, t2 = int(0.2 * t_decay), int(1.2 * t_decay)
    s.step(t1)
    _, a1, b1 = s.moments()
    s.step(t2 - t1)
    _, a2, b2 = s.moments()
    amp1 = (a1 * ux + b1 * uy).sum()
    amp2 = (a2 * ux + b2 * uy).sum()
    rate = -math.log(amp2 / amp1) / (t2 - t1)
    exact = 2 * math.pi ** 2 * nu / (L * L)   # Eqs. 40-41 with Re = u0 L / nu
    return abs(rate / exact - 1.0)


def test_taylor_green_decay_second_order():
    e16, e32 = _tg_rate(16), _tg_rate(32)
    assert e16 < 0.02 and e32 < 0.005
    assert 3.0 < e16 / e32 < 5.0
