"""Seeded synthetic inputs for the BTDF-IB / D2Q9 LBM cases.

This module only *generates inputs*: lattice sizes, relaxation times, initial
macroscopic fields and Lagrangian marker positions.  It contains none of the
method's arithmetic (no delta function, no equilibrium, no collision, no
interpolation or spreading).  Both the CPU oracle and the CUDA library are fed
from here, so the two sides see bit-identical inputs.

Lattice units throughout: dh = dt = c = 1, rho0 = 1.

Cases (the paper's cylinder benchmark, Sec. 5.2, scaled as stated):
  * ``small_cylinder``  160 x 80 lattice, D = 16, 50 markers, Re = 40.
  * ``paper_cylinder``  1600 x 800 lattice, D = 40, 126 markers,
                        Re in {0.1, 40, 200}, delta in {2, 3, 4}.
  * ``many_cylinders``  8192 x 4096 lattice, 400 cylinders of D = 20.
  * ``adjoint_cylinder`` 800 x 400 lattice, D = 24, 76 markers, Re = 100.
The inflow speed is U = 0.05; tau = 0.5 + 3 nu with nu = U D / Re (Sec. 2.1,
the relation below Eq. 7).  Boundary handling of the channel: inlet on x = 0,
zero-gradient outlet on x = nx-1, free-slip walls on y = 0 and y = ny-1
(Sec. 5.2 describes Dirichlet inflow and far-field walls with u_y = 0).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

# Boundary kinds, shared vocabulary of both implementations' C interfaces.
BCX_PERIODIC = 0
BCX_INOUT = 1
BCX_CONVECTIVE = 2
BCX_BOX = 3
BCY_PERIODIC = 0
BCY_FREESLIP = 1
BCY_NOSLIP = 2

U_IN = 0.05
NOISE = 1e-4


@dataclass
class Body:
    """One rigid body given by its Lagrangian markers."""
    X: np.ndarray
    Y: np.ndarray
    ds: float
    Ubx: np.ndarray
    Uby: np.ndarray
    D: float = 0.0


@dataclass
class Case:
    name: str
    nx: int
    ny: int
    tau: float
    u_in: float
    delta: int
    bc_x: int
    bc_y: int
    bodies: List[Body] = field(default_factory=list)
    gx: float = 0.0
    gy: float = 0.0
    drs: float = 0.0          # <= 0: the paper's constant for `delta`
    nf: int = 1
    seed: int = 0
    noise: float = NOISE
    Re: float = 0.0
    D: float = 0.0            # reference length for Cd / Cl

    def initial_fields(self) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
        return initial_fields(self.nx, self.ny, self.u_in, self.noise, self.seed)


def tau_from_re(re: float, u: float, d: float) -> float:
    """tau = 0.5 + 3 nu with nu = U D / Re (lattice units)."""
    return 0.5 + 3.0 * u * d / re


def circle_markers(cx: float, cy: float, d: float, n: int) -> Body:
    """n equally spaced markers on a circle of diameter d, at rest.

    X_l = cx + d/2 cos(2 pi l / n), Y_l = cy + d/2 sin(2 pi l / n),
    ds = pi d / n (arc length per marker).
    """
    th = 2.0 * np.pi * np.arange(n, dtype=np.float64) / n
    X = cx + 0.5 * d * np.cos(th)
    Y = cy + 0.5 * d * np.sin(th)
    return Body(X=X, Y=Y, ds=math.pi * d / n, Ubx=np.zeros(n), Uby=np.zeros(n), D=d)


def initial_fields(nx: int, ny: int, u: float, noise: float, seed: int):
    """rho = 1 and u = (U, 0) plus seeded Gaussian noise on both components.

    Returns float64 arrays of shape (ny, nx), x fastest.
    """
    rng = np.random.default_rng(seed)
    rho = np.ones((ny, nx), dtype=np.float64)
    ux = u + noise * rng.standard_normal((ny, nx))
    uy = noise * rng.standard_normal((ny, nx))
    return rho, ux, uy


def small_cylinder(delta: int = 4, seed: int = 1, re: float = 40.0) -> Case:
    """160 x 80, D = 16 at (40, 40), 50 markers, Re = 40 -> tau = 0.56."""
    d = 16.0
    c = Case("cyl160x80", 160, 80, tau_from_re(re, U_IN, d), U_IN, delta,
             BCX_INOUT, BCY_FREESLIP, seed=seed, Re=re, D=d)
    c.bodies.append(circle_markers(40.0, 40.0, d, 50))
    return c


def paper_cylinder(re: float = 200.0, delta: int = 3, seed: int = 2) -> Case:
    """1600 x 800, D = 40 at (400, 400), 126 markers."""
    d = 40.0
    c = Case(f"cyl1600x800_re{re:g}_d{delta}", 1600, 800, tau_from_re(re, U_IN, d),
             U_IN, delta, BCX_INOUT, BCY_FREESLIP, seed=seed, Re=re, D=d)
    c.bodies.append(circle_markers(400.0, 400.0, d, 126))
    return c


def paper_domain_cylinder(re: float = 200.0, delta: int = 3, seed: int = 4,
                          u: float = U_IN) -> Case:
    """The paper's own cylinder domain (Sec. 5.2): 40D x 40D with D/dh = 40,
    i.e. a 1601 x 1601 lattice, cylinder at (18D, 20D), 126 markers, inflow
    speed u (the paper does not state it)."""
    d = 40.0
    c = Case(f"cyl1601sq_re{re:g}_d{delta}", 1601, 1601, tau_from_re(re, u, d), u, delta,
             BCX_INOUT, BCY_FREESLIP, seed=seed, Re=re, D=d)
    c.bodies.append(circle_markers(18.0 * d, 20.0 * d, d, 126))
    return c


def batch_cases(count: int = 512, seed: int = 7) -> List[Case]:
    """Independent single-cylinder cases of uneven sizes: nx = 16 k with
    k uniform in 8..64 (128..1024), ny = nx / 2, D uniform in [10, min(40,
    ny / 5)], cylinder at (nx / 4, ny / 2), Re drawn from {0.1, 40, 200}."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        nx = 16 * int(rng.integers(8, 65))
        ny = nx // 2
        d = float(rng.uniform(10.0, min(40.0, ny / 5.0)))
        re = float(rng.choice([0.1, 40.0, 200.0]))
        n = max(8, int(round(math.pi * d)))
        c = Case(f"batch{i}", nx, ny, tau_from_re(re, U_IN, d), U_IN, 3, BCX_INOUT, BCY_FREESLIP,
                 seed=seed * 100003 + i, Re=re, D=d)
        c.bodies.append(circle_markers(nx / 4.0 + 0.31, ny / 2.0 + 0.17, d, n))
        out.append(c)
    return out


def adjoint_cylinder(seed: int = 5) -> Case:
    """800 x 400, D = 24 at (200, 200), 76 markers, Re = 100."""
    d = 24.0
    c = Case("cyl800x400_re100", 800, 400, tau_from_re(100.0, U_IN, d), U_IN, 3,
             BCX_INOUT, BCY_FREESLIP, seed=seed, Re=100.0, D=d)
    c.bodies.append(circle_markers(200.0, 200.0, d, 76))
    return c


def random_centres(nx: int, ny: int, d: float, count: int, seed: int,
                   min_gap: float = 2.0, wall_gap: float = 2.0,
                   inlet_gap: float = 4.0, max_tries: int = 2_000_000):
    """Rejection-sampled non-overlapping centres (centre distance >= min_gap*d,
    >= wall_gap*d from every wall, x >= inlet_gap*d)."""
    rng = np.random.default_rng(seed)
    pts: List[Tuple[float, float]] = []
    lo_x, hi_x = inlet_gap * d, nx - 1 - wall_gap * d
    lo_y, hi_y = wall_gap * d, ny - 1 - wall_gap * d
    cell = min_gap * d
    grid = {}
    tries = 0
    while len(pts) < count:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place the requested number of cylinders")
        x = rng.uniform(lo_x, hi_x)
        y = rng.uniform(lo_y, hi_y)
        gx, gy = int(x // cell), int(y // cell)
        ok = True
        for i in range(gx - 1, gx + 2):
            for j in range(gy - 1, gy + 2):
                for (px, py) in grid.get((i, j), ()):
                    if (px - x) ** 2 + (py - y) ** 2 < cell * cell:
                        ok = False
                        break
                if not ok:
                    break
            if not ok:
                break
        if ok:
            pts.append((x, y))
            grid.setdefault((gx, gy), []).append((x, y))
    return pts


def many_cylinders(nx: int = 8192, ny: int = 4096, count: int = 400, d: float = 20.0,
                   re: float = 200.0, delta: int = 3, seed: int = 3,
                   n_markers: int = 63) -> Case:
    """Large lattice with `count` cylinders at seeded random centres."""
    c = Case(f"cyl{nx}x{ny}_{count}cyl", nx, ny, tau_from_re(re, U_IN, d), U_IN, delta,
             BCX_INOUT, BCY_FREESLIP, seed=seed, Re=re, D=d)
    for (x, y) in random_centres(nx, ny, d, count, seed):
        c.bodies.append(circle_markers(x, y, d, n_markers))
    return c


def periodic_box(nx: int, ny: int, tau: float, seed: int = 0, u: float = 0.0,
                 noise: float = NOISE) -> Case:
    """Fully periodic box (used by the invariant and parity tests)."""
    return Case(f"periodic{nx}x{ny}", nx, ny, tau, u, 3, BCX_PERIODIC, BCY_PERIODIC,
                seed=seed, noise=noise)


def taylor_green_fields(n: int, u0: float):
    """Taylor-Green vortex on [-L, L]^2 sampled at n x n cell centres, L = n/2.

    u_x = -u0 cos(pi x/L) sin(pi y/L), u_y = u0 sin(pi x/L) cos(pi y/L)
    (Eqs. 40-41 at t = 0); rho = 1.
    """
    L = n / 2.0
    c = (np.arange(n) + 0.5) - L
    X, Y = np.meshgrid(c, c)
    ux = -u0 * np.cos(np.pi * X / L) * np.sin(np.pi * Y / L)
    uy = u0 * np.sin(np.pi * X / L) * np.cos(np.pi * Y / L)
    return np.ones((n, n)), ux, uy


def perimeter_nodes(nx: int, ny: int):
    """Outer nodes of an nx x ny lattice in the order the prescribed-velocity
    box takes its boundary velocities: row 0, row ny-1, column 0 without its
    corners, column nx-1 without its corners.  Returns (x, y) int arrays."""
    xs = [np.arange(nx), np.arange(nx), np.zeros(ny - 2, int), np.full(ny - 2, nx - 1)]
    ys = [np.zeros(nx, int), np.full(nx, ny - 1), np.arange(1, ny - 1), np.arange(1, ny - 1)]
    return np.concatenate(xs), np.concatenate(ys)


@dataclass
class TaylorGreenBox:
    """The decaying Taylor-Green vortex of Sec. 5.1 on [-L, L]^2 with L = N
    lattice units (dh = L / N): 2N + 1 nodes per side at x_i = -L + i, the
    outer ones on the box.  Re = u0 L / nu = 10 and tau = 0.65 as in the
    paper, so u0 = Re nu / L; T = u0 t / L = 1 is reached after 2 N^2 steps.
    Optionally a circle of diameter L at the centre, ds = dh."""
    N: int
    re: float = 10.0
    tau: float = 0.65

    @property
    def n(self) -> int:
        return 2 * self.N + 1

    @property
    def nu(self) -> float:
        return (self.tau - 0.5) / 3.0

    @property
    def u0(self) -> float:
        return self.re * self.nu / self.N

    def steps_to(self, T: float) -> int:
        return int(round(T * self.N / self.u0))

    def coords(self):
        c = np.arange(self.n, dtype=np.float64) - self.N
        return np.meshgrid(c, c)

    def velocity(self, x, y, t):
        """Eqs. 40-41 at lattice time t."""
        L, k = float(self.N), np.exp(-2.0 * np.pi ** 2 * self.nu * t / self.N ** 2)
        ux = -self.u0 * np.cos(np.pi * x / L) * np.sin(np.pi * y / L) * k
        uy = self.u0 * np.sin(np.pi * x / L) * np.cos(np.pi * y / L) * k
        return ux, uy

    def density(self, x, y, t):
        """Eq. 42 read with cos(2 pi y / L) (the printed sin is taken for a
        typo), c_s^2 = 1/3."""
        L, k = float(self.N), np.exp(-4.0 * np.pi ** 2 * self.nu * t / self.N ** 2)
        return 1.0 - 0.75 * self.u0 ** 2 * (np.cos(2 * np.pi * x / L) + np.cos(2 * np.pi * y / L)) * k

    def fields(self, t=0.0):
        X, Y = self.coords()
        ux, uy = self.velocity(X, Y, t)
        return self.density(X, Y, t), ux, uy

    def boundary(self, t):
        px, py = perimeter_nodes(self.n, self.n)
        return self.velocity(px - float(self.N), py - float(self.N), t)

    def circle(self) -> Body:
        m = max(8, int(round(np.pi * self.N)))
        return circle_markers(float(self.N), float(self.N), float(self.N), m)

    def marker_velocity(self, body: Body, t):
        return self.velocity(body.X - self.N, body.Y - self.N, t)

