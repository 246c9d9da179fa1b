"""The Taylor-Green test of Sec. 5.1 on the GPU: the decaying vortex
(Eqs. 40-42) in the box [-L, L]^2 whose outer nodes carry the exact velocity
(BTDF_BCX_BOX, non-equilibrium extrapolation), with a circle of diameter L
at its centre whose markers carry the exact velocity (BTDF forcing,
3-point delta).  Re = 10, tau = 0.65, ds = dh, up to T = u0 t / L = 1.

* Against the FP64 oracle step for step (N = 10 and 20, with the circle;
  N = 16 without it): velocity field within max(1e-5, n 2^-24).
* Fig. 5's claim: the overall velocity error and the boundary error of the
  interpolated velocity converge at about second order, N = 10 .. 80.

Time levels: the library applies the box rule when it streams into the next
step, so the velocity set before step k belongs to the state of step k-1;
the oracle applies it at the end of step k.  Markers act on the state each
step starts from, time k-1, in both.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1806_09403_gb300 import _build  # noqa: E402
from paper_1806_09403_gb300 import btdf as B  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()


def gpu_run(N, T=1.0, circle=True):
    tg = W.TaylorGreenBox(N)
    lat = B.Lattice(tg.n, tg.n, tg.tau, 0.0, 3, 1, B.BTDF_F32, B.BTDF_BCX_BOX, B.BTDF_BCY_PERIODIC,
                    history_len=64)
    lat.init_fields(*tg.fields(0.0))
    b = tg.circle() if circle else None
    if circle:
        lat.add_markers(b.X, b.Y, b.ds)
    K = tg.steps_to(T)
    for k in range(1, K + 1):
        if k > 1:
            lat.set_boundary_velocity(*tg.boundary(k - 1))
        if circle:
            lat.set_marker_velocity(0, *tg.marker_velocity(b, k - 1))
        lat.step(1)
    lat.set_boundary_velocity(*tg.boundary(K))   # the read-back pulls the state of step K
    return tg, lat, b, K


def oracle_run(N, T=1.0, circle=True):
    tg = W.TaylorGreenBox(N)
    s = O.Sim(tg.n, tg.n, tg.tau, 0.0, W.BCX_BOX, 0, 0.0, 0.0, 3, 1)
    s.init_fields(*tg.fields(0.0))
    b = tg.circle() if circle else None
    if circle:
        s.add_body(b.X, b.Y, b.ds)
    K = tg.steps_to(T)
    for k in range(1, K + 1):
        s.set_boundary_velocity(*tg.boundary(k))
        if circle:
            s.set_marker_velocity(0, *tg.marker_velocity(b, k - 1))
        s.step(1)
    return s


def rel(ax, ay, bx, by):
    return math.sqrt((((ax - bx) ** 2 + (ay - by) ** 2).sum()) / ((bx ** 2 + by ** 2).sum()))


@pytest.mark.parametrize("N,circle", [(10, True), (20, True), (16, False)])
def test_against_oracle(N, circle):
    tg, lat, b, K = gpu_run(N, circle=circle)
    sim = oracle_run(N, circle=circle)
    _, ux, uy = lat.moments()
    _, rx, ry = sim.moments()
    e = rel(ux.astype(np.float64), uy.astype(np.float64), rx, ry)
    print(f"\n[Taylor-Green box, N {N}, circle {circle}, {K} steps] velocity vs FP64 {e:.2e}")
    assert e <= max(1e-5, K * 2.0 ** -24)
    if circle:
        m = lat.markers(0)
        d = sim.marker_diag(0)
        assert np.abs(m["Usx"] - d["Usx"]).max() <= 1e-5 * tg.u0


def test_second_order_convergence():
    rows = []
    for N in (10, 20, 40, 80):
        tg, lat, b, K = gpu_run(N)
        _, ux, uy = lat.moments()
        X, Y = tg.coords()
        ax, ay = tg.velocity(X, Y, K)
        e = rel(ux.astype(np.float64), uy.astype(np.float64), ax, ay)
        m = lat.markers(0)                       # D_I u* of the last step (time K-1)
        bx, by = tg.marker_velocity(b, K - 1)
        eb = rel(m["Usx"].astype(np.float64), m["Usy"].astype(np.float64), bx, by)
        rows.append((N, e, eb))
    slopes = [(math.log2(a[1] / c[1]), math.log2(a[2] / c[2])) for a, c in zip(rows[:-1], rows[1:])]
    print("\n[Taylor-Green with circle, T = 1] " + "; ".join(f"N {n}: overall {e:.2e}, boundary {eb:.2e}"
                                                         for n, e, eb in rows)
          + " | slopes " + ", ".join(f"{a:.2f}/{b:.2f}" for a, b in slopes))
    for a, b in slopes:
        assert 1.7 < a < 2.4 and b > 1.7
