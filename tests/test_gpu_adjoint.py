"""The discrete adjoint (btdf_adjoint_forward / btdf_adjoint_backward) and
its torch.autograd.Function.

Objective: the drag coefficient averaged over a window of steps,
J = mean Fx / (U^2 D / 2).  Gradients with respect to the inflow speed U and
the radial offsets dr_l of the markers.

* 160 x 80 cylinder (D = 16, 50 markers, Re = 40, 4-point cosine delta):
  the FP32 adjoint against central differences (eps = 1e-4) of the FP64
  oracle stored in tests/golden/adjoint_fd_cyl160x80.json, for a 100-step
  window from the initial fields (first step in place) with a checkpoint
  every 30 steps (a ragged last segment) and a 500-step window after 300
  steps with a checkpoint every 50.  Bar: 1e-3 relative, for dJ/dU, for the
  vector dJ/d dr (norm-wise) and for each component against the largest.
* 800 x 400 cylinder (D = 24, 76 markers, Re = 100, 3-point delta), 500-step
  window after 2000 steps with a checkpoint every 50: the adjoint against
  central differences of the FP32 forward itself, for U and for the radial
  offsets along one random direction.  FP32 rounding makes those differences
  noisy where the step changes J by only a few ulps, so this comparison is
  indicative; a larger step is reported beside eps = 1e-4.
* The gradients do not depend on the checkpoint spacing.
"""
import json
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1806_09403_gb300 import _build  # noqa: E402
from paper_1806_09403_gb300 import btdf as B  # noqa: E402
from paper_1806_09403_gb300.autograd import CdWindow, DragWindow  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "adjoint_fd_cyl160x80.json")))
TOL = 1e-3


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()


def small_window(name, every):
    w = next(x for x in GOLD["windows"] if x["name"] == name)
    case = W.small_cylinder(delta=5)
    lat = B.Lattice.from_case(case, history_len=1024)
    if w["t0"]:
        lat.step(w["t0"])
    win = DragWindow.for_lattice(lat, 40.0, 40.0, 0.5 * case.D, w["nsteps"], every=every, dref=case.D)
    return case, w, win


def rel(a, b):
    return abs(a / b - 1.0)


@pytest.mark.parametrize("name,every", [("init", 30), ("spun_up", 50)])
def test_adjoint_against_fp64_finite_differences(name, every):
    case, w, win = small_window(name, every)
    n = GOLD["markers"]
    U = torch.tensor(case.u_in, dtype=torch.float64, requires_grad=True)
    dr = torch.zeros(n, dtype=torch.float64, requires_grad=True)
    J = CdWindow.apply(U, dr, win)
    J.backward()
    g = dr.grad.numpy()
    ref = np.asarray(w["dJddr"])
    e_J = rel(float(J), w["J"])
    e_U = rel(float(U.grad), w["dJdU"])
    e_dr = float(np.linalg.norm(g - ref) / np.linalg.norm(ref))
    e_c = float(np.abs(g - ref).max() / np.abs(ref).max())
    print(f"\n[{name}, every {every}] J {float(J):.8f} (FP64 {w['J']:.8f}, {e_J:.1e}); "
          f"dJ/dU {float(U.grad):.6e} (FD {w['dJdU']:.6e}, {e_U:.1e}); "
          f"dJ/d dr rel L2 {e_dr:.1e}, max component {e_c:.1e}")
    assert e_J <= 1e-4
    assert e_U <= TOL
    assert e_dr <= TOL and e_c <= TOL


def test_gradients_do_not_depend_on_checkpoint_spacing():
    case, w, win = small_window("init", 7)
    z = np.zeros(GOLD["markers"])
    J7 = win.evaluate(case.u_in, z)
    dU7, g7 = win.gradients(case.u_in, z)
    win.every = 100
    J1 = win.evaluate(case.u_in, z)
    dU1, g1 = win.gradients(case.u_in, z)
    assert J7 == J1
    assert np.array_equal(g7, g1)
    assert rel(dU7, dU1) < 1e-12       # the inlet part is summed with double atomics


def test_window_leaves_context_state_alone():
    case, w, win = small_window("init", 30)
    before = win.lattice.field(B.FIELD_UX)
    steps = win.lattice.steps
    win.evaluate(case.u_in, np.zeros(GOLD["markers"]))
    win.gradients(case.u_in, np.zeros(GOLD["markers"]))
    assert win.lattice.steps == steps
    assert np.array_equal(win.lattice.field(B.FIELD_UX), before)


def test_adjoint_rejects_unsupported_configurations():
    case = W.small_cylinder(delta=5)
    lat = B.Lattice.from_case(case, storage=B.BTDF_F16DEV)
    with pytest.raises(B.BtdfError):
        lat.adjoint_forward(10, 5, 0, 16.0)
    lat = B.Lattice.from_case(case)
    with pytest.raises(B.BtdfError):
        lat.adjoint_backward()                      # no forward window yet
    lat.adjoint_forward(10, 5, 0, 16.0)
    lat.set_inflow(0.04)
    with pytest.raises(B.BtdfError):
        lat.adjoint_backward()                      # invalidated by the new inflow
    c2 = W.small_cylinder(delta=5)
    c2.bodies[0].X = c2.bodies[0].X - 31.0          # support reaches the inlet column
    lat2 = B.Lattice.from_case(c2)
    with pytest.raises(B.BtdfError):
        lat2.adjoint_forward(10, 5, 0, 16.0)


def test_adjoint_800x400_against_fp32_finite_differences():
    case = W.adjoint_cylinder()
    lat = B.Lattice.from_case(case, history_len=1024)
    lat.step(2000)
    n = len(case.bodies[0].X)
    win = DragWindow.for_lattice(lat, 200.0, 200.0, 0.5 * case.D, 500, every=50, dref=case.D)
    z = np.zeros(n)
    J0 = win.evaluate(case.u_in, z)
    dU, g = win.gradients(case.u_in, z)
    v = np.random.default_rng(11).standard_normal(n)
    dirn = float(g @ v)
    eU, ev = {}, {}
    for eps in (1e-4, 1e-3):
        fdU = (win.evaluate(case.u_in + eps, z) - win.evaluate(case.u_in - eps, z)) / (2 * eps)
        eU[eps] = rel(dU, fdU)
        print(f"\n[800x400] J {J0:.6f}; dJ/dU adjoint {dU:.6e}, FD eps {eps:g} {fdU:.6e} ({eU[eps]:.1e})")
    for eps in (1e-4, 1e-2):
        fdv = (win.evaluate(case.u_in, eps * v) - win.evaluate(case.u_in, -eps * v)) / (2 * eps)
        ev[eps] = rel(dirn, fdv)
        print(f"[800x400] dJ/d dr along a random direction: adjoint {dirn:.6e}, FD eps {eps:g} "
              f"{fdv:.6e} ({ev[eps]:.1e})")
    # eps = 1e-4 in U changes J by ~6e-3 relative: well above FP32 noise
    assert eU[1e-4] <= TOL
    # a marker offset of 1e-4 changes J by ~1e-5 relative, ~100 FP32 ulps:
    # the difference quotient carries ~1e-3 noise, so the larger step decides
    assert ev[1e-2] <= 5e-3 and ev[1e-4] <= 2e-2
