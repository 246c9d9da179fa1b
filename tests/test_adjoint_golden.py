"""The stored finite-difference gradients of the FP64 oracle
(tests/golden/adjoint_fd_cyl160x80.json, written by make_adjoint_fd.py) that
the GPU adjoint is compared with.

* They are reproduced by the oracle as it stands: the window-averaged drag
  coefficient and its central difference in U for the 100-step window from
  the initial fields.
* The cylinder sits on the channel's centre line and the initial noise is
  1e-4, so the flow is mirror-symmetric about y = 40 up to that noise: the
  sensitivity to the radial offset of marker l (angle t) equals that of the
  marker at -t.
* dJ/dU differs from the pure normalization term -2 J / U: the inflow speed
  also acts through the inlet extrapolation, and the stored value carries
  that part.
"""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "adjoint_fd_cyl160x80.json")))


def _maker():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "make_adjoint_fd", os.path.join(HERE, "golden", "make_adjoint_fd.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def window(name):
    return next(w for w in GOLD["windows"] if w["name"] == name)


def test_stored_values_reproduced_by_oracle():
    O.build()
    O.set_threads(1)
    m = _maker()
    case = m.base_case()
    w = window("init")
    n = GOLD["markers"]
    J = m.window_J(case, case.u_in, np.zeros(n), None, w["nsteps"])
    assert abs(J / w["J"] - 1.0) < 1e-12
    eps = GOLD["eps"]
    jp = m.window_J(case, case.u_in + eps, np.zeros(n), None, w["nsteps"])
    jm = m.window_J(case, case.u_in - eps, np.zeros(n), None, w["nsteps"])
    assert abs((jp - jm) / (2 * eps) / w["dJdU"] - 1.0) < 1e-9


@pytest.mark.parametrize("name,tol", [("init", 2e-3), ("spun_up", 5e-2)])
def test_radial_sensitivity_mirror_symmetric(name, tol):
    g = np.asarray(window(name)["dJddr"])
    n = len(g)
    mirror = g[(-np.arange(n)) % n]
    assert np.abs(g - mirror).max() <= tol * np.abs(g).max()


@pytest.mark.parametrize("name", ["init", "spun_up"])
def test_inflow_sensitivity_includes_inlet_path(name):
    w = window(name)
    norm_only = -2.0 * w["J"] / GOLD["u_in"]
    assert abs(w["dJdU"] - norm_only) > 1e-2 * abs(norm_only)
    assert abs(w["dJdU_2eps"] / w["dJdU"] - 1.0) < 1e-4


def test_apply_inlet_is_the_inlet_rule_of_the_step():
    """Re-applying the inlet rule to a state the same simulation just
    streamed changes nothing; with another inlet speed only column 0 changes."""
    O.build()
    m = _maker()
    case = m.base_case()
    s = O.Sim.from_case(case)
    s.step(20)
    f = s.pops()
    s.apply_inlet()
    assert np.array_equal(s.pops(), f)
    t = O.Sim(case.nx, case.ny, case.tau, case.u_in + 0.01, case.bc_x, case.bc_y, 0.0, 0.0,
              case.delta, case.nf)
    t.set_pops(f)
    t.apply_inlet()
    g = t.pops()
    assert np.array_equal(g[:, 1:], f[:, 1:]) and not np.array_equal(g[:, 0], f[:, 0])
    _, ux, _ = t.moments()
    assert np.allclose(ux[:, 0], case.u_in + 0.01, rtol=0, atol=1e-12)

