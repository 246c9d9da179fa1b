"""Writes adjoint_fd_cyl160x80.json: central finite differences of the
window-averaged drag coefficient of the FP64 oracle on the 160 x 80 cylinder
(D = 16, 50 markers, Re = 40, 4-point cosine delta), with respect to the
inflow speed U and every marker's radial offset dr_l.

    J(U, dr) = (1 / N) sum_{n < N} Fx^n / (U^2 D / 2)

over the N steps that follow a fixed start state: the initial fields
(window "init", N = 100, the first step reads the initial populations in
place) or the post-collision state after 300 steps at the base parameters
(window "spun_up", N = 500).  In the second window the streaming that
follows that state, inlet rule included, belongs to the window: the oracle
holds post-streaming populations, so the inlet column of the loaded state
is re-derived with the perturbed U before stepping.  tau, ds and drs are
held fixed.  eps = 1e-4; dJ/dU is also taken with 2 eps so that the
truncation error can be checked.

Only the oracle and the seeded input generators are used.  Run from the
repository root:  python tests/golden/make_adjoint_fd.py
"""
from __future__ import annotations

import json
import math
import multiprocessing as mp
import os
import sys
from concurrent.futures import ProcessPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import oracle as O  # noqa: E402

EPS = 1e-4
WINDOWS = [("init", 0, 100), ("spun_up", 300, 500)]
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "adjoint_fd_cyl160x80.json")


def base_case():
    return W.small_cylinder(delta=5)


def geometry(case):
    b = case.bodies[0]
    n = len(b.X)
    theta = 2.0 * np.pi * np.arange(n) / n
    return 40.0, 40.0, 0.5 * case.D, theta, b.ds


def window_J(case, u, dr, start, nsteps):
    """Window-averaged Cd of the oracle from `start` (None: initial fields)."""
    cx, cy, R, theta, ds = geometry(case)
    s = O.Sim(case.nx, case.ny, case.tau, u, case.bc_x, case.bc_y, case.gx, case.gy,
              case.delta, case.nf)
    rho, ux, uy = case.initial_fields()
    s.init_fields(rho, ux, uy)
    if start is not None:
        s.set_pops(start)
        s.apply_inlet()
    r = R + np.asarray(dr)
    s.add_body(cx + r * np.cos(theta), cy + r * np.sin(theta), ds, drs=case.drs)
    s.step(nsteps)
    fx, _ = s.history(0)
    return float(np.mean(fx) / (0.5 * u * u * case.D))


def _job(args):
    O.set_threads(1)
    kind, idx, sign, h, start, nsteps = args
    case = base_case()
    n = len(case.bodies[0].X)
    u = case.u_in
    dr = np.zeros(n)
    if kind == "U":
        u += sign * h
    elif kind == "dr":
        dr[idx] += sign * h
    return (kind, idx, sign, h), window_J(case, u, dr, start, nsteps)


def spun_up_state(case, t0):
    s = O.Sim.from_case(case)
    s.step(t0)
    return s.pops()


def main():
    O.build()
    case = base_case()
    n = len(case.bodies[0].X)
    out = {"case": case.name, "delta": case.delta, "tau": case.tau, "u_in": case.u_in,
           "D": case.D, "markers": n, "eps": EPS, "windows": []}
    workers = max(1, (os.cpu_count() or 1))
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as pool:
        for name, t0, nsteps in WINDOWS:
            start = spun_up_state(case, t0) if t0 > 0 else None
            jobs = [("base", 0, 0, 0.0, start, nsteps)]
            for sign in (1, -1):
                jobs.append(("U", 0, sign, EPS, start, nsteps))
                jobs.append(("U", 0, sign, 2 * EPS, start, nsteps))
                jobs += [("dr", l, sign, EPS, start, nsteps) for l in range(n)]
            res = dict(pool.map(_job, jobs))
            J = res[("base", 0, 0, 0.0)]
            dU = (res[("U", 0, 1, EPS)] - res[("U", 0, -1, EPS)]) / (2 * EPS)
            dU2 = (res[("U", 0, 1, 2 * EPS)] - res[("U", 0, -1, 2 * EPS)]) / (4 * EPS)
            ddr = [(res[("dr", l, 1, EPS)] - res[("dr", l, -1, EPS)]) / (2 * EPS) for l in range(n)]
            # The central difference's truncation error is O(eps^2); with
            # J ~ 1 / U^2 its relative size is about 2 eps^2 / U^2 = 8e-6 at
            # eps = 1e-4, four times that at 2 eps: far below the 1e-3 bar.
            assert abs(dU2 / dU - 1.0) < 1e-4, (name, dU, dU2)
            out["windows"].append({"name": name, "t0": t0, "nsteps": nsteps, "J": J, "dJdU": dU,
                                   "dJdU_2eps": dU2, "dJddr": ddr})
            print(f"{name}: J {J:.10f} dJ/dU {dU:.8e} (2 eps {dU2:.8e}) "
                  f"|dJ/ddr| {math.sqrt(sum(x * x for x in ddr)):.6e}")
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
