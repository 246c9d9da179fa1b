"""The batched form: many independent lattices in one IB launch and one
persistent collide-stream launch per step.

Each lattice of a batch must compute exactly what a single context computes
for the same case (bitwise: the same kernels run the same arithmetic), and
therefore match the FP64 oracle like the single-lattice path does.
"""
import os

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
    O.set_threads(min(os.cpu_count() or 1, 32))


def mixed_cases():
    cases = []
    for i, (nx, ny, re, d) in enumerate([(96, 48, 40.0, 10.0), (130, 70, 200.0, 12.0),
                                         (200, 100, 0.1, 16.0), (64, 40, 40.0, 8.0),
                                         (257, 96, 100.0, 14.0)]):
        c = W.Case(f"m{i}", nx, ny, W.tau_from_re(re, W.U_IN, d), W.U_IN, 3, W.BCX_INOUT,
                   W.BCY_FREESLIP, seed=40 + i, Re=re, D=d)
        c.bodies.append(W.circle_markers(nx / 4 + 0.3, ny / 2 + 0.2, d, int(round(np.pi * d))))
        cases.append(c)
    # a periodic box without bodies and a no-slip channel with two bodies
    p = W.Case("box", 48, 36, 0.8, 0.02, 3, W.BCX_PERIODIC, W.BCY_PERIODIC, seed=50, noise=1e-3)
    cases.append(p)
    q = W.Case("two", 150, 60, 0.7, 0.03, 3, W.BCX_PERIODIC, W.BCY_NOSLIP, seed=51, D=8.0)
    q.bodies.append(W.circle_markers(40.2, 30.1, 8.0, 25))
    q.bodies.append(W.circle_markers(100.7, 25.3, 8.0, 25))
    cases.append(q)
    return cases


@pytest.mark.parametrize("variant", [1, 2, 3, 4])
def test_batch_matches_single_contexts_bitwise(variant):
    cases = mixed_cases()
    bt = B.Batch.from_cases(cases, history_len=300)
    bt.tune(variant)
    bt.step(200)
    bt.sync()
    body = 0
    for i, c in enumerate(cases):
        lat = B.Lattice.from_case(c, history_len=300)
        lat.step(200)
        for kind in (B.FIELD_RHO, B.FIELD_UX, B.FIELD_UY):
            assert np.array_equal(bt.field(i, kind), lat.field(kind)), (c.name, kind)
        for j in range(len(c.bodies)):
            gx, gy = bt.forces(body)
            rx, ry = lat.forces(j)
            assert np.array_equal(gx, rx) and np.array_equal(gy, ry), (c.name, j)
            body += 1
        lat.close()


def test_batch_against_oracle():
    cases = mixed_cases()
    bt = B.Batch.from_cases(cases, history_len=300)
    bt.step(300)
    body = 0
    for i, c in enumerate(cases):
        sim = O.Sim.from_case(c)
        sim.step(300)
        _, ux, uy = sim.moments()
        gx_, gy_ = bt.field(i, B.FIELD_UX), bt.field(i, B.FIELD_UY)
        e = np.sqrt((((gx_ - ux) ** 2 + (gy_ - uy) ** 2).sum()) / ((ux ** 2 + uy ** 2).sum()))
        assert e <= max(1e-5, 300 * 2.0 ** -24), (c.name, e)
        for j in range(len(c.bodies)):
            fx, _ = bt.forces(body)
            rx, _ = sim.history(j)
            scale = np.abs(rx).mean()
            assert (np.abs(fx - rx) / np.maximum(np.abs(rx), scale)).max() <= 1e-4, (c.name, j)
            body += 1


def test_batch_graph_replay_and_fp16():
    cases = mixed_cases()[:3]
    a = B.Batch.from_cases(cases, storage=B.BTDF_F16DEV)
    b = B.Batch.from_cases(cases, storage=B.BTDF_F16DEV)
    a.step(100)               # 1 local step, 3 graphs of 32, 3 direct
    for _ in range(100):
        b.step(1)
    for i in range(len(cases)):
        assert np.array_equal(a.field(i, B.FIELD_UX), b.field(i, B.FIELD_UX))
