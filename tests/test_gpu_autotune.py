"""The native autotuners (btdf_autotune, btdf_batch_autotune) and the
launch-shape cache: tuning picks a timed variant, and leaves the simulation
exactly where it was (populations, step counter, force history, the last
step's marker results), so a tuned run equals an untuned one bit for bit."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1806_09403_gb300 import _build  # noqa: E402
from paper_1806_09403_gb300 import autotune as T  # noqa: E402
from paper_1806_09403_gb300 import btdf as B  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()


@pytest.mark.parametrize("first", [0, 37])
def test_autotune_leaves_the_run_unchanged(first):
    case = W.small_cylinder(delta=3)
    a = B.Lattice.from_case(case, history_len=256)
    b = B.Lattice.from_case(case, history_len=256)
    a.step(first)
    b.step(first)
    mk = a.markers(0)
    chosen, ms = a.autotune(steps=3, flush_l2=(first == 0))
    assert 1 <= chosen < B.VARIANT_COUNT and chosen in ms and all(t > 0 for t in ms.values())
    assert ms[chosen] == min(ms.values())
    assert a.steps == first
    if first:
        for k, v in a.markers(0).items():
            assert np.array_equal(v, mk[k])
    a.step(150)
    b.step(150)
    for kind in (B.FIELD_RHO, B.FIELD_UX, B.FIELD_UY):
        assert np.array_equal(a.field(kind), b.field(kind))
    fa, fb = a.forces(0, 0, first + 150), b.forces(0, 0, first + 150)
    assert np.array_equal(fa[0], fb[0]) and np.array_equal(fa[1], fb[1])


def test_batch_autotune_leaves_the_run_unchanged():
    cases = [W.small_cylinder(delta=3), W.small_cylinder(delta=3, seed=9)]
    a = B.Batch.from_cases(cases, history_len=128)
    b = B.Batch.from_cases(cases, history_len=128)
    a.step(20)
    b.step(20)
    chosen, ms = a.autotune(steps=3)
    assert chosen in (1, 2, 3, 4) and all(t > 0 for t in ms.values())
    a.step(80)
    b.step(80)
    for i in range(2):
        assert np.array_equal(a.field(i, B.FIELD_UX), b.field(i, B.FIELD_UX))
        assert np.array_equal(a.forces(i, 0, 100)[0], b.forces(i, 0, 100)[0])


def test_cache_round_trip(tmp_path):
    case = W.small_cylinder(delta=3)
    lat = B.Lattice.from_case(case)
    cache = T.TuneCache(str(tmp_path / "t.json"))
    e1 = T.tune_lattice(lat, cache, steps=2, flush_l2=False)
    e2 = T.tune_lattice(lat, T.TuneCache(str(tmp_path / "t.json")))
    assert not e1["cached"] and e2["cached"] and e1["variant"] == e2["variant"]
