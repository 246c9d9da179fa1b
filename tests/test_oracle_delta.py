"""Pins of the oracle's regularized delta functions (Sec. 4.3, Eqs. 37-39).

The kernels are pinned by the discrete identities they were built to satisfy
(partition of unity, vanishing first moment, constant sum of squares, even/odd
split of the 4-point kernel), by closed-form values at integer offsets, by
continuity at their branch points and by their support width (Sec. 4.3 gives
drf/dh = 2, 3, 4).  A wrong coefficient or sign inside any branch breaks at
least one of these.
"""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
R = np.linspace(-0.5, 0.5, 1001)


def _sum(kind, r, power=1, moment=0, parity=None):
    acc = 0.0
    for j in range(-4, 5):
        if parity is not None and (j % 2) != parity:
            continue
        d = O.delta(kind, r - j)
        acc += (r - j) ** moment * d ** power
    return acc


@pytest.mark.parametrize("kind", [2, 3, 4, 5])
def test_partition_of_unity(kind):
    for r in R:
        assert abs(_sum(kind, r) - 1.0) < 1e-14


@pytest.mark.parametrize("kind", [2, 3, 4])
def test_first_moment_vanishes(kind):
    for r in R:
        assert abs(_sum(kind, r, moment=1)) < 1e-14


def test_cosine_kernel_first_moment_nonzero():
    # The cosine kernel is not in the paper; it reproduces constants but not
    # linear fields, unlike Eqs. 37-39.
    m = max(abs(_sum(5, r, moment=1)) for r in R)
    assert 0.01 < m < 0.05


@pytest.mark.parametrize("kind,val", [(3, 0.5), (4, 3.0 / 8.0), (5, 3.0 / 8.0)])
def test_sum_of_squares_constant(kind, val):
    for r in R:
        assert abs(_sum(kind, r, power=2) - val) < 1e-14


def test_four_point_even_odd_split():
    for r in R:
        assert abs(_sum(4, r, parity=0) - 0.5) < 1e-14
        assert abs(_sum(4, r, parity=1) - 0.5) < 1e-14


def test_integer_values():
    assert O.delta(2, 0.0) == 1.0 and O.delta(2, 0.5) == 0.5
    assert abs(O.delta(3, 0.0) - 2.0 / 3.0) < 1e-15
    assert abs(O.delta(3, 1.0) - 1.0 / 6.0) < 1e-15
    assert abs(O.delta(4, 0.0) - 0.5) < 1e-15
    assert abs(O.delta(4, 1.0) - 0.25) < 1e-15
    assert abs(O.delta(5, 0.0) - 0.5) < 1e-15
    assert abs(O.delta(5, 1.0) - 0.25) < 1e-15


@pytest.mark.parametrize("kind", [2, 3, 4, 5])
def test_support_and_symmetry(kind):
    half = GOLD["delta_support_over_dh"].get(str(min(kind, 4)), 4.0) / 2.0
    assert O.lib().oracle_support_width(kind) == int(2 * half)
    for r in np.linspace(0, 3, 301):
        assert O.delta(kind, r) == O.delta(kind, -r)
        if r >= half:
            assert O.delta(kind, r) == 0.0
        elif r < half - 1e-9:
            assert O.delta(kind, r) > 0.0


@pytest.mark.parametrize("kind,points", [(3, [0.5, 1.5]), (4, [1.0, 2.0]), (2, [1.0]), (5, [2.0])])
def test_continuity_at_branch_points(kind, points):
    for p in points:
        lo, hi = O.delta(kind, p - 1e-12), O.delta(kind, p + 1e-12)
        assert abs(lo - hi) < 1e-6


def test_paper_thickness_constants():
    for k in (2, 3, 4):
        assert O.drs_paper(k) == GOLD["drs_over_dh"][str(k)]
