"""Host-side metrics the benchmark reports, on the CPU: the two-body elements
of the black-hole pair and the momentum drift."""
import numpy as np
import pytest

import bench
from paper_1312_1789_b300 import ics


@pytest.mark.parametrize("a,e", [(0.05, 0.5), (0.1, 0.0), (0.02, 0.9)])
def test_binary_elements_of_a_keplerian_pair(a, e):
    m, x, v = ics.bh_binary(0.01, a, e)
    S = {"x": np.vstack([np.zeros((3, 3)), x]), "v": np.vstack([np.zeros((3, 3)), v])}
    got_a, got_e = bench.binary_elements(S, np.concatenate([np.ones(3), m]))
    assert got_a == pytest.approx(a, rel=1e-12)
    # e = sqrt(1 + 2 E h^2 / mu^2): near e = 0 the square root turns a rounding
    # of the bracket (~1e-16) into ~1e-8
    assert got_e == pytest.approx(e, abs=1e-7)


def test_momentum_drift():
    rng = np.random.default_rng(3)
    m = rng.uniform(0.5, 1.5, 50)
    S0 = {"v": rng.normal(size=(50, 3))}
    assert bench.momentum_drift(S0, S0, m) == 0.0
    S1 = {"v": S0["v"].copy()}
    S1["v"][7] += np.array([1e-3, 0.0, 0.0])
    expect = m[7] * 1e-3 / (m * np.linalg.norm(S0["v"], axis=1)).sum()
    assert bench.momentum_drift(S0, S1, m) == pytest.approx(expect, rel=1e-9)
