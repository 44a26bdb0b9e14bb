"""Pins for the Philox4x32-10 generator: published known-answer vectors and
the distribution of the derived uniforms."""
import os

import numpy as np
import scipy.stats as stats

from oracle.philox import philox4x32, uniform

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def test_known_answer_vectors():
    rows = [l.split() for l in open(GOLD) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert philox4x32(v[0:4], v[4:6]) == tuple(v[6:10])


def test_uniform_exact_open_interval():
    for d in range(50):
        u = uniform(12345, 7, d)
        assert 0.0 < u < 1.0
        x = u * 2.0 ** 52 - 0.5
        assert x == int(x)


def test_uniform_distribution_and_independence():
    u = np.array([uniform(1, j, 0) for j in range(4000)] + [uniform(1, 0, d) for d in range(4000)])
    assert stats.kstest(u, "uniform").pvalue > 1e-4
    a = np.array([uniform(99, j, 0) for j in range(3000)])
    b = np.array([uniform(99, j, 1) for j in range(3000)])
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.08
    assert uniform(1, 0, 0) != uniform(2, 0, 0)
    assert uniform(1 << 40, 0, 0) != uniform(0, 0, 0)
