"""Pins for the Runge-Kutta tableaus: every rooted-tree order condition
(Butcher) up to order 5 for the propagating weights b and up to order 4 for
the embedded weights bhat, the row-sum condition, and the observed
convergence order of the integrator."""
from fractions import Fraction

import numpy as np
import pytest

from oracle.integrate import integrate
from oracle.tableau import DP5, TSIT5


def _trees(order):
    """All rooted trees with `order` nodes; a tree is the sorted tuple of its
    children (a leaf is ())."""
    if order == 1:
        return [()]
    out = set()

    def grow(t):
        # attach a new leaf at every node of t
        res = [tuple(sorted(t + ((),)))]
        for i, ch in enumerate(t):
            for g in grow(ch):
                res.append(tuple(sorted(t[:i] + (g,) + t[i + 1:])))
        return res

    for t in _trees(order - 1):
        out.update(grow(t))
    return sorted(out)


def _size(t):
    return 1 + sum(_size(c) for c in t)


def _density(t):
    g = _size(t)
    for c in t:
        g *= _density(c)
    return g


def _weights(t, a, one):
    """Vector g_i(t) = prod_children sum_j a_ij g_j(child)."""
    s = len(a)
    v = [one] * s
    for ch in t:
        gc = _weights(ch, a, one)
        av = [sum((a[i][j] * gc[j] for j in range(s)), one * 0) for i in range(s)]
        v = [v[i] * av[i] for i in range(s)]
    return v


def _check(b, a, order, one, tol):
    bad = []
    for p in range(1, order + 1):
        for t in _trees(p):
            phi = sum((bi * gi for bi, gi in zip(b, _weights(t, a, one))), one * 0)
            target = one / _density(t)
            if abs(phi - target) > tol:
                bad.append((t, float(phi), float(target)))
    return bad


def test_tree_counts():
    assert [len(_trees(p)) for p in range(1, 6)] == [1, 1, 2, 4, 9]


def test_dp5_exact_order_conditions():
    c, a, b, bhat = DP5.exact
    one = Fraction(1)
    assert _check(b, a, 5, one, 0) == []
    assert _check(bhat, a, 4, one, 0) == []
    # the embedded pair must genuinely differ at order 5 (else no error estimate)
    assert _check(bhat, a, 5, one, 0) != []
    for i in range(7):
        assert sum(a[i]) == c[i]


def test_tsit5_order_conditions():
    a = [list(r) for r in TSIT5.a]
    assert _check(list(TSIT5.b), a, 5, 1.0, 5e-14) == []
    assert _check(list(TSIT5.bhat), a, 4, 1.0, 5e-14) == []
    assert _check(list(TSIT5.bhat), a, 5, 1.0, 5e-14) != []
    for i in range(7):
        assert abs(sum(TSIT5.a[i]) - TSIT5.c[i]) < 2e-15
    assert np.allclose(TSIT5.a[6][:6], TSIT5.b[:6]) and TSIT5.b[6] == 0.0


@pytest.mark.parametrize("tab", [DP5, TSIT5], ids=["dp5", "tsit5"])
def test_convergence_order_five(tab):
    """Fixed-step error on y' = lam y and on a 2x2 rotation halves by 2^5."""
    lam = -0.7 + 2.0j
    M = np.array([[0.0, 1.0], [-1.0, 0.0]], dtype=np.complex128)

    def run(f, y0, h, T=2.0):
        out = {}
        integrate(f, y0, np.array([0.0, T]), tab, 1e-8, 1e-10,
                  lambda i, t, y: out.__setitem__(i, y.copy()), fixed_dt=h)
        return out[1]

    for f, y0, exact in [
        (lambda t, y: lam * y, np.array([1.0 + 0.5j]), np.array([(1.0 + 0.5j) * np.exp(lam * 2.0)])),
        (lambda t, y: M @ y, np.array([1.0, 0.0], dtype=np.complex128),
         np.array([np.cos(2.0), -np.sin(2.0)], dtype=np.complex128)),
    ]:
        # Tsit5's leading error constant is small, so its ratio reaches 2^5
        # from above only for small h; order 4 would give 16, order 6 64.
        e1 = np.max(np.abs(run(f, y0, 0.04) - exact))
        e2 = np.max(np.abs(run(f, y0, 0.02) - exact))
        ratio = e1 / e2
        assert 26 < ratio < 46, ratio
