"""GPU stationary states (qtl_steadystate, qtl_steadystate_fourier) through
the C ABI against the oracle's direct solves (Sec. 3.2, Appendix A), the
driven cavity's coherent steady state (Sec. 5), and the edge cases."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle.steadystate import steadystate as o_ss
from oracle.steadystate import steadystate_fourier as o_ssf
from tests.gpu_util import maxabs, require_gpu

pytestmark = pytest.mark.gpu


def destroy(N):
    return sp.diags(np.sqrt(np.arange(1, N)), 1, format="csr", dtype=complex)


def _kerr(N=30, D=0.5, K=0.2, F=1.0, kap=0.1):
    s = W.kerr_cavity(N, D, K, F, kap)
    return s.H, s.c_ops


@pytest.mark.parametrize("name", ["cavity40", "jc40x2", "kerr30"])
def test_steadystate_matches_the_direct_solve(name):
    qtl = require_gpu()
    if name == "cavity40":
        s = W.driven_cavity(N=40)
        H, c = s.H, s.c_ops
    elif name == "jc40x2":
        s = W.jaynes_cummings(N=40)
        H, c = s.H, s.c_ops
    else:
        H, c = _kerr()
    ref = o_ss(H, c)
    g = qtl.System(H, c, [])
    try:
        got = g.steadystate()
    finally:
        g.free()
    assert maxabs(got["rho"], ref) <= 1e-10
    assert got["stats"]["residual"] <= 1e-11
    assert abs(np.trace(got["rho"]) - 1) <= 1e-12
    assert got["stats"]["iterations"] <= 200


def test_driven_cavity_coherent_steady_state():
    """<a> = -i F / (k/2 + i D) and n = F^2 / (D^2 + k^2/4) (Sec. 5) at N = 40."""
    qtl = require_gpu()
    N, D, F, kap = 40, 1.0, 0.5, 0.2
    a = destroy(N)
    ad = a.conj().T
    g = qtl.System(D * (ad @ a) + F * (a + ad), [math.sqrt(kap) * a], [])
    try:
        rho = g.steadystate()["rho"]
    finally:
        g.free()
    assert abs(np.trace(a @ rho) - (-1j * F / (kap / 2 + 1j * D))) <= 1e-11
    assert abs(np.trace(ad @ a @ rho) - F ** 2 / (D ** 2 + kap ** 2 / 4)) <= 1e-11
    assert np.max(np.abs(rho - rho.conj().T)) <= 1e-11


def test_fourier_components_match_the_direct_solve():
    """A driven Kerr cavity under F cos(w t)(a + a'): every Fourier component
    rho_k, |k| <= 4, against the oracle's block-tridiagonal direct solve."""
    qtl = require_gpu()
    N = 20
    a = destroy(N)
    ad = a.conj().T
    H0 = 0.3 * (ad @ a) + 0.1 * (ad @ ad @ a @ a)
    c = [math.sqrt(0.2) * a]
    X = a + ad
    ref = o_ssf(H0, c, X, 0.8, 1.0, 4)
    g = qtl.System(H0, c, [])
    try:
        got = g.steadystate_fourier(X, 0.8, 1.0, 4)
    finally:
        g.free()
    for k in range(-4, 5):
        assert maxabs(got["rho"][k], ref[k]) <= 1e-9
    assert abs(np.trace(got["rho"][0]) - 1) <= 1e-12


def test_fourier_cos_driven_cavity_closed_form():
    """The cos-driven damped cavity: <a> has only the k = +-1 components
    A+- = -i (F/2) / (i D + k/2 +- i w) (the exact periodic coherent state)."""
    qtl = require_gpu()
    N, D, kap, F, w = 30, 0.7, 0.5, 0.2, 1.1
    a = destroy(N)
    ad = a.conj().T
    g = qtl.System(D * (ad @ a), [math.sqrt(kap) * a], [])
    try:
        comps = g.steadystate_fourier(a + ad, F, w, 4)["rho"]
    finally:
        g.free()
    z = 1j * D + kap / 2
    assert abs(np.trace(a @ comps[1]) - (-0.5j * F / (z + 1j * w))) <= 1e-10
    assert abs(np.trace(a @ comps[-1]) - (-0.5j * F / (z - 1j * w))) <= 1e-10
    assert abs(np.trace(a @ comps[0])) <= 1e-10


def test_steadystate_edge_cases():
    qtl = require_gpu()
    s = W.driven_cavity(N=10)
    g = qtl.System(s.H, s.c_ops, [])
    try:
        # a budget of two products cannot reach 1e-12: QTL_ESTEP, iterate still returned
        with pytest.raises(qtl.QtlError) as e:
            g.steadystate(max_iter=2)
        assert e.value.status == qtl.QTL_ESTEP
        with pytest.raises(qtl.QtlError) as e:
            g.steadystate(restart=0)
        assert e.value.status == qtl.QTL_EINVAL
        with pytest.raises(qtl.QtlError) as e:
            g.steadystate_fourier(np.eye(10), 0.1, 1.0, 65)
        assert e.value.status == qtl.QTL_EINVAL
        # a second call reuses the preconditioner and gives the same state
        r1 = g.steadystate()["rho"]
        r2 = g.steadystate()["rho"]
        assert maxabs(r1, r2) == 0.0
    finally:
        g.free()
    big = qtl.System(sp.identity(1025, dtype=complex, format="csr"), [], [])
    try:
        with pytest.raises(qtl.QtlError) as e:
            big.steadystate()
        assert e.value.status == qtl.QTL_ETOOBIG
    finally:
        big.free()


def test_steadystate_beyond_the_cluster_kernel_capacity():
    """A Kerr cavity at N = 132 (17,424 unknowns, above the 16,384 rows the
    cluster mesolve kernel holds) in FP64 and with the split-BF16
    preconditioner; the system's mesolve afterwards still refuses the cluster
    engine and runs on the grid engine."""
    qtl = require_gpu()
    H, c = _kerr(N=132, D=0.5, K=0.02, F=1.5, kap=0.2)
    ref = o_ss(H, c)
    g = qtl.System(H, c, [c[0].conj().T @ c[0]])
    try:
        for prec in ("fp64", "mixed"):
            got = g.steadystate(precision=prec)
            assert maxabs(got["rho"], ref) <= 1e-10, prec
            assert got["stats"]["residual"] <= 1e-11, prec
        rho0 = np.zeros((132, 132), complex)
        rho0[0, 0] = 1.0
        tl = np.linspace(0.0, 0.5, 3)
        with pytest.raises(qtl.QtlError) as e:
            g.mesolve(rho0, tl, engine="cluster")
        assert e.value.status == qtl.QTL_ETOOBIG
        out = g.mesolve(rho0, tl, engine="grid")
        assert np.all(np.isfinite(out["expect"]))
    finally:
        g.free()
