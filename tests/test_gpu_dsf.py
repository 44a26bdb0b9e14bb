"""GPU dynamical shifted Fock master equation (qtl_dsf_mesolve, Sec. 3.6,
Appendix B Algorithm 1) through the C ABI against the oracle on its four
pinned systems: a strongly driven cavity followed at a Fock cutoff of 8, the
paper's two-mode Kerr model, two displaced coupled cavities, and a threshold
that is never reached."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.dsf import dsf_mesolve as o_dsf
from tests.gpu_util import maxabs, require_gpu

pytestmark = pytest.mark.gpu

TOL = dict(rtol=1e-10, atol=1e-12)


def destroy(N):
    return sp.diags(np.sqrt(np.arange(1, N)), 1, format="csr", dtype=complex)


def _both(qtl, H, c, e, ops, alpha0, psi0, tl, thr):
    ref = o_dsf(H, c, e, ops, alpha0, psi0, tl, thr, **TOL)
    got = qtl.dsf_mesolve(H, c, e, ops, alpha0, psi0, tl, thr, **TOL)
    return got, ref


def test_driven_cavity_small_cutoff():
    qtl = require_gpu()
    N, D, F, kap = 8, 0.5, 7.0, 1.0
    a = destroy(N)
    tl = np.linspace(0.0, 6.0, 301)
    H = lambda o: D * (o[0].conj().T @ o[0]) + F * (o[0] + o[0].conj().T)
    c = lambda o: [math.sqrt(kap) * o[0]]
    e = lambda o: [o[0], o[0].conj().T @ o[0]]
    got, ref = _both(qtl, H, c, e, [a], [0.0], np.eye(N)[0], tl, 0.05)
    assert got["shifts"] == ref["shifts"] > 100
    assert maxabs(got["alpha"], ref["alpha"]) <= 1e-8
    assert maxabs(got["expect"], ref["expect"]) <= 1e-8
    ass = -1j * F / (kap / 2 + 1j * D)
    al = ass * (1 - np.exp(-(kap / 2 + 1j * D) * tl))
    assert maxabs(got["expect"][0], al) <= 1e-6


def test_two_mode_kerr_model():
    qtl = require_gpu()
    D1, D2, U, J, F, k1, k22 = 0.5, 0.5, 0.05, 0.3, 1.5, 1.0, 0.01
    N1, N2 = 9, 6
    tl = np.linspace(0.0, 4.0, 81)
    a1 = sp.kron(destroy(N1), sp.identity(N2), format="csr")
    a2 = sp.kron(sp.identity(N1), destroy(N2), format="csr")
    a2d = a2.conj().T

    def H(o):
        b = o[0]
        return (D1 * (b.conj().T @ b) + D2 * (a2d @ a2) - U * (a2d @ a2d @ a2 @ a2)
                + J * (b @ a2d @ a2d + b.conj().T @ a2 @ a2) + F * (b + b.conj().T))

    c = lambda o: [math.sqrt(k1) * o[0], math.sqrt(k22) * (a2 @ a2)]
    e = lambda o: [o[0].conj().T @ o[0], a2d @ a2, o[0], a2]
    psi0 = np.zeros(N1 * N2)
    psi0[0] = 1.0
    got, ref = _both(qtl, H, c, e, [a1], [0.0], psi0, tl, 0.1)
    assert got["shifts"] == ref["shifts"] > 10
    assert maxabs(got["expect"], ref["expect"]) <= 1e-8
    assert maxabs(got["alpha"], ref["alpha"]) <= 1e-8


def test_two_displaced_modes():
    qtl = require_gpu()
    N, D1, D2, J, F, k1, k2 = 5, 0.4, -0.3, 0.8, 4.0, 1.0, 0.6
    a1 = sp.kron(destroy(N), sp.identity(N), format="csr")
    a2 = sp.kron(sp.identity(N), destroy(N), format="csr")
    tl = np.linspace(0.0, 5.0, 251)
    H = lambda o: (D1 * (o[0].conj().T @ o[0]) + D2 * (o[1].conj().T @ o[1])
                   + J * (o[0].conj().T @ o[1] + o[0] @ o[1].conj().T) + F * (o[0] + o[0].conj().T))
    c = lambda o: [math.sqrt(k1) * o[0], math.sqrt(k2) * o[1]]
    e = lambda o: [o[0], o[1]]
    psi0 = np.zeros(N * N)
    psi0[0] = 1.0
    got, ref = _both(qtl, H, c, e, [a1, a2], [0.0, 0.0], psi0, tl, 0.03)
    assert got["shifts"] == ref["shifts"] > 10
    assert maxabs(got["expect"], ref["expect"]) <= 1e-8
    assert maxabs(got["alpha"], ref["alpha"]) <= 1e-8


def test_unreached_threshold_and_edge_cases():
    qtl = require_gpu()
    N = 6
    a = destroy(N)
    tl = np.linspace(0.0, 2.0, 11)
    H = lambda o: 0.3 * (o[0].conj().T @ o[0]) + 0.2 * (o[0] + o[0].conj().T)
    c = lambda o: [math.sqrt(0.5) * o[0]]
    e = lambda o: [o[0], o[0].conj().T @ o[0]]
    rho0 = np.zeros((N, N), complex)
    rho0[0, 0] = 1.0
    got, ref = _both(qtl, H, c, e, [a], [0.0], rho0, tl, 1e9)
    assert got["shifts"] == 0
    assert maxabs(got["expect"], ref["expect"]) <= 1e-9
    with pytest.raises(qtl.QtlError) as ex:
        qtl.dsf_mesolve(H, c, e, [a], [0.0], rho0, tl, 0.0)
    assert ex.value.status == qtl.QTL_EINVAL
    # a builder that fails is reported
    def bad(o):
        raise ValueError("no operators")
    with pytest.raises(ValueError):
        qtl.dsf_mesolve(bad, c, e, [a], [0.0], rho0, tl, 0.1)
