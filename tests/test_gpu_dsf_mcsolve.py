"""GPU dynamical shifted Fock on quantum trajectories (qtl_dsf_mcsolve, Sec.
3.6 with Algorithm 1 of Appendix B applied per trajectory) through the C ABI
against the oracle's dsf_mcsolve, trajectory by trajectory (the same Philox
streams): the strongly driven cavity whose trajectories stay coherent, a
driven Kerr cavity, two displaced coupled cavities, a threshold that is never
reached; mixed precision against the closed form; edge cases."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.dsf import dsf_mcsolve as o_dsf_mc
from tests.gpu_util import maxabs, require_gpu

pytestmark = pytest.mark.gpu

TOL = dict(rtol=1e-10, atol=1e-12)


def destroy(N):
    return sp.diags(np.sqrt(np.arange(1, N)), 1, format="csr", dtype=complex)


def _cavity(D=0.5, F=7.0, kap=1.0):
    H = lambda o: D * (o[0].conj().T @ o[0]) + F * (o[0] + o[0].conj().T)
    c = lambda o: [math.sqrt(kap) * o[0]]
    e = lambda o: [o[0], o[0].conj().T @ o[0]]
    return H, c, e


def _both(qtl, H, c, e, ops, alpha0, psi0, tl, thr, ntraj, seed, **kw):
    tol = dict(TOL, **kw)
    ref = o_dsf_mc(H, c, e, ops, alpha0, psi0, tl, thr, ntraj=ntraj, seed=seed, keep_trajectories=True, **tol)
    got = qtl.dsf_mcsolve(H, c, e, ops, alpha0, psi0, tl, thr, ntraj, seed, keep_trajectories=True, **tol)
    return got, ref


@pytest.mark.parametrize("rebuild", ["device", "callback"])
def test_driven_cavity_trajectories_equal_the_oracle(rebuild, monkeypatch):
    """About 98 photons at a Fock cutoff of 8: every trajectory is displaced
    about 60 times and jumps; trajectory by trajectory equal to the oracle
    and to the exact coherent alpha(t).  By default the operators of a new
    frame are assembled on the device from the polynomial fit (the frames
    outgrow the first fit's range, so it is fitted once more), and the
    callback runs only for the fits' sample frames; with
    QTL_DSF_REBUILD=callback it runs at every displacement."""
    qtl = require_gpu()
    if rebuild == "callback":
        monkeypatch.setenv("QTL_DSF_REBUILD", "callback")
    else:
        monkeypatch.delenv("QTL_DSF_REBUILD", raising=False)
    N, D, F, kap = 8, 0.5, 7.0, 1.0
    H0, c, e = _cavity(D, F, kap)
    calls = [0]

    def H(o):
        calls[0] += 1
        return H0(o)
    tl = np.linspace(0.0, 3.0, 61)
    ref = o_dsf_mc(H0, c, e, [destroy(N)], [0.0], np.eye(N)[0], tl, 0.05, ntraj=8, seed=3,
                   keep_trajectories=True, **TOL)
    got = qtl.dsf_mcsolve(H, c, e, [destroy(N)], [0.0], np.eye(N)[0], tl, 0.05, 8, 3, keep_trajectories=True,
                          **TOL)
    assert got["shifts"] == ref["shifts"] > 8 * 40
    if rebuild == "device":
        assert calls[0] < 60
    else:
        assert calls[0] > got["shifts"] // 2
    assert got["stats"]["jumps"] == ref["stats"]["jumps"] > 10
    assert maxabs(got["traj_expect"], ref["traj_expect"]) <= 1e-8
    assert maxabs(got["expect"], ref["expect"]) <= 1e-8
    ass = -1j * F / (kap / 2 + 1j * D)
    al = ass * (1 - np.exp(-(kap / 2 + 1j * D) * tl))
    assert maxabs(got["traj_expect"][:, 0], np.broadcast_to(al, (8, len(tl)))) <= 1e-6


def test_driven_kerr_cavity_trajectories_equal_the_oracle():
    """A driven Kerr cavity (N = 10, <n> up to 12): its states are not
    coherent, jumps change them, and the shifts differ from trajectory to
    trajectory."""
    qtl = require_gpu()
    N, D, K, F, kap = 10, 0.5, 0.05, 3.0, 1.0
    H = lambda o: (D * (o[0].conj().T @ o[0]) + (K / 2) * (o[0].conj().T @ o[0].conj().T @ o[0] @ o[0])
                   + F * (o[0] + o[0].conj().T))
    c = lambda o: [math.sqrt(kap) * o[0]]
    e = lambda o: [o[0].conj().T @ o[0], o[0]]
    tl = np.linspace(0.0, 3.0, 31)
    got, ref = _both(qtl, H, c, e, [destroy(N)], [0.0], np.eye(N)[0], tl, 0.1, 16, 5, rtol=1e-9, atol=1e-11)
    assert got["shifts"] == ref["shifts"] > 16
    assert got["stats"]["jumps"] == ref["stats"]["jumps"]
    assert maxabs(got["traj_expect"], ref["traj_expect"]) <= 1e-7
    assert np.max(np.abs(got["expect"][0])) > 5.0


def test_two_displaced_modes_trajectories_equal_the_oracle():
    qtl = require_gpu()
    N, D1, D2, J, F, k1, k2 = 5, 0.4, -0.3, 0.8, 4.0, 1.0, 0.6
    a1 = sp.kron(destroy(N), sp.identity(N), format="csr")
    a2 = sp.kron(sp.identity(N), destroy(N), format="csr")
    tl = np.linspace(0.0, 2.0, 41)
    H = lambda o: (D1 * (o[0].conj().T @ o[0]) + D2 * (o[1].conj().T @ o[1])
                   + J * (o[0].conj().T @ o[1] + o[0] @ o[1].conj().T) + F * (o[0] + o[0].conj().T))
    c = lambda o: [math.sqrt(k1) * o[0], math.sqrt(k2) * o[1]]
    e = lambda o: [o[0], o[1]]
    psi0 = np.zeros(N * N)
    psi0[0] = 1.0
    got, ref = _both(qtl, H, c, e, [a1, a2], [0.0, 0.0], psi0, tl, 0.03, 6, 7)
    assert got["shifts"] == ref["shifts"] > 6 * 10
    assert maxabs(got["traj_expect"], ref["traj_expect"]) <= 1e-8


def test_unreached_threshold_equals_the_oracle():
    """No displacement: interval by interval, the trajectories keep their
    streams and thresholds across the checks."""
    qtl = require_gpu()
    N = 6
    a = destroy(N)
    tl = np.linspace(0.0, 4.0, 9)
    H = lambda o: 0.3 * (o[0].conj().T @ o[0]) + 0.4 * (o[0] + o[0].conj().T)
    c = lambda o: [math.sqrt(0.5) * o[0]]
    e = lambda o: [o[0], o[0].conj().T @ o[0]]
    got, ref = _both(qtl, H, c, e, [a], [0.0], np.eye(N)[0], tl, 1e9, 12, 11)
    assert got["shifts"] == ref["shifts"] == 0
    assert got["stats"]["jumps"] == ref["stats"]["jumps"] > 0
    assert maxabs(got["traj_expect"], ref["traj_expect"]) <= 1e-8


def test_mixed_precision_follows_the_coherent_state():
    qtl = require_gpu()
    N, D, F, kap = 8, 0.5, 7.0, 1.0
    H, c, e = _cavity(D, F, kap)
    tl = np.linspace(0.0, 3.0, 61)
    got = qtl.dsf_mcsolve(H, c, e, [destroy(N)], [0.0], np.eye(N)[0], tl, 0.05, 8, 3,
                          precision="mixed", rtol=1e-7, atol=1e-9)
    ass = -1j * F / (kap / 2 + 1j * D)
    al = ass * (1 - np.exp(-(kap / 2 + 1j * D) * tl))
    assert got["shifts"] > 8 * 40
    assert maxabs(got["expect"][0], al) <= 1e-5


def test_dsf_mcsolve_edge_cases():
    qtl = require_gpu()
    N = 6
    a = destroy(N)
    H, c, e = _cavity(0.3, 0.4, 0.5)
    tl = np.linspace(0.0, 1.0, 5)
    psi0 = np.eye(N)[0]
    for bad in [dict(threshold=0.0), dict(ntraj=0)]:
        kw = dict(threshold=0.1, ntraj=4)
        kw.update(bad)
        with pytest.raises(qtl.QtlError) as ex:
            qtl.dsf_mcsolve(H, c, e, [a], [0.0], psi0, tl, kw["threshold"], kw["ntraj"], 1)
        assert ex.value.status == qtl.QTL_EINVAL
    with pytest.raises(qtl.QtlError) as ex:
        qtl.dsf_mcsolve(H, c, e, [a], [0.0], psi0, tl, 0.1, 4, 1, engine="grid")
    assert ex.value.status == qtl.QTL_EINVAL
    big = destroy(1030)
    with pytest.raises(qtl.QtlError) as ex:
        qtl.dsf_mcsolve(H, c, e, [big], [0.0], np.eye(1030)[0], tl, 0.1, 2, 1)
    assert ex.value.status == qtl.QTL_ETOOBIG

    def bad(o):
        raise ValueError("no operators")
    with pytest.raises(ValueError):
        qtl.dsf_mcsolve(bad, c, e, [a], [0.0], psi0, tl, 0.1, 4, 1)
    # a single time: the observables of the initial ket, no integration (the
    # operators come from the polynomial fit, exact to its rounding)
    r = qtl.dsf_mcsolve(H, c, e, [a], [0.0], psi0, tl[:1], 0.1, 3, 1, keep_trajectories=True)
    assert maxabs(r["traj_expect"][:, :, 0], np.zeros((3, 2))) <= 1e-13
