"""ssesolve (Sec. 3.5) through the C ABI: trajectory means of the
expectation values and of the homodyne currents against the oracle (the
same Euler-Maruyama steps and Wiener increments), a homodyne-monitored
damped cavity whose trajectories keep their coherent state, and the
argument checks."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.stochastic import ssesolve as o_ssesolve
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def destroy(N):
    return sp.diags(np.sqrt(np.arange(1, N)), 1, format="csr", dtype=complex)


def coherent(N, alpha):
    # c_k = e^{-|alpha|^2/2} alpha^k / sqrt(k!), by the recurrence c_k = c_{k-1} alpha / sqrt(k)
    v = np.zeros(N, dtype=complex)
    v[0] = np.exp(-abs(alpha) ** 2 / 2)
    for k in range(1, N):
        v[k] = v[k - 1] * alpha / math.sqrt(k)
    return v / np.linalg.norm(v)


def _jc(N=5, wc=1.0, wq=1.0, g=0.3, kappa=1.0, gamma=0.4, two=False):
    """The paper's homodyne example (JC, S = sqrt(k) a, X = S + S^dag,
    psi0 = |alpha, e>) at a small cutoff and slower frequencies."""
    a = sp.kron(destroy(N), sp.identity(2), format="csr")
    sm = sp.kron(sp.identity(N), sp.csr_matrix(np.array([[0, 0], [1, 0]], dtype=complex)), format="csr")
    sz = sp.kron(sp.identity(N), sp.csr_matrix(np.diag([1.0, -1.0]).astype(complex)), format="csr")
    H = (wc * a.conj().T @ a + wq * sz / 2 + g * (a.conj().T @ sm + a @ sm.conj().T)).tocsr()
    sc = [math.sqrt(kappa) * a] + ([math.sqrt(gamma) * sm] if two else [])
    X = (math.sqrt(kappa) * (a + a.conj().T)).tocsr()
    psi0 = np.kron(coherent(N, 0.5), np.array([1.0, 0.0]))
    return H, sc, [X, (a.conj().T @ a).tocsr()], psi0


@pytest.mark.parametrize("two", [False, True], ids=["one_sc", "two_sc"])
def test_ssesolve_matches_oracle(two):
    qtl = require_gpu()
    H, sc, e_ops, psi0 = _jc(two=two)
    tl = np.linspace(0, 2, 5)
    g = qtl.System(H, sc, e_ops)
    try:
        got = g.ssesolve(psi0, tl, 8, 21, fixed_dt=0.002, keep_trajectories=True)
    finally:
        g.free()
    ref = o_ssesolve(H, sc, e_ops, psi0, tl, 0.002, 8, 21, keep_trajectories=True)
    # trajectory by trajectory (same Wiener increments), then the means
    assert np.max(np.abs(got["traj_expect"] - ref["traj_expect"])) <= 1e-10
    assert np.max(np.abs(got["traj_measurement"] - ref["traj_measurement"])) <= 1e-8
    assert np.max(np.abs(got["expect"] - ref["expect"])) <= 1e-10
    assert np.max(np.abs(got["measurement"] - ref["measurement"])) <= 1e-8
    assert got["stats"]["steps_acc"] == 8 * 1000


def test_ssesolve_homodyne_keeps_coherent_states():
    qtl = require_gpu()
    N, w, kap, a0 = 20, 1.0, 0.5, 1.0 + 0.5j
    a = destroy(N)
    tl = np.linspace(0, 1, 6)
    g = qtl.System(w * (a.conj().T @ a), [math.sqrt(kap) * a], [a])
    try:
        got = g.ssesolve(coherent(N, a0), tl, 64, 5, fixed_dt=1e-3)
    finally:
        g.free()
    al = a0 * np.exp(-(1j * w + kap / 2) * tl)
    assert np.max(np.abs(got["expect"][0] - al)) <= 5e-3
    assert abs(got["measurement"][0, 0] - 2 * math.sqrt(kap) * a0.real) <= 1e-9


def test_ssesolve_refuses_bad_arguments():
    qtl = require_gpu()
    H, sc, e_ops, psi0 = _jc()
    tl = np.linspace(0, 1, 3)
    g = qtl.System(H, sc, e_ops)
    with pytest.raises(qtl.QtlError) as e1:
        g.ssesolve(psi0, tl, 2, 1)                                   # adaptive: no fixed step
    with pytest.raises(qtl.QtlError) as e2:
        g.ssesolve(psi0, tl, 2, 1, fixed_dt=0.01, precision="mixed")
    with pytest.raises(qtl.QtlError) as e4:
        g.ssesolve(psi0, tl, 2, 1, fixed_dt=0.01, max_steps=50)     # 100 steps needed
    assert e4.value.status == qtl.QTL_ESTEP
    g.free()
    g2 = qtl.System(H, [], e_ops)
    with pytest.raises(qtl.QtlError) as e3:
        g2.ssesolve(psi0, tl, 2, 1, fixed_dt=0.01)                   # no stochastic operator
    g2.free()
    for e in (e1, e2, e3):
        assert e.value.status == qtl.QTL_EINVAL


@pytest.mark.parametrize("N", [300, 600], ids=["rows2", "rows4"])
def test_ssesolve_two_and_four_rows_per_thread(N):
    """Dimensions above 256 take 2 and 4 rows per thread: parity with the
    oracle over a short horizon."""
    qtl = require_gpu()
    a = destroy(N)
    H = (1.3 * (a.conj().T @ a) + 0.2 * (a + a.conj().T)).tocsr()
    sc = [math.sqrt(0.7) * a]
    e_ops = [a, (a.conj().T @ a).tocsr()]
    psi0 = coherent(N, 1.5 - 0.5j)
    tl = np.linspace(0, 0.04, 3)
    g = qtl.System(H, sc, e_ops)
    try:
        got = g.ssesolve(psi0, tl, 2, 9, fixed_dt=0.002)
    finally:
        g.free()
    ref = o_ssesolve(H, sc, e_ops, psi0, tl, 0.002, 2, 9)
    assert np.max(np.abs(got["expect"] - ref["expect"])) <= 1e-10
    assert np.max(np.abs(got["measurement"] - ref["measurement"])) <= 1e-8
