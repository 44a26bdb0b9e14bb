"""smesolve (Sec. 3.5) through the C ABI: trajectory means of Tr(O rho) and
of the homodyne currents against the oracle (the same Euler-Maruyama steps
and Wiener increments) at 1, 2 and 4 density-matrix entries per thread, a
homodyne-monitored damped cavity whose trajectories stay coherent, and the
argument checks."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.stochastic import smesolve as o_smesolve
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def destroy(N):
    return sp.diags(np.sqrt(np.arange(1, N)), 1, format="csr", dtype=complex)


def coherent(N, alpha):
    v = np.zeros(N, dtype=complex)
    v[0] = np.exp(-abs(alpha) ** 2 / 2)
    for k in range(1, N):
        v[k] = v[k - 1] * alpha / math.sqrt(k)
    return v / np.linalg.norm(v)


def _jc(N, kappa=1.0, gamma=0.4):
    """The paper's SME example at a small cutoff: JC with qubit decay as an
    unmeasured loss and homodyne detection of sqrt(kappa) a."""
    a = sp.kron(destroy(N), sp.identity(2), format="csr")
    sm = sp.kron(sp.identity(N), sp.csr_matrix(np.array([[0, 0], [1, 0]], dtype=complex)), format="csr")
    sz = sp.kron(sp.identity(N), sp.csr_matrix(np.diag([1.0, -1.0]).astype(complex)), format="csr")
    H = (a.conj().T @ a + sz / 2 + 0.3 * (a.conj().T @ sm + a @ sm.conj().T)).tocsr()
    C = [math.sqrt(gamma) * sm]
    S = [math.sqrt(kappa) * a]
    X = (math.sqrt(kappa) * (a + a.conj().T)).tocsr()
    psi0 = np.kron(coherent(N, 0.5), np.array([1.0, 0.0]))
    return H, C, S, [X, (a.conj().T @ a).tocsr()], psi0


@pytest.mark.parametrize("N,tl,dt", [(5, np.linspace(0, 1, 5), 0.002), (20, np.linspace(0, 0.04, 3), 0.002),
                                     (32, np.linspace(0, 0.02, 3), 0.002)], ids=["ept1", "ept2", "ept4"])
def test_smesolve_matches_oracle(N, tl, dt):
    qtl = require_gpu()
    H, C, S, e_ops, psi0 = _jc(N)
    g = qtl.System(H, C + S, e_ops)
    try:
        got = g.smesolve(1, psi0, tl, 2, 19, fixed_dt=dt, keep_trajectories=True)
    finally:
        g.free()
    ref = o_smesolve(H, C, S, e_ops, psi0, tl, dt, 2, 19, keep_trajectories=True)
    # trajectory by trajectory (same Wiener increments), then the means
    assert np.max(np.abs(got["traj_expect"] - ref["traj_expect"])) <= 1e-10
    assert np.max(np.abs(got["traj_measurement"] - ref["traj_measurement"])) <= 1e-8
    assert np.max(np.abs(got["expect"] - ref["expect"])) <= 1e-10
    assert np.max(np.abs(got["measurement"] - ref["measurement"])) <= 1e-8


def test_smesolve_homodyne_keeps_coherent_states():
    qtl = require_gpu()
    N, w, kap, a0 = 16, 1.0, 0.5, 1.0 + 0.5j
    a = destroy(N)
    tl = np.linspace(0, 1, 6)
    g = qtl.System(w * (a.conj().T @ a), [math.sqrt(kap) * a], [a])
    try:
        got = g.smesolve(1, coherent(N, a0), tl, 16, 5, fixed_dt=1e-3)
    finally:
        g.free()
    al = a0 * np.exp(-(1j * w + kap / 2) * tl)
    assert np.max(np.abs(got["expect"][0] - al)) <= 5e-3
    assert abs(got["measurement"][0, 0] - 2 * math.sqrt(kap) * a0.real) <= 1e-9


def test_smesolve_refuses_bad_arguments():
    qtl = require_gpu()
    H, C, S, e_ops, psi0 = _jc(5)
    tl = np.linspace(0, 1, 3)
    g = qtl.System(H, C + S, e_ops)
    with pytest.raises(qtl.QtlError) as e1:
        g.smesolve(1, psi0, tl, 2, 1)                       # adaptive: no fixed step
    with pytest.raises(qtl.QtlError) as e2:
        g.smesolve(3, psi0, tl, 2, 1, fixed_dt=0.01)        # more measured than collapse operators
    with pytest.raises(qtl.QtlError) as e4:
        g.smesolve(1, psi0, tl, 2, 1, fixed_dt=0.01, max_steps=50)   # 100 steps needed
    assert e4.value.status == qtl.QTL_ESTEP
    r = g.smesolve(1, psi0, tl, 2, 1, fixed_dt=0.01, max_steps=100)  # the system is still usable
    assert np.all(np.isfinite(r["expect"]))
    g.free()
    H2, C2, S2, e2_ops, p2 = _jc(40)                        # n = 80: n*n > 4096
    g2 = qtl.System(H2, C2 + S2, e2_ops)
    with pytest.raises(qtl.QtlError) as e3:
        g2.smesolve(1, p2, tl, 2, 1, fixed_dt=0.01)
    g2.free()
    assert e1.value.status == qtl.QTL_EINVAL and e2.value.status == qtl.QTL_EINVAL
    assert e3.value.status == qtl.QTL_ETOOBIG
