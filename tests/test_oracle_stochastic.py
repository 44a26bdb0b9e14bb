"""Pins of the stochastic Schroedinger equation oracle (oracle/stochastic.py,
Sec. 3.5): the Box-Muller normals, the scheme's exact phase without
monitoring, a homodyne-monitored damped cavity whose coherent state every
trajectory keeps, and the dephasing rate of the ensemble mean."""
import math

import numpy as np
import scipy.sparse as sp
from scipy import stats

from oracle.stochastic import normal, sse_trajectory, ssesolve

SX = np.array([[0, 1], [1, 0]], dtype=complex)
SY = np.array([[0, -1j], [1j, 0]])
SZ = np.array([[1, 0], [0, -1]], dtype=complex)


def test_box_muller_normals():
    z = np.array([normal(7, 3, j) for j in range(20000)])
    assert abs(z.mean()) <= 4 / math.sqrt(len(z))
    assert abs(z.var() - 1.0) <= 4 * math.sqrt(2.0 / len(z))
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # different trajectories give different streams
    assert normal(7, 3, 0) != normal(7, 4, 0)


def test_without_monitoring_the_scheme_rotates_by_atan():
    """No stochastic operator: each step multiplies the sz components by
    1 -/+ i w h / 2 and renormalises, a relative phase of 2 atan(w h / 2) per
    step, so <sx> = cos(2 k atan(w h/2)) after k steps from |+>."""
    w, dt = 3.0, 0.01
    tl = np.linspace(0, 1, 11)
    psi0 = np.array([1, 1], dtype=complex) / math.sqrt(2)
    ex, ms = sse_trajectory(0.5 * w * SZ, [], [SX, SY], psi0, tl, dt, 1, 0)
    ph = 2 * 10 * np.arange(11) * math.atan(w * dt / 2)
    assert np.max(np.abs(ex[0] - np.cos(ph))) <= 1e-12
    assert np.max(np.abs(ex[1] - np.sin(ph))) <= 1e-12
    assert ms.shape == (0, 11)


def test_homodyne_detection_keeps_a_coherent_state():
    """S = sqrt(k) a on a damped cavity: S|alpha> = sqrt(k) alpha |alpha> and
    M = S - e/2 is then i sqrt(k) Im(alpha) times the identity, so the noise
    only multiplies the state by a scalar: every trajectory keeps
    <a> = alpha0 e^{-(i w + k/2) t} up to the scheme's O(dt) error, whatever
    its Wiener increments."""
    N, w, kap, a0 = 20, 1.0, 0.5, 1.0 + 0.5j
    a = sp.diags(np.sqrt(np.arange(1, N)), 1, format="csr", dtype=complex)
    n = np.arange(N)
    coh = np.exp(-abs(a0) ** 2 / 2) * a0 ** n / np.sqrt([math.factorial(int(k)) for k in n])
    coh /= np.linalg.norm(coh)
    tl = np.linspace(0, 1, 6)
    al = a0 * np.exp(-(1j * w + kap / 2) * tl)
    for traj in range(3):
        ex, ms = sse_trajectory(w * (a.conj().T @ a), [math.sqrt(kap) * a], [a], coh, tl, 1e-3, 5, traj)
        assert np.max(np.abs(ex[0] - al)) <= 5e-3
    # e_n at t0 is <S + S^dag> = 2 sqrt(k) Re(alpha0)
    assert abs(ms[0, 0] - 2 * math.sqrt(kap) * a0.real) <= 1e-9


def test_dephasing_monitor_ensemble_rate():
    """S = sqrt(g) sz on |+>: the ensemble mean follows D[sqrt(g) sz], so
    E<sx>(t) = exp(-2 g t) and E<sz> = 0 (within the sampling error and the
    scheme's O(dt) bias)."""
    g = 0.5
    tl = np.linspace(0, 1, 3)
    psi0 = np.array([1, 1], dtype=complex) / math.sqrt(2)
    r = ssesolve(np.zeros((2, 2)), [math.sqrt(g) * SZ], [SX, SZ], psi0, tl, 5e-3, 600, 11,
                 keep_trajectories=True)
    sd = r["traj_expect"][:, 0, :].real.std(axis=0)
    tol = 4 * sd / math.sqrt(600) + 0.01
    assert np.all(np.abs(r["expect"][0].real - np.exp(-2 * g * tl)) <= tol)
    sdz = r["traj_expect"][:, 1, :].real.std(axis=0)
    assert np.all(np.abs(r["expect"][1].real) <= 4 * sdz / math.sqrt(600) + 0.01)


from oracle.stochastic import sme_trajectory, smesolve  # noqa: E402


def test_sme_without_measurement_is_euler_on_lindblad():
    """No measured operator: explicit Euler on the master equation; for a
    decaying two-level system the excited population is (1 - g h)^k."""
    g, dt = 0.8, 0.01
    sm = np.array([[0, 0], [1, 0]], dtype=complex)
    tl = np.linspace(0, 1, 6)
    ex, ms = sme_trajectory(np.zeros((2, 2)), [math.sqrt(g) * sm], [], [np.diag([1.0, 0.0]).astype(complex)],
                            np.diag([1.0, 0.0]).astype(complex), tl, dt, 1, 0)
    k = 20 * np.arange(6)
    assert np.max(np.abs(ex[0] - (1 - g * dt) ** k)) <= 1e-12


def test_sme_homodyne_keeps_a_coherent_state():
    """S = sqrt(k) a on a damped cavity: H[S] maps |a><a| to a multiple of
    itself with zero trace, so every trajectory keeps <a> = alpha(t) up to
    the scheme's O(dt) error."""
    N, w, kap, a0 = 16, 1.0, 0.5, 1.0 + 0.5j
    a = sp.diags(np.sqrt(np.arange(1, N)), 1, format="csr", dtype=complex)
    v = np.zeros(N, dtype=complex)
    v[0] = math.exp(-abs(a0) ** 2 / 2)
    for q in range(1, N):
        v[q] = v[q - 1] * a0 / math.sqrt(q)
    v /= np.linalg.norm(v)
    tl = np.linspace(0, 1, 6)
    al = a0 * np.exp(-(1j * w + kap / 2) * tl)
    for traj in range(2):
        ex, ms = sme_trajectory(w * (a.conj().T @ a), [], [math.sqrt(kap) * a], [a], np.outer(v, v.conj()),
                                tl, 1e-3, 5, traj)
        assert np.max(np.abs(ex[0] - al)) <= 5e-3


def test_sme_ensemble_mean_is_euler_on_lindblad():
    """Given rho_k the Euler-Maruyama step's noise term has zero mean, and the
    master equation is linear, so the ensemble mean follows explicit Euler on
    the master equation: monitored dephasing S = sqrt(g) sz on |+> gives
    E<sx> = (1 - 2 g h)^k within the sampling error."""
    g, dt = 0.5, 0.01
    SZ_ = np.diag([1.0, -1.0]).astype(complex)
    SX_ = np.array([[0, 1], [1, 0]], dtype=complex)
    tl = np.linspace(0, 1, 3)
    r = smesolve(np.zeros((2, 2)), [], [math.sqrt(g) * SZ_], [SX_], np.array([1, 1]) / math.sqrt(2), tl, dt,
                 400, 13, keep_trajectories=True)
    sd = r["traj_expect"][:, 0, :].real.std(axis=0)
    k = 50 * np.arange(3)
    assert np.all(np.abs(r["expect"][0].real - (1 - 2 * g * dt) ** k) <= 4 * sd / math.sqrt(400) + 1e-12)
