"""Pins of the oracle's time-dependent Hamiltonians and sesolve
(oracle/timedep.py) against closed forms and a library integrator."""
import math

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.integrate import solve_ivp
from scipy.special import erf

from oracle.lindblad import lindblad_rhs, liouvillian, unvec, vec
from oracle.timedep import Coef, hamiltonian_at, mcsolve_td, mesolve_td, sesolve

SX = np.array([[0, 1], [1, 0]], dtype=complex)
SY = np.array([[0, -1j], [1j, 0]])
SZ = np.array([[1, 0], [0, -1]], dtype=complex)


def destroy(N):
    return sp.diags(np.sqrt(np.arange(1, N)), 1, format="csr", dtype=complex)


def test_coefficient_forms():
    c = Coef("cos", 2.0, 3.0, 0.5)
    assert c(0.7) == pytest.approx(2.0 * math.cos(3.0 * 0.7 + 0.5), abs=1e-15)
    e = Coef("exp", 1 - 2j, 1.5, -0.25, t0=1.0, sigma=0.5)
    t = 1.3
    ref = (1 - 2j) * math.exp(-(t - 1.0) ** 2 / (2 * 0.25)) * np.exp(1j * (1.5 * t - 0.25))
    assert abs(e(t) - ref) <= 1e-15


def test_sz_phase_drive_closed_form():
    """H = A cos(w t) sz, psi0 = |+>: psi(t) = exp(-i Phi sz)|+> with
    Phi = (A/w) sin(w t), so <sx> = cos 2 Phi and <sy> = sin 2 Phi."""
    A, w = 1.3, 2.1
    tl = np.linspace(0, 6, 25)
    psi0 = np.array([1, 1], dtype=complex) / math.sqrt(2)
    r = sesolve(np.zeros((2, 2)), [(SZ, Coef("cos", A, w))], [SX, SY], psi0, tl, rtol=1e-11, atol=1e-13)
    phi = (A / w) * np.sin(w * tl)
    assert np.max(np.abs(r["expect"][0] - np.cos(2 * phi))) <= 1e-9
    assert np.max(np.abs(r["expect"][1] - np.sin(2 * phi))) <= 1e-9


def test_gaussian_pulse_rotation_closed_form():
    """H = f(t) sx / 2 with a Gaussian f: a rotation about x by
    theta(t) = int_0^t f, so from |0> (sz = +1) <sz> = cos theta, <sy> = -sin theta."""
    Om, t0, sig = 2.0, 3.0, 0.7
    tl = np.linspace(0, 6, 31)
    r = sesolve(np.zeros((2, 2)), [(SX / 2, Coef("cos", Om, 0.0, 0.0, t0, sig))], [SZ, SY],
                np.array([1, 0], dtype=complex), tl, rtol=1e-11, atol=1e-13)
    th = Om * sig * math.sqrt(math.pi / 2) * (erf((tl - t0) / (sig * math.sqrt(2))) + erf(t0 / (sig * math.sqrt(2))))
    assert np.max(np.abs(r["expect"][0] - np.cos(th))) <= 1e-9
    assert np.max(np.abs(r["expect"][1] + np.sin(th))) <= 1e-9


def _alpha_exp_pair(t, wc, gam, F, w):
    # a' = -(i wc + g/2) a - i conj(f(t)), f = F e^{i w t}, alpha(0) = 0
    z = 1j * wc + gam / 2
    return -1j * np.conj(F) * (np.exp(-1j * w * t) - np.exp(-z * t)) / (z - 1j * w)


def _alpha_cos(t, D, kap, F, w):
    # a' = -(i D + k/2) a - i F cos(w t), alpha(0) = 0
    z = 1j * D + kap / 2
    return -0.5j * F * ((np.exp(1j * w * t) - np.exp(-z * t)) / (z + 1j * w)
                        + (np.exp(-1j * w * t) - np.exp(-z * t)) / (z - 1j * w))


def test_complex_exp_pair_drive_coherent_mesolve_and_trajectories():
    """H = wc a'a + f(t) a + conj(f(t)) a' (the pair of Sec. 5) with loss
    sqrt(g) a keeps a coherent state coherent: <a> = alpha(t) for mesolve and
    for every single trajectory (a jump leaves a coherent state unchanged)."""
    N, wc, gam, F, w = 16, 1.0, 0.8, 0.3 + 0.1j, 1.2
    a = destroy(N)
    terms = [(a, Coef("exp", F, w)), (a.conj().T, Coef("exp", np.conj(F), -w))]
    tl = np.linspace(0, 8, 17)
    psi0 = np.zeros(N, dtype=complex)
    psi0[0] = 1
    al = _alpha_exp_pair(tl, wc, gam, F, w)
    me = mesolve_td(wc * (a.conj().T @ a), terms, [math.sqrt(gam) * a], [a, a.conj().T @ a], psi0, tl,
                    rtol=1e-10, atol=1e-12)
    assert np.max(np.abs(me["expect"][0] - al)) <= 1e-8
    assert np.max(np.abs(me["expect"][1] - np.abs(al) ** 2)) <= 1e-8
    mc = mcsolve_td(wc * (a.conj().T @ a), terms, [math.sqrt(gam) * a], [a], psi0, tl, 6, 3,
                    rtol=1e-10, atol=1e-12, keep_trajectories=True)
    assert sum(len(j) for j in mc["jump_times"]) > 0          # trajectories did jump
    assert np.max(np.abs(mc["traj_expect"][:, 0, :] - al[None, :])) <= 1e-7


def test_cos_drive_closed_form_both_rhs_forms():
    """The drive of Sec. 3.4, F cos(w_d t)(a + a'), on a damped cavity."""
    N, D, kap, F, w = 16, 0.7, 0.5, 0.4, 1.1
    a = destroy(N)
    tl = np.linspace(0, 10, 21)
    psi0 = np.zeros(N, dtype=complex)
    psi0[0] = 1
    al = _alpha_cos(tl, D, kap, F, w)
    for rhs in ("product", "liouvillian"):
        me = mesolve_td(D * (a.conj().T @ a), [(a + a.conj().T, Coef("cos", F, w))], [math.sqrt(kap) * a],
                        [a], psi0, tl, rtol=1e-10, atol=1e-12, rhs=rhs)
        assert np.max(np.abs(me["expect"][0] - al)) <= 1e-8


def _random_system(rng, n):
    def herm():
        m = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        return (m + m.conj().T) / 2
    C = 0.4 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    B = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    terms = [(herm(), Coef("cos", 0.7, 1.3, 0.2, t0=1.0, sigma=0.8)),
             (B, Coef("exp", 0.3 - 0.2j, 0.9)), (B.conj().T, Coef("exp", 0.3 + 0.2j, -0.9))]
    return herm(), terms, [C]


def test_liouvillian_and_product_forms_agree_at_random_times():
    rng = np.random.default_rng(8)
    H0, terms, c_ops = _random_system(rng, 4)
    rho = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    L0 = liouvillian(H0, c_ops)
    for t in (0.0, 0.37, 2.9):
        a = vec(lindblad_rhs(hamiltonian_at(H0, terms, t), c_ops, rho))
        b = L0 @ vec(rho)
        for Hk, fk in terms:
            b = b + fk(t) * (liouvillian(Hk, []) @ vec(rho))
        assert np.max(np.abs(a - b)) <= 1e-13 * max(1.0, np.max(np.abs(a)))


def test_mesolve_and_sesolve_match_a_library_integrator():
    """Random 4-level system with three driven terms: the oracle's adaptive
    integration against scipy's DOP853 at tight tolerances."""
    rng = np.random.default_rng(9)
    H0, terms, c_ops = _random_system(rng, 4)
    n = 4
    psi0 = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    psi0 /= np.linalg.norm(psi0)
    tl = np.linspace(0, 3, 7)
    me = mesolve_td(H0, terms, c_ops, [], psi0, tl, rtol=1e-11, atol=1e-13, save_states=True)

    def f(t, y):
        return vec(lindblad_rhs(hamiltonian_at(H0, terms, t), c_ops, unvec(y, n)))
    ref = solve_ivp(f, (0, 3), vec(np.outer(psi0, psi0.conj())), method="DOP853", t_eval=tl,
                    rtol=1e-13, atol=1e-15)
    got = np.array([vec(r) for r in me["states"]]).T
    assert np.max(np.abs(got - ref.y)) <= 1e-8
    se = sesolve(H0, terms, [], psi0, tl, rtol=1e-11, atol=1e-13, save_states=True)
    ref2 = solve_ivp(lambda t, y: -1j * (hamiltonian_at(H0, terms, t) @ y), (0, 3), psi0,
                     method="DOP853", t_eval=tl, rtol=1e-13, atol=1e-15)
    assert np.max(np.abs(se["states"].T - ref2.y)) <= 1e-8


def test_trajectory_without_collapse_operators_is_sesolve():
    """No collapse operator: no jump, and the trajectory equals sesolve."""
    rng = np.random.default_rng(10)
    H0, terms, _ = _random_system(rng, 4)
    terms = terms[:1]
    psi0 = np.array([1, 0, 0, 0], dtype=complex)
    tl = np.linspace(0, 2, 5)
    O = [np.diag([1.0, 2.0, 3.0, 4.0]).astype(complex)]
    mc = mcsolve_td(H0, terms, [], O, psi0, tl, 3, 1, rtol=1e-9, atol=1e-11, keep_trajectories=True)
    se = sesolve(H0, terms, O, psi0, tl, rtol=1e-9, atol=1e-11)
    assert all(len(j) == 0 for j in mc["jump_times"])
    assert np.max(np.abs(mc["traj_expect"][0] - se["expect"])) <= 1e-13
