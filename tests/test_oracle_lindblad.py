"""Pins for the master-equation oracle (Sec. 3.2): closed forms, brute-force
matrix exponentials, the two codings of the right-hand side against each
other, and the invariants of a Lindblad evolution."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import workloads as W
from oracle.lindblad import (effective_hamiltonian, liouvillian, lindblad_rhs,
                             unvec, vec)
from oracle.mesolve import initial_density_matrix, mesolve


def _rand_herm_dm(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    rho = A @ A.conj().T
    return rho / np.trace(rho)


def _superop_by_columns(H, c_ops):
    """The superoperator assembled by applying the map to each basis matrix
    E_ij (column i + n j), independent of the Kronecker formula."""
    n = H.shape[0]
    M = np.zeros((n * n, n * n), dtype=np.complex128)
    for j in range(n):
        for i in range(n):
            E = np.zeros((n, n), dtype=np.complex128)
            E[i, j] = 1.0
            # D[C] E written out entry by entry from its definition
            out = -1j * (H @ E - E @ H)
            for C in c_ops:
                Cd = C.conj().T
                out = out + C @ E @ Cd - 0.5 * (Cd @ C @ E + E @ Cd @ C)
            M[:, i + n * j] = out.reshape(-1, order="F")
    return M


SMALL = [
    ("cavity8", lambda: W.driven_cavity(N=8)),
    ("jc3x2", lambda: W.jaynes_cummings(N=3, kappa=0.05, gamma=0.02)),
    ("ising3", lambda: W.ising_chain(3, h=0.8)),
    ("thermal6", lambda: W.thermal_oscillator(N=6)),
]


@pytest.mark.parametrize("name,mk", SMALL, ids=[s[0] for s in SMALL])
def test_liouvillian_matches_map_by_columns(name, mk):
    s = mk()
    Hd = s.H.toarray()
    cd = [c.toarray() for c in s.c_ops]
    L = liouvillian(s.H, s.c_ops).toarray()
    M = _superop_by_columns(Hd, cd)
    assert np.max(np.abs(L - M)) < 1e-14


@pytest.mark.parametrize("mk", [W.driven_cavity, W.jaynes_cummings,
                                lambda: W.ising_chain(6, h=0.9)])
def test_liouvillian_vs_product_form(mk):
    s = mk()
    L = liouvillian(s.H, s.c_ops)
    rho = _rand_herm_dm(s.n, 7)
    a = unvec(L @ vec(rho), s.n)
    b = lindblad_rhs(s.H, s.c_ops, rho)
    assert np.max(np.abs(a - b)) <= 1e-13 * max(1.0, np.max(np.abs(b)))


@pytest.mark.parametrize("mk", [W.driven_cavity, W.jaynes_cummings,
                                lambda: W.ising_chain(5, h=1.1)])
def test_generator_invariants(mk):
    """Tr(L rho) = 0 and (L rho)^dag = L rho for Hermitian rho."""
    s = mk()
    rho = _rand_herm_dm(s.n, 3)
    d = lindblad_rhs(s.H, s.c_ops, rho)
    assert abs(np.trace(d)) < 1e-13
    assert np.max(np.abs(d - d.conj().T)) < 1e-13


def test_commutator_reading_breaks_trace():
    """The dissipator printed with a commutator is not trace preserving; the
    anticommutator form (used) is.  Plant the printed sign in a copy."""
    s = W.driven_cavity(N=6)
    rho = _rand_herm_dm(6, 1)
    C = s.c_ops[0].toarray()
    Cd = C.conj().T
    printed = C @ rho @ Cd - 0.5 * (Cd @ C @ rho - rho @ Cd @ C)
    assert abs(np.trace(printed)) > 1e-3
    used = C @ rho @ Cd - 0.5 * (Cd @ C @ rho + rho @ Cd @ C)
    assert abs(np.trace(used)) < 1e-14


def test_effective_hamiltonian():
    s = W.jaynes_cummings(N=5)
    Heff = effective_hamiltonian(s.H, s.c_ops).toarray()
    anti = Heff - Heff.conj().T
    target = -1j * sum(c.toarray().conj().T @ c.toarray() for c in s.c_ops)
    assert np.max(np.abs(anti - target)) < 1e-15
    assert np.max(np.abs((Heff + Heff.conj().T) / 2 - s.H.toarray())) < 1e-15


@pytest.mark.parametrize("name,mk", SMALL, ids=[s[0] for s in SMALL])
@pytest.mark.parametrize("method", ["dp5", "tsit5"])
def test_mesolve_vs_expm_bruteforce(name, mk, method):
    """Adaptive solve vs expm(M t) vec(rho0), M built column by column."""
    s = mk()
    tl = np.linspace(0, 6.0, 13)
    M = _superop_by_columns(s.H.toarray(), [c.toarray() for c in s.c_ops])
    r0 = vec(initial_density_matrix(s.psi0))
    res = mesolve(s.H, s.c_ops, s.e_ops, s.psi0, tl, method=method, rtol=1e-11, atol=1e-13)
    for it, t in enumerate(tl):
        rho = unvec(sla.expm(M * t) @ r0, s.n)
        for k, O in enumerate(s.e_ops):
            ref = np.trace(O.toarray() @ rho)
            assert abs(res["expect"][k, it] - ref) < 2e-9, (t, k)


def test_damped_oscillator_closed_form():
    """The GPU example of Sec. 4: <a'a>(t) = 3 exp(-gamma t)."""
    s = W.damped_oscillator()
    res = mesolve(s.H, s.c_ops, s.e_ops, s.psi0, s.tlist, rtol=1e-10, atol=1e-12)
    ref = 3 * np.exp(-0.1 * s.tlist)
    assert np.max(np.abs(res["expect"][0] - ref)) < 1e-8


def test_thermal_oscillator_closed_form():
    s = W.thermal_oscillator()
    p = s.params
    res = mesolve(s.H, s.c_ops, s.e_ops, s.psi0, s.tlist, rtol=1e-10, atol=1e-12)
    e = np.exp(-p["kappa"] * s.tlist)
    ref = p["n0"] * e + p["nth"] * (1 - e)
    assert np.max(np.abs(res["expect"][0] - ref)) < 1e-8


def test_driven_cavity_coherent_closed_form():
    """Coherent states stay coherent: alpha(t) = a_ss + (a0 - a_ss) e^{-(k/2 + i D) t},
    a_ss = -iF/(k/2 + iD); the long-time photon number is the paper's
    F^2/((w_c - w_d)^2 + k^2/4) (Sec. 5).  N = 40 so truncation is negligible."""
    s = W.driven_cavity(N=40)
    p = s.params
    k, D, F, a0 = p["kappa"], p["delta"], p["F"], p["alpha0"]
    ass = -1j * F / (k / 2 + 1j * D)
    tl = np.concatenate([s.tlist, [200.0]])
    res = mesolve(s.H, s.c_ops, s.e_ops, s.psi0, tl, rtol=1e-10, atol=1e-12)
    al = ass + (a0 - ass) * np.exp(-(k / 2 + 1j * D) * tl)
    assert np.max(np.abs(res["expect"][1] - al)) < 1e-8
    assert np.max(np.abs(res["expect"][0] - np.abs(al) ** 2)) < 1e-7
    assert abs(res["expect"][0][-1] - F ** 2 / (D ** 2 + k ** 2 / 4)) < 1e-8
    assert abs(ass - (-0.4950495049504950 - 0.0495049504950495j)) < 1e-15


@pytest.mark.parametrize("N", [2, 3, 6])
def test_jaynes_cummings_single_excitation(N):
    """rho0 = |0,e>, w_c = w_q: <a'a> = (g/W)^2 e^{-(k+g_)t/2} sin^2(W t),
    W = sqrt(g^2 - ((k - g_)/4)^2), exact for any cutoff N >= 2."""
    s = W.jaynes_cummings(N=N, nt=41, t_end=60.0)
    p = s.params
    g, k, gm = p["g"], p["kappa"], p["gamma"]
    Om = np.sqrt(g ** 2 - ((k - gm) / 4) ** 2)
    res = mesolve(s.H, s.c_ops, s.e_ops, s.psi0, s.tlist, rtol=1e-10, atol=1e-12)
    ref = (g / Om) ** 2 * np.exp(-(k + gm) * s.tlist / 2) * np.sin(Om * s.tlist) ** 2
    assert np.max(np.abs(res["expect"][0] - ref)) < 1e-8


def test_coupled_cavities_single_excitation():
    s = W.coupled_cavities(3, 4, J=0.7, kappa1=0.2, kappa2=0.05, nt=21, t_end=10.0)
    p = s.params
    M = np.array([[-0.5j * p["kappa1"], p["J"]], [p["J"], -0.5j * p["kappa2"]]])
    res = mesolve(s.H, s.c_ops, s.e_ops, s.psi0, s.tlist, rtol=1e-10, atol=1e-12)
    for it, t in enumerate(s.tlist):
        c = sla.expm(-1j * M * t) @ np.array([1.0, 0.0])
        assert abs(res["expect"][0, it] - abs(c[0]) ** 2) < 1e-8
        assert abs(res["expect"][1, it] - abs(c[1]) ** 2) < 1e-8


def test_ising_h0_population_decay():
    """h = 0: H diagonal, each spin decays independently, Sz = N(2 e^{-g t} - 1)."""
    s = W.ising_chain(4, h=0.0, t_end=5.0, nt=11)
    res = mesolve(s.H, s.c_ops, s.e_ops, s.psi0, s.tlist, rtol=1e-10, atol=1e-12)
    ref = 4 * (2 * np.exp(-0.1 * s.tlist) - 1)
    assert np.max(np.abs(res["expect"][2] - ref)) < 1e-8


def test_solution_invariants():
    """Along a solve: Tr rho = 1, rho = rho^dag, rho >= 0."""
    s = W.jaynes_cummings(N=4, nt=21, t_end=40.0)
    res = mesolve(s.H, s.c_ops, s.e_ops, s.psi0, s.tlist, save_states=True)
    for rho in res["states"]:
        assert abs(np.trace(rho) - 1) < 1e-12
        assert np.max(np.abs(rho - rho.conj().T)) < 1e-13
        assert np.min(np.linalg.eigvalsh((rho + rho.conj().T) / 2)) > -1e-10


def test_fixed_step_lands_on_tlist_and_counts():
    s = W.driven_cavity(N=6)
    tl = np.array([0.0, 0.25, 0.5, 1.0])
    res = mesolve(s.H, s.c_ops, s.e_ops, s.psi0, tl, fixed_dt=0.1)
    # 0.1, 0.1, 0.05 | 0.1, 0.1, 0.05 | 0.1 x 5  -> 11 steps, 6 RHS each + k1
    assert res["stats"]["steps_acc"] == 11
    assert res["stats"]["rhs_evals"] == 1 + 6 * 11
