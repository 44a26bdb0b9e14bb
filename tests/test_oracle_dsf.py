"""Pins of the dynamical-shifted-Fock oracle (oracle/dsf.py; Sec. 3.6,
Appendix B): a strongly driven damped cavity, whose exact state is the
coherent state alpha(t) = alpha_ss (1 - e^{-(k/2 + i D) t}), followed with a
Fock cutoff of 8 where the plain solve fails; the paper's two-mode model with
a Kerr mode and a nonlinear coupling against a plain mesolve at a cutoff that
holds the whole displaced state; two displaced modes against their exact
linear equations; and an unreached threshold, which reduces DSF to the plain
solve."""
import math

import numpy as np
import scipy.sparse as sp

from oracle.dsf import dsf_mesolve
from oracle.mesolve import mesolve


def destroy(N):
    return sp.diags(np.sqrt(np.arange(1, N)), 1, format="csr", dtype=complex)


def test_driven_cavity_follows_the_coherent_state_with_a_small_cutoff():
    N, D, F, kap = 8, 0.5, 7.0, 1.0
    a = destroy(N)
    tl = np.linspace(0.0, 6.0, 301)
    H = lambda o: D * (o[0].conj().T @ o[0]) + F * (o[0] + o[0].conj().T)
    c = lambda o: [math.sqrt(kap) * o[0]]
    e = lambda o: [o[0], o[0].conj().T @ o[0]]
    r = dsf_mesolve(H, c, e, [a], [0.0], np.eye(N)[0], tl, 0.05, rtol=1e-10, atol=1e-12)
    ass = -1j * F / (kap / 2 + 1j * D)
    al = ass * (1 - np.exp(-(kap / 2 + 1j * D) * tl))
    assert abs(ass) > 9.8                                   # <n> near 98 photons
    assert np.max(np.abs(r["expect"][0] - al)) <= 1e-6
    assert np.max(np.abs(r["expect"][1] - np.abs(al) ** 2)) <= 1e-5
    assert np.max(np.abs(r["alpha"][0] - al)) <= 0.06      # tracked within the threshold
    assert r["shifts"] > 100
    plain = mesolve(H([a]), c([a]), [a], np.eye(N)[0], tl, rtol=1e-10, atol=1e-12)
    assert np.max(np.abs(plain["expect"][0] - al)) > 1.0    # the cutoff alone cannot hold it


def test_two_mode_kerr_model_matches_a_large_cutoff_solve():
    """Sec. 3.6's model: D1 a1'a1 + D2 a2'a2 - U a2'^2 a2^2 + J (a1 a2'^2 +
    a1' a2^2) + F (a1 + a1'), losses a1, a2^2; DSF on mode 1 only.  F is
    lowered to 1.5 so that a plain solve with mode 1 cut at 30 holds the state
    (cut at 22 it is already within 2e-6).  DSF converges in its own cutoff:
    5 states leave 2e-3, 7 leave 2e-5, 9 leave the reference's error."""
    D1, D2, U, J, F, k1, k22 = 0.5, 0.5, 0.05, 0.3, 1.5, 1.0, 0.01
    N1s, N1, N2 = 9, 30, 6
    tl = np.linspace(0.0, 4.0, 81)

    def model(N1_):
        a1 = sp.kron(destroy(N1_), sp.identity(N2), format="csr")
        a2 = sp.kron(sp.identity(N1_), destroy(N2), format="csr")
        a2d = a2.conj().T

        def H(o):
            b = o[0]
            return (D1 * (b.conj().T @ b) + D2 * (a2d @ a2) - U * (a2d @ a2d @ a2 @ a2)
                    + J * (b @ a2d @ a2d + b.conj().T @ a2 @ a2) + F * (b + b.conj().T))

        c = lambda o: [math.sqrt(k1) * o[0], math.sqrt(k22) * (a2 @ a2)]
        e = lambda o: [o[0].conj().T @ o[0], a2d @ a2, o[0], a2]
        return a1, H, c, e

    a1, H, c, e = model(N1s)
    psi0 = np.zeros(N1s * N2)
    psi0[0] = 1.0
    r = dsf_mesolve(H, c, e, [a1], [0.0], psi0, tl, 0.1, rtol=1e-10, atol=1e-12)
    b1, Hb, cb, eb = model(N1)
    p0 = np.zeros(N1 * N2)
    p0[0] = 1.0
    ref = mesolve(Hb([b1]), cb([b1]), eb([b1]), p0, tl, rtol=1e-10, atol=1e-12)
    assert np.max(np.abs(ref["expect"][0])) > 3.0           # mode 1 well beyond the small cutoff
    assert np.max(np.abs(ref["expect"][1])) > 1e-3          # mode 2 fed by the coupling
    assert np.max(np.abs(r["expect"] - ref["expect"])) <= 1e-6
    assert r["shifts"] > 10
    small = mesolve(H([a1]), c([a1]), e([a1]), psi0, tl, rtol=1e-10, atol=1e-12)
    assert np.max(np.abs(small["expect"] - ref["expect"])) > 1e-3   # the same cutoff without DSF


def test_unreached_threshold_is_the_plain_solve():
    N = 6
    a = destroy(N)
    tl = np.linspace(0.0, 2.0, 11)
    H = lambda o: 0.3 * (o[0].conj().T @ o[0]) + 0.2 * (o[0] + o[0].conj().T)
    c = lambda o: [math.sqrt(0.5) * o[0]]
    e = lambda o: [o[0], o[0].conj().T @ o[0]]
    r = dsf_mesolve(H, c, e, [a], [0.0], np.eye(N)[0], tl, 1e9, rtol=1e-10, atol=1e-12)
    ref = mesolve(H([a]), c([a]), e([a]), np.eye(N)[0], tl, rtol=1e-10, atol=1e-12)
    assert r["shifts"] == 0
    assert np.max(np.abs(r["expect"] - ref["expect"])) <= 1e-9


def test_two_displaced_modes_follow_the_linear_coherent_solution():
    """DSF on both modes of two driven, lossy cavities with a beam-splitter
    coupling J (a1' a2 + a1 a2'): the state stays coherent, with
    d alpha/dt = M alpha + f, M = [[-i D1 - k1/2, -i J], [-i J, -i D2 - k2/2]],
    f = (-i F, 0), solved exactly by the exponential of the augmented 3x3
    system.  Each mode keeps its own tracked coherence."""
    import scipy.linalg as sla
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
    r = dsf_mesolve(H, c, e, [a1, a2], [0.0, 0.0], psi0, tl, 0.03, rtol=1e-10, atol=1e-12)
    M = np.array([[-1j * D1 - k1 / 2, -1j * J, -1j * F],
                  [-1j * J, -1j * D2 - k2 / 2, 0.0],
                  [0.0, 0.0, 0.0]])
    exact = np.array([(sla.expm(M * t) @ np.array([0.0, 0.0, 1.0]))[:2] for t in tl]).T
    assert np.min(np.max(np.abs(exact), axis=1)) > 1.5        # both modes leave the small cutoff
    assert np.max(np.abs(r["expect"] - exact)) <= 1e-6
    assert np.max(np.abs(r["alpha"] - exact)) <= 0.04


# ------------------------------------------------------------ dsf_mcsolve
from oracle.dsf import dsf_mcsolve  # noqa: E402
from oracle.mcsolve import mcsolve  # noqa: E402


def _cavity(N=8, D=0.5, F=7.0, kap=1.0):
    a = destroy(N)
    H = lambda o: D * (o[0].conj().T @ o[0]) + F * (o[0] + o[0].conj().T)
    c = lambda o: [math.sqrt(kap) * o[0]]
    e = lambda o: [o[0], o[0].conj().T @ o[0]]
    return a, H, c, e


def test_dsf_trajectories_of_a_driven_cavity_stay_coherent():
    """A jump of sqrt(k) a leaves a coherent state unchanged, so every DSF
    trajectory of the strongly driven cavity (about 98 photons, cutoff 8)
    follows alpha(t) exactly, jumps and displacements included."""
    N, D, F, kap = 8, 0.5, 7.0, 1.0
    a, H, c, e = _cavity(N, D, F, kap)
    tl = np.linspace(0.0, 3.0, 61)
    r = dsf_mcsolve(H, c, e, [a], [0.0], np.eye(N)[0], tl, 0.05, ntraj=4, seed=3,
                    rtol=1e-10, atol=1e-12, keep_trajectories=True)
    ass = -1j * F / (kap / 2 + 1j * D)
    al = ass * (1 - np.exp(-(kap / 2 + 1j * D) * tl))
    assert r["stats"]["jumps"] > 10 and r["shifts"] > 100
    for j in range(4):
        assert np.max(np.abs(r["traj_expect"][j, 0] - al)) <= 1e-6
        assert np.max(np.abs(r["traj_expect"][j, 1] - np.abs(al) ** 2)) <= 1e-5


def test_dsf_mcsolve_with_an_unreached_threshold_is_mcsolve():
    """No displacement: the DSF trajectories are mcsolve's trajectories with
    the same random streams, integrated check to check."""
    N = 6
    a = destroy(N)
    tl = np.linspace(0.0, 4.0, 9)
    H = lambda o: 0.3 * (o[0].conj().T @ o[0]) + 0.4 * (o[0] + o[0].conj().T)
    c = lambda o: [math.sqrt(0.5) * o[0]]
    e = lambda o: [o[0], o[0].conj().T @ o[0]]
    r = dsf_mcsolve(H, c, e, [a], [0.0], np.eye(N)[0], tl, 1e9, ntraj=6, seed=11,
                    rtol=1e-10, atol=1e-12, keep_trajectories=True)
    ref = mcsolve(H([a]), c([a]), e([a]), np.eye(N)[0], tl, ntraj=6, seed=11, rtol=1e-10, atol=1e-12,
                  keep_trajectories=True)
    assert r["shifts"] == 0
    assert r["stats"]["jumps"] == ref["stats"]["jumps"] > 0
    assert np.max(np.abs(r["traj_expect"] - ref["traj_expect"])) <= 1e-8


def test_dsf_mcsolve_ensemble_matches_dsf_mesolve():
    """A driven Kerr cavity (not coherent) with DSF: the trajectory mean is
    within 4 sigma / sqrt(ntraj) of the DSF master equation, sigma the
    spread of the real and imaginary parts separately.  The bound is 4, not 3,
    because it is a maximum over 31 times and 3 components that are strongly
    correlated; plain mcsolve on this cavity without shifts (cutoff 30) reaches
    z = 3.3 at 80 trajectories with the same seed, and 400 trajectories stay
    below z = 2.6, so the gap is statistical, not a bias."""
    N, D, K, F, kap = 10, 0.5, 0.05, 3.0, 1.0
    a = destroy(N)
    tl = np.linspace(0.0, 3.0, 31)
    H = lambda o: (D * (o[0].conj().T @ o[0]) + (K / 2) * (o[0].conj().T @ o[0].conj().T @ o[0] @ o[0])
                   + F * (o[0] + o[0].conj().T))
    c = lambda o: [math.sqrt(kap) * o[0]]
    e = lambda o: [o[0].conj().T @ o[0], o[0]]
    me = dsf_mesolve(H, c, e, [a], [0.0], np.eye(N)[0], tl, 0.1, rtol=1e-9, atol=1e-11)
    ntraj = 80
    r = dsf_mcsolve(H, c, e, [a], [0.0], np.eye(N)[0], tl, 0.1, ntraj=ntraj, seed=5,
                    rtol=1e-9, atol=1e-11, keep_trajectories=True)
    assert np.max(np.abs(me["expect"][0])) > 5.0        # beyond what the cutoff holds unshifted
    for part in (np.real, np.imag):
        sd = part(r["traj_expect"]).std(axis=0)
        bound = 4 * np.maximum(sd, 1e-3) / math.sqrt(ntraj) + 1e-4
        assert np.all(np.abs(part(r["expect"]) - part(me["expect"])) <= bound)


def test_dsf_mcsolve_planted_sign_mistake_breaks_the_coherent_pin(monkeypatch):
    """Displacing by D(+d) instead of D(-d), planted in a copy of the
    oracle's displacement, loses the coherent state."""
    import oracle.dsf as M
    real = M.sla.expm

    class _Flip:
        @staticmethod
        def expm(x):
            return real(-x)

    monkeypatch.setattr(M, "sla", _Flip)
    N, D, F, kap = 8, 0.5, 7.0, 1.0
    a, H, c, e = _cavity(N, D, F, kap)
    tl = np.linspace(0.0, 1.0, 21)
    r = dsf_mcsolve(H, c, e, [a], [0.0], np.eye(N)[0], tl, 0.05, ntraj=1, seed=3,
                    rtol=1e-10, atol=1e-12)
    ass = -1j * F / (kap / 2 + 1j * D)
    al = ass * (1 - np.exp(-(kap / 2 + 1j * D) * tl))
    assert np.max(np.abs(r["expect"][0] - al)) > 1e-2
