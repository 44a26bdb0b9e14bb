"""Pins of the stationary-state oracle (oracle/steadystate.py): the driven
damped cavity's coherent steady state and the paper's photon number
F^2 / (D^2 + k^2/4) (Sec. 5), the thermal occupation, the residual and
invariants, long-time mesolve, a random system's SVD null space, the
derivative in the drive frequency printed in Sec. 5, and the Fourier components of a cos-driven
cavity against its exact periodic solution (Appendix A)."""
import math

import numpy as np
import scipy.sparse as sp

from oracle.lindblad import liouvillian, vec
from oracle.mesolve import mesolve
from oracle.steadystate import steadystate, steadystate_fourier


def destroy(N):
    return sp.diags(np.sqrt(np.arange(1, N)), 1, format="csr", dtype=complex)


def test_driven_cavity_steady_state_closed_form():
    N, D, F, kap = 40, 1.0, 0.5, 0.2
    a = destroy(N)
    ad = a.conj().T
    H = D * (ad @ a) + F * (a + ad)
    rho = steadystate(H, [math.sqrt(kap) * a])
    ass = -1j * F / (kap / 2 + 1j * D)
    assert abs(np.trace(a @ rho) - ass) <= 1e-12
    assert abs(np.trace(ad @ a @ rho) - F ** 2 / (D ** 2 + kap ** 2 / 4)) <= 1e-12
    assert abs(np.trace(rho) - 1) <= 1e-13
    assert np.max(np.abs(rho - rho.conj().T)) <= 1e-13
    assert np.min(np.linalg.eigvalsh((rho + rho.conj().T) / 2)) >= -1e-12
    assert np.max(np.abs(liouvillian(H, [math.sqrt(kap) * a]) @ vec(rho))) <= 1e-12


def test_thermal_occupation_and_long_time_mesolve():
    N, w, kap, nth = 40, 1.0, 0.3, 0.4
    a = destroy(N)
    ad = a.conj().T
    H = w * (ad @ a)
    c = [math.sqrt(kap * (1 + nth)) * a, math.sqrt(kap * nth) * ad]
    rho = steadystate(H, c)
    assert abs(np.trace(ad @ a @ rho) - nth) <= 1e-9      # thermal tail beyond N = 40 only
    r = mesolve(H, c, [ad @ a], np.eye(N)[0], [0.0, 120.0], rtol=1e-10, atol=1e-12)
    assert abs(r["expect"][0, -1] - np.trace(ad @ a @ rho)) <= 1e-8


def test_fourier_components_of_a_cos_driven_cavity():
    """H = D a'a + F cos(w t)(a + a'), loss sqrt(k) a: the periodic steady
    state is coherent with alpha(t) = A+ e^{i w t} + A- e^{-i w t},
    A+- = -i (F/2) / (z +- i w), z = i D + k/2, so <a> has only the n = +-1
    components and the period-averaged photon number is |A+|^2 + |A-|^2."""
    N, D, kap, F, w = 30, 0.7, 0.5, 0.2, 1.1
    a = destroy(N)
    ad = a.conj().T
    comps = steadystate_fourier(D * (ad @ a), [math.sqrt(kap) * a], a + ad, F, w, 4)
    z = 1j * D + kap / 2
    Ap, Am = -0.5j * F / (z + 1j * w), -0.5j * F / (z - 1j * w)
    assert abs(np.trace(a @ comps[1]) - Ap) <= 1e-10
    assert abs(np.trace(a @ comps[-1]) - Am) <= 1e-10
    assert abs(np.trace(a @ comps[0])) <= 1e-10
    assert abs(np.trace(ad @ a @ comps[0]) - (abs(Ap) ** 2 + abs(Am) ** 2)) <= 1e-10
    assert abs(np.trace(comps[0]) - 1) <= 1e-12


def test_fourier_without_drive_is_the_steady_state():
    N, D, kap = 12, 0.9, 0.4
    a = destroy(N)
    ad = a.conj().T
    H = D * (ad @ a) + 0.3 * (a + ad)
    c = [math.sqrt(kap) * a]
    comps = steadystate_fourier(H, c, a + ad, 0.0, 1.3, 2)
    assert np.max(np.abs(comps[0] - steadystate(H, c))) <= 1e-12
    assert all(np.max(np.abs(comps[k])) <= 1e-12 for k in (-2, -1, 1, 2))


def test_fourier_components_match_the_long_time_periodic_solution():
    """A nonlinear case with no closed form: a Kerr cavity under F cos(w t)(a + a').
    After the transient has decayed, rho(t) is periodic, and its Fourier
    coefficients avg_t rho(t) e^{-i n w t} over one period (the trapezoid sum
    on M equispaced points is exact for harmonics below M) must equal the
    rho_n of the linear system.  The time-dependent mesolve oracle is pinned
    separately, so this checks the block structure, the -i n w shift and the
    trace row."""
    from oracle.timedep import Coef, mesolve_td
    N, D, K, kap, F, w = 10, 0.4, 0.3, 0.8, 0.35, 1.3
    a = destroy(N)
    ad = a.conj().T
    H0 = (D * (ad @ a) + K * (ad @ ad @ a @ a)).tocsr()
    X = (a + ad).tocsr()
    c = [math.sqrt(kap) * a]
    comps = steadystate_fourier(H0, c, X, F, w, 10)
    P, M = 2 * math.pi / w, 32
    T = 16.0 * P                              # e^{-kap T / 2} < 1e-13
    tl = [0.0] + [T + j * P / M for j in range(M)]
    r = mesolve_td(H0, [(X, Coef("cos", F, w))], c, [], np.eye(N)[0], tl,
                   rtol=1e-11, atol=1e-13, save_states=True)
    rhos = [np.asarray(s).reshape((N, N), order="F") if np.ndim(s) == 1 else np.asarray(s)
            for s in r["states"][1:]]
    for k in (-2, -1, 0, 1, 2):
        avg = sum(rho * np.exp(-1j * k * w * t) for rho, t in zip(rhos, tl[1:])) / M
        assert np.max(np.abs(avg - comps[k])) <= 1e-8, k
    assert np.max(np.abs(comps[1] - comps[-1].conj().T)) <= 1e-13   # rho(t) Hermitian


def test_photon_number_derivative_in_the_drive_frequency():
    """Sec. 5's driven oscillator in the frame rotating at w_d (D = w_c - w_d):
    a central difference of the steady-state photon number in w_d equals the
    printed derivative 2 F^2 D / (D^2 + g^2/4)^2, at several detunings."""
    N, wc, F, g, h = 40, 1.0, 0.3, 0.5, 1e-4
    a = destroy(N)
    ad = a.conj().T

    def n_ss(wd):
        rho = steadystate((wc - wd) * (ad @ a) + F * (a + ad), [math.sqrt(g) * a])
        return np.trace(ad @ a @ rho).real

    for wd in (0.6, 0.9, 1.0, 1.2):
        D = wc - wd
        fd = (n_ss(wd + h) - n_ss(wd - h)) / (2 * h)
        exact = 2 * F ** 2 * D / (D ** 2 + g ** 2 / 4) ** 2
        assert abs(fd - exact) <= 1e-6 * max(1.0, abs(exact)), wd


def test_random_system_against_the_null_space():
    """A random 5-level system with three random collapse operators: the
    direct solve equals the null vector of the full Liouvillian (an SVD),
    scaled to unit trace, and that null space is one-dimensional."""
    import scipy.linalg as sla
    rng = np.random.default_rng(7)
    n = 5
    M = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    H = sp.csr_matrix((M + M.conj().T) / 2)
    cs = [sp.csr_matrix(0.5 * (rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)))) for _ in range(3)]
    rho = steadystate(H, cs)
    L = np.asarray(liouvillian(H, cs).todense())
    ns = sla.null_space(L, rcond=1e-10)
    assert ns.shape[1] == 1
    v = ns[:, 0].reshape((n, n), order="F")
    v = v / np.trace(v)
    assert np.max(np.abs(rho - v)) <= 1e-12
