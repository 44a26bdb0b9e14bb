"""Seeded synthetic systems shaped like the paper's workloads.

Each builder returns a `System`: H, collapse operators, observables (scipy CSR,
complex128), an initial ket, a time grid and the tolerances to solve with.
The parameters follow the worked examples of the paper (Sec. 3.2-3.3
Jaynes-Cummings, Sec. 4 damped oscillator and 2D dissipative Ising, Sec. 6
driven Kerr oscillator and 1D Ising chain); where the paper prints no value
the stated synthetic stand-in is used and the seed is fixed here.
"""
from dataclasses import dataclass, field

import numpy as np

from .operators import (coherent, dag, destroy, fock, qeye, sigmam, sigmap, sigmax,
                        sigmay, sigmaz, site_operator, tensor)


@dataclass
class System:
    name: str
    H: object
    c_ops: list
    e_ops: list
    psi0: np.ndarray
    tlist: np.ndarray
    rtol: float = 1e-8
    atol: float = 1e-10
    method: str = "tsit5"
    params: dict = field(default_factory=dict)

    @property
    def n(self):
        return self.H.shape[0]


def driven_cavity(N=20, delta=1.0, F=0.5, kappa=0.2, alpha0=2.0, t_end=20.0, nt=201):
    """Driven damped cavity H = delta a'a + F (a + a'), C = sqrt(kappa) a,
    rho0 = coherent(alpha0); e_ops {a'a, a}.  Closed form: the state stays
    coherent with alpha_ss = -iF / (kappa/2 + i delta) (cf. Sec. 5, Fig. 6)."""
    a = destroy(N)
    H = delta * (dag(a) @ a) + F * (a + dag(a))
    return System("driven_cavity", H.tocsr(), [np.sqrt(kappa) * a], [dag(a) @ a, a],
                  coherent(N, alpha0), np.linspace(0.0, t_end, nt), 1e-8, 1e-10, "tsit5",
                  dict(N=N, delta=delta, F=F, kappa=kappa, alpha0=alpha0))


def jaynes_cummings(N=40, wc=1.0, wq=1.0, g=0.1, kappa=0.05, gamma=0.02, nt=1000,
                    t_end=None):
    """Jaynes-Cummings model, Sec. 3.1-3.3: cavity (x) qubit, cavity index most
    significant.  rho0 = |0> (x) |e> (basis(2,0) with sigmaz = diag(1,-1)).
    e_ops {a'a, sigma+ sigma-}.  Default grid range(0, 10 pi / g, nt)."""
    if t_end is None:
        t_end = 10 * np.pi / g
    a = tensor(destroy(N), qeye(2))
    sz = tensor(qeye(N), sigmaz())
    sm = tensor(qeye(N), sigmam())
    sp_ = tensor(qeye(N), sigmap())
    H = wc * (dag(a) @ a) + (wq / 2) * sz + g * (a @ sp_ + dag(a) @ sm)
    c_ops = [np.sqrt(kappa) * a, np.sqrt(gamma) * sm]
    psi0 = np.kron(fock(N, 0), fock(2, 0))
    return System("jaynes_cummings", H.tocsr(), c_ops, [dag(a) @ a, sp_ @ sm], psi0,
                  np.linspace(0.0, t_end, nt), 1e-8, 1e-10, "tsit5",
                  dict(N=N, wc=wc, wq=wq, g=g, kappa=kappa, gamma=gamma))


def ising_chain(n_spins=10, J=1.0, h=None, gamma=0.1, seed=3, t_end=10.0, nt=100,
                rtol=1e-8, atol=1e-10):
    """Dissipative transverse-field Ising chain with open boundary,
    H = J sum_i sz_i sz_{i+1} + h sum_i sx_i, C_i = sqrt(gamma) sigma-_i (the
    2D example of Sec. 4 restricted to a chain).  h is one scalar drawn from
    U[0.5, 1.5] with `seed` unless given.  rho0 = all spins excited (basis
    index 0, as fock(2^N, 0) in Sec. 4).  e_ops {Sx, Sy, Sz} totals."""
    if h is None:
        h = float(np.random.default_rng(seed).uniform(0.5, 1.5))
    sx = [site_operator(sigmax(), i, n_spins) for i in range(n_spins)]
    sy = [site_operator(sigmay(), i, n_spins) for i in range(n_spins)]
    sz = [site_operator(sigmaz(), i, n_spins) for i in range(n_spins)]
    H = sum(J * (sz[i] @ sz[i + 1]) for i in range(n_spins - 1)) + sum(h * s for s in sx)
    c_ops = [np.sqrt(gamma) * site_operator(sigmam(), i, n_spins) for i in range(n_spins)]
    e_ops = [sum(sx), sum(sy), sum(sz)]
    e_ops = [e.tocsr() for e in e_ops]
    psi0 = fock(2 ** n_spins, 0)
    H = H.tocsr()
    H.eliminate_zeros()
    return System("ising_chain", H, [c.tocsr() for c in c_ops], e_ops, psi0,
                  np.linspace(0.0, t_end, nt), rtol, atol, "tsit5",
                  dict(n_spins=n_spins, J=J, h=h, gamma=gamma))


def kerr_cavity(N, delta, K, F, kappa, t_end=50.0, nt=101, rtol=1e-8, atol=1e-10):
    """Driven Kerr cavity H = delta a'a + (K/2) a'a'aa + F (a + a'), C = sqrt(kappa) a,
    rho0 = vacuum, e_ops {a'a, a} (Sec. 6 benchmark model, sign as configured)."""
    a = destroy(N)
    ad = dag(a)
    H = delta * (ad @ a) + (K / 2) * (ad @ ad @ a @ a) + F * (a + ad)
    H = H.tocsr()
    H.eliminate_zeros()
    return System("kerr_cavity", H, [np.sqrt(kappa) * a], [ad @ a, a], fock(N, 0),
                  np.linspace(0.0, t_end, nt), rtol, atol, "tsit5",
                  dict(N=N, delta=delta, K=K, F=F, kappa=kappa))


def kerr_sweep(n_inst=1024, seed=4, n_min=10, n_max=60, t_end=50.0, nt=101,
               rtol=1e-8, atol=1e-10):
    """Parameter sweep of uneven Kerr cavities: N ~ U{n_min..n_max},
    delta ~ U[-2,2], K ~ U[0.01,0.5], F ~ U[0.1,2], kappa ~ U[0.05,0.5]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_inst):
        N = int(rng.integers(n_min, n_max + 1))
        delta = float(rng.uniform(-2, 2))
        K = float(rng.uniform(0.01, 0.5))
        F = float(rng.uniform(0.1, 2))
        kappa = float(rng.uniform(0.05, 0.5))
        out.append(kerr_cavity(N, delta, K, F, kappa, t_end, nt, rtol, atol))
    return out


def coupled_cavities(N1, N2, J, kappa1, kappa2, t_end=20.0, nt=101, rtol=1e-8, atol=1e-10):
    """Two cavities in the rotating frame, H = J (a'b + b'a), C = sqrt(k1) a,
    sqrt(k2) b, rho0 = |1> (x) |0>, e_ops {a'a, b'b}.  The single-excitation
    dynamics has a 2x2 closed form."""
    a = tensor(destroy(N1), qeye(N2))
    b = tensor(qeye(N1), destroy(N2))
    H = J * (dag(a) @ b + dag(b) @ a)
    H = H.tocsr()
    H.eliminate_zeros()
    psi0 = np.kron(fock(N1, 1), fock(N2, 0))
    return System("coupled_cavities", H, [np.sqrt(kappa1) * a, np.sqrt(kappa2) * b],
                  [dag(a) @ a, dag(b) @ b], psi0, np.linspace(0.0, t_end, nt), rtol, atol, "tsit5",
                  dict(N1=N1, N2=N2, J=J, kappa1=kappa1, kappa2=kappa2))


def damped_oscillator(N=20, omega=1.0, gamma=0.1, n0=3, t_end=10.0, nt=100):
    """The GPU example of Sec. 4: H = omega a'a, C = sqrt(gamma) a, psi0 = |3>,
    tlist = range(0, 10, 100), e_ops {a'a}.  <a'a>(t) = n0 exp(-gamma t)."""
    a = destroy(N)
    return System("damped_oscillator", (omega * (dag(a) @ a)).tocsr(), [np.sqrt(gamma) * a],
                  [dag(a) @ a], fock(N, n0), np.linspace(0.0, t_end, nt), 1e-8, 1e-10, "tsit5",
                  dict(N=N, omega=omega, gamma=gamma, n0=n0))


def thermal_oscillator(N=40, omega=1.0, kappa=0.3, nth=0.4, n0=2, t_end=8.0, nt=41):
    """Oscillator coupled to a thermal bath: C1 = sqrt(kappa (1+nth)) a,
    C2 = sqrt(kappa nth) a'.  <a'a>(t) = n0 e^{-kappa t} + nth (1 - e^{-kappa t})."""
    a = destroy(N)
    c_ops = [np.sqrt(kappa * (1 + nth)) * a, np.sqrt(kappa * nth) * dag(a)]
    return System("thermal_oscillator", (omega * (dag(a) @ a)).tocsr(), c_ops, [dag(a) @ a],
                  fock(N, n0), np.linspace(0.0, t_end, nt), 1e-9, 1e-11, "tsit5",
                  dict(N=N, omega=omega, kappa=kappa, nth=nth, n0=n0))


def two_level_decay(gamma=0.5, omega=0.0, t_end=10.0, nt=51):
    """Two-level atom H = omega/2 sigmaz, C = sqrt(gamma) sigma-, psi0 = |e>.
    Populations p_e(t) = exp(-gamma t); in a quantum trajectory the first jump
    happens where exp(-gamma t) equals the drawn threshold."""
    return System("two_level_decay", (omega / 2 * sigmaz()).tocsr(),
                  [np.sqrt(gamma) * sigmam()], [sigmap() @ sigmam(), sigmaz()], fock(2, 0),
                  np.linspace(0.0, t_end, nt), 1e-9, 1e-11, "tsit5",
                  dict(gamma=gamma, omega=omega))


def serving_mix(n_requests=200, seed=5, rate=100.0, ising_spins=(8, 14),
                ntraj=(100, 2000), cav=(4, 32), mesolve_frac=0.6):
    """Poisson stream of mixed requests: mesolve on coupled-cavity pairs with
    N1, N2 ~ U{cav}, J ~ U[0,1], kappa_i ~ U[0.01,0.3]; mcsolve on Ising chains
    with spins ~ U{ising_spins}, ntraj ~ U{ntraj}.  Returns a list of dicts with
    arrival time (s), kind, system and (for mcsolve) ntraj and seed."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for i in range(n_requests):
        t += float(rng.exponential(1.0 / rate))
        if rng.uniform() < mesolve_frac:
            N1 = int(rng.integers(cav[0], cav[1] + 1))
            N2 = int(rng.integers(cav[0], cav[1] + 1))
            sysm = coupled_cavities(N1, N2, float(rng.uniform(0, 1)),
                                    float(rng.uniform(0.01, 0.3)), float(rng.uniform(0.01, 0.3)))
            reqs.append(dict(arrival=t, kind="mesolve", system=sysm))
        else:
            ns = int(rng.integers(ising_spins[0], ising_spins[1] + 1))
            sysm = ising_chain(ns, seed=int(rng.integers(0, 2**31)), t_end=10.0, nt=101)
            reqs.append(dict(arrival=t, kind="mcsolve", system=sysm,
                             ntraj=int(rng.integers(ntraj[0], ntraj[1] + 1)),
                             seed=int(rng.integers(0, 2**63))))
    return reqs


CONFIGS = {
    "driven_cavity_n20": lambda: driven_cavity(),
    "jc_40x2": lambda: jaynes_cummings(),
    "ising10": lambda: ising_chain(10),
    "ising14": lambda: ising_chain(14),
}
