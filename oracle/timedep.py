"""Time-dependent Hamiltonians and the Schroedinger equation.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 2 builds time-dependent operators as a constant part plus operators
multiplied by scalar coefficient functions of t, H(t) = H0 + sum_k f_k(t) H_k
(QobjEvo); Sec. 3.4 solves the master equation of a driven optomechanical
system with the drive term f(t) (a + a^dag), f(t) = F cos(w_d t), and the
automatic-differentiation example of Sec. 5 uses the complex pair
f(t) = A exp(i w t) on a and its conjugate on a^dag.  Sec. 3.1 solves the
Schroedinger equation d psi/dt = -i H psi (sesolve).

Coefficient functions here take the form the library accepts,
    f(t) = A * env(t) * g(w t + phi),
    g = cos (kind "cos") or exp(i .) (kind "exp"),
    env(t) = exp(-(t - t0)^2 / (2 sigma^2)) if sigma > 0, else 1,
with a complex amplitude A.  The master equation keeps its form with H(t) in
place of H: the right-hand side at time t is the time-independent one for
the Hamiltonian H(t) (Sec. 3.4; the dissipator of lindblad.py), and a
trajectory evolves under H_eff(t) = H(t) - (i/2) sum_k C_k^dag C_k (Sec. 3.3).
"""
import math

import numpy as np
import scipy.sparse as sp

from .integrate import Stats, integrate
from .lindblad import effective_hamiltonian, lindblad_rhs, liouvillian, unvec, vec
from .mcsolve import trajectory
from .mesolve import initial_density_matrix
from .tableau import TABLEAUS


class Coef:
    """f(t) = amp * env(t) * g(omega t + phi)."""

    def __init__(self, kind="cos", amp=1.0, omega=0.0, phi=0.0, t0=0.0, sigma=0.0):
        if kind not in ("cos", "exp"):
            raise ValueError(kind)
        self.kind, self.amp, self.omega, self.phi = kind, complex(amp), float(omega), float(phi)
        self.t0, self.sigma = float(t0), float(sigma)

    def __call__(self, t):
        env = math.exp(-(t - self.t0) ** 2 / (2.0 * self.sigma ** 2)) if self.sigma > 0 else 1.0
        x = self.omega * t + self.phi
        g = math.cos(x) if self.kind == "cos" else complex(math.cos(x), math.sin(x))
        return self.amp * env * g


def hamiltonian_at(H0, terms, t):
    """H(t) = H0 + sum_k f_k(t) H_k for terms = [(H_k, f_k), ...]."""
    H = sp.csr_matrix(H0, dtype=np.complex128)
    for Hk, fk in terms:
        H = H + fk(t) * sp.csr_matrix(Hk, dtype=np.complex128)
    return sp.csr_matrix(H)


def mesolve_td(H0, terms, c_ops, e_ops, state0, tlist, method="tsit5", rtol=1e-8, atol=1e-10,
               rhs="product", fixed_dt=None, dt0=0.0, save_states=False, max_steps=10_000_000):
    """The master equation with H(t).  rhs = "product": the matrix-product
    right-hand side of lindblad.py for H(t); rhs = "liouvillian": the
    superoperator of H0 and the collapse operators plus f_k(t) times the
    superoperator of H_k alone (no collapse operators).  Returns
    dict(expect, states, stats) as mesolve."""
    tab = TABLEAUS[method]
    rho0 = initial_density_matrix(state0)
    n = rho0.shape[0]
    tlist = np.asarray(tlist, dtype=np.float64)
    if rhs == "liouvillian":
        L0 = liouvillian(H0, c_ops)
        Lk = [(liouvillian(Hk, []), fk) for Hk, fk in terms]

        def f(t, y):
            out = L0 @ y
            for L, fk in Lk:
                out = out + fk(t) * (L @ y)
            return out
    else:
        def f(t, y):
            return vec(lindblad_rhs(hamiltonian_at(H0, terms, t), c_ops, unvec(y, n)))

    n_e = len(e_ops)
    expect = np.zeros((n_e, len(tlist)), dtype=np.complex128)
    states = np.zeros((len(tlist), n, n), dtype=np.complex128) if save_states else None

    def on_save(idx, t, y):
        rho = unvec(y, n)
        for k, O in enumerate(e_ops):
            expect[k, idx] = np.trace(np.asarray(O @ rho))
        if states is not None:
            states[idx] = rho

    st = integrate(f, vec(rho0), tlist, tab, rtol, atol, on_save, dt0=dt0, fixed_dt=fixed_dt,
                   max_steps=max_steps)
    return dict(expect=expect, states=states, stats=st.as_dict())


def mcsolve_td(H0, terms, c_ops, e_ops, psi0, tlist, ntraj, seed, method="tsit5", rtol=1e-8,
               atol=1e-10, fixed_dt=None, dt0=0.0, keep_trajectories=False):
    """Trajectories under H_eff(t) = H_eff0 + sum_k f_k(t) H_k, with the jump
    rules of mcsolve.py.  Returns dict(expect, traj_expect?, jump_times,
    jump_channels, stats)."""
    Heff0 = effective_hamiltonian(H0, c_ops)
    Hs = [(sp.csr_matrix(Hk, dtype=np.complex128), fk) for Hk, fk in terms]

    def heff_apply(t, psi):
        out = Heff0 @ psi
        for Hk, fk in Hs:
            out = out + fk(t) * (Hk @ psi)
        return out
    tlist = np.asarray(tlist, dtype=np.float64)
    st = Stats()
    per, jt, jc = [], [], []
    for j in range(ntraj):
        ex, times, chans = trajectory(heff_apply, c_ops, e_ops, psi0, tlist, seed, j, method, rtol,
                                      atol, fixed_dt, dt0, st)
        per.append(ex)
        jt.append(times)
        jc.append(chans)
    per = np.array(per)
    out = dict(expect=per.mean(axis=0), jump_times=jt, jump_channels=jc, stats=st.as_dict())
    if keep_trajectories:
        out["traj_expect"] = per
    return out


def sesolve(H0, terms, e_ops, psi0, tlist, method="tsit5", rtol=1e-8, atol=1e-10, fixed_dt=None,
            dt0=0.0, save_states=False):
    """d psi/dt = -i H(t) psi (Sec. 3.1) with <psi|O|psi>/<psi|psi> at each
    time of tlist.  Returns dict(expect, states[t] (kets) or None, stats)."""
    tab = TABLEAUS[method]
    H0 = sp.csr_matrix(H0, dtype=np.complex128)
    Hs = [(sp.csr_matrix(Hk, dtype=np.complex128), fk) for Hk, fk in terms]

    def f(t, psi):
        out = H0 @ psi
        for Hk, fk in Hs:
            out = out + fk(t) * (Hk @ psi)
        return -1j * out
    tlist = np.asarray(tlist, dtype=np.float64)
    psi0 = np.asarray(psi0, dtype=np.complex128)
    expect = np.zeros((len(e_ops), len(tlist)), dtype=np.complex128)
    states = np.zeros((len(tlist), len(psi0)), dtype=np.complex128) if save_states else None

    def on_save(idx, t, psi):
        nrm = np.vdot(psi, psi)
        for k, O in enumerate(e_ops):
            expect[k, idx] = np.vdot(psi, O @ psi) / nrm
        if states is not None:
            states[idx] = psi

    st = integrate(f, psi0, tlist, tab, rtol, atol, on_save, dt0=dt0, fixed_dt=fixed_dt)
    return dict(expect=expect, states=states, stats=st.as_dict())
