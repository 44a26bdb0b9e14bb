"""Dynamical shifted Fock (DSF) master equation (Sec. 3.6; Appendix B,
Algorithm 1): the state is kept in a frame displaced by a tracked coherence
alpha_k for each DSF mode, so that a small Fock cutoff describes the
fluctuations around a large coherent amplitude.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings taken here:
  * H, the collapse operators and the observables are functions of the DSF
    mode operators (the paper passes them as functions of op_list).  The
    operator update D(-d) X D(d) of Algorithm 1 is taken as rebuilding each
    operator with a_k replaced by a_k + alpha_k I, which is the identity
    D(-a) a D(a) = a + a before truncation.
  * The coherence of mode k at a check is Tr(rho (a_k + alpha_k)), so the
    shift is d_k = Tr(rho a_k) in the current frame.  When |d_k| exceeds the
    threshold, rho <- D_k(-d_k) rho D_k(d_k), with D_k(b) = exp(b a_k^dag -
    conj(b) a_k) exponentiated in the truncated space, and alpha_k += d_k.
  * Checks happen at the times of tlist (the fixed step of Algorithm 1 is
    tlist's spacing); between checks the adaptive mesolve of mesolve.py
    integrates.  Observables are recorded at a check before its
    displacement.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .integrate import Stats
from .lindblad import effective_hamiltonian
from .mcsolve import trajectory
from .mesolve import mesolve


def dsf_mesolve(H_fn, c_fn, e_fn, op_list, alpha0, state0, tlist, threshold,
                method="tsit5", rtol=1e-8, atol=1e-10):
    """H_fn(ops), c_fn(ops), e_fn(ops): the Hamiltonian, the list of collapse
    operators and the list of observables built from ops = [a_k + alpha_k I].
    op_list: the truncated annihilation operators a_k of the DSF modes on the
    full space.  alpha0: initial coherences; state0: the initial state in the
    frame displaced by alpha0 (a ket or a density matrix).
    Returns dict(expect[k, t], alpha[k, t] (the coherences tracked at each
    time, after that time's displacement), shifts (displacements applied))."""
    ops = [sp.csr_matrix(a, dtype=np.complex128) for a in op_list]
    dim = ops[0].shape[0]
    eye = sp.identity(dim, dtype=np.complex128, format="csr")
    alpha = np.array(alpha0, dtype=np.complex128)
    tlist = np.asarray(tlist, dtype=np.float64)
    state = np.asarray(state0, dtype=np.complex128)
    rho = np.outer(state, state.conj()) if state.ndim == 1 else state.copy()
    dense_a = [a.toarray() for a in ops]

    def shifted():
        return [a + al * eye for a, al in zip(ops, alpha)]

    def expect_now():
        return [np.trace(np.asarray(O.todense() if hasattr(O, "todense") else O) @ rho)
                for O in e_fn(shifted())]

    n_e = len(e_fn(shifted()))
    expect = np.zeros((n_e, len(tlist)), dtype=np.complex128)
    alphas = np.zeros((len(ops), len(tlist)), dtype=np.complex128)
    shifts = 0
    for idx in range(len(tlist)):
        if idx > 0:
            cur = shifted()
            r = mesolve(H_fn(cur), c_fn(cur), [], rho, [tlist[idx - 1], tlist[idx]],
                        method=method, rtol=rtol, atol=atol, save_states=True)
            rho = r["states"][-1]
        expect[:, idx] = expect_now()
        for k, a in enumerate(dense_a):
            d = np.trace(a @ rho)
            if abs(d) > threshold:
                D = sla.expm(-d * a.conj().T + np.conj(d) * a)   # D_k(-d)
                rho = D @ rho @ D.conj().T
                alpha[k] += d
                shifts += 1
        alphas[:, idx] = alpha
    return dict(expect=expect, alpha=alphas, shifts=shifts)


def dsf_mcsolve(H_fn, c_fn, e_fn, op_list, alpha0, psi0, tlist, threshold, ntraj, seed,
                method="tsit5", rtol=1e-8, atol=1e-10, keep_trajectories=False):
    """Dynamical shifted Fock on quantum trajectories (Sec. 3.6 applies
    Algorithm 1 of Appendix B to both solvers).  Each trajectory carries its
    own frame alpha^(j): between checks it is the trajectory of mcsolve.py
    under H_eff and the collapse operators built from a_k + alpha_k^(j) I
    (its random stream and threshold carried over from check to check); at
    each time of tlist the observables are recorded, then for each mode
    d_k = <psi|a_k|psi>/<psi|psi> and, when |d_k| > threshold, the ket is
    displaced, psi <- D_k(-d_k) psi, and alpha_k^(j) += d_k.  The readings of
    dsf_mesolve (operator rebuild, displacement, check times) apply.
    Returns dict(expect = mean over trajectories of the normalised
    observables, traj_expect?, shifts, stats)."""
    ops = [sp.csr_matrix(a, dtype=np.complex128) for a in op_list]
    dim = ops[0].shape[0]
    eye = sp.identity(dim, dtype=np.complex128, format="csr")
    dense_a = [a.toarray() for a in ops]
    tlist = np.asarray(tlist, dtype=np.float64)
    nt = len(tlist)
    n_e = len(e_fn(ops))
    st = Stats()
    per = []
    shifts = 0
    for j in range(ntraj):
        alpha = np.array(alpha0, dtype=np.complex128)
        psi = np.array(psi0, dtype=np.complex128)
        state = None
        ex = np.zeros((n_e, nt), dtype=np.complex128)
        for idx in range(nt):
            cur = [a + al * eye for a, al in zip(ops, alpha)]
            if idx > 0:
                c_cur = c_fn(cur)
                out = {}
                trajectory(effective_hamiltonian(H_fn(cur), c_cur), c_cur, [], psi,
                           [tlist[idx - 1], tlist[idx]], seed, j, method, rtol, atol, stats=st,
                           resume=state, state_out=out)
                psi = out["psi"]
                state = {"draws": out["draws"], "r": out["r"]}
            nrm = np.vdot(psi, psi)
            for k, O in enumerate(e_fn(cur)):
                ex[k, idx] = np.vdot(psi, O @ psi) / nrm
            for k, a in enumerate(dense_a):
                d = np.vdot(psi, a @ psi) / nrm
                if abs(d) > threshold:
                    psi = sla.expm(-d * a.conj().T + np.conj(d) * a) @ psi   # D_k(-d)
                    alpha[k] += d
                    shifts += 1
        per.append(ex)
    per = np.array(per)
    out = dict(expect=per.mean(axis=0), shifts=shifts, stats=st.as_dict())
    if keep_trajectories:
        out["traj_expect"] = per
    return out
