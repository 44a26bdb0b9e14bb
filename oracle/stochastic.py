"""ssesolve: the stochastic Schroedinger equation under homodyne detection.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 3.5 writes the equation in Ito form,
    d psi = -i K psi dt + sum_n M_n psi dW_n,
    K   = H + i sum_n ( e_n/2 S_n - 1/2 S_n^dag S_n - e_n^2/8 ),
    M_n = S_n - e_n/2,   e_n = <psi| S_n + S_n^dag |psi>,
with real Wiener increments (E[dW_n] = 0, E[dW_n^2] = dt), and the homodyne
current J_n = e_n + dW_n/dt.  So -i K psi = A psi + sum_n (e_n/2) S_n psi -
sum_n (e_n^2/8) psi with A = -i H - 1/2 sum_n S_n^dag S_n.

Readings where the paper is silent (the library implements the same):
  * integrator: Euler-Maruyama with a fixed step dt, each step clamped to
    land on the next tlist time (the landing rule of integrate.py); e_n and
    both operator products are taken at the step's start;
  * the state is renormalised after every step (the equation conserves the
    norm, the scheme does not), so e_n is always evaluated on a unit vector;
  * Wiener increments dW_n = sqrt(h) z with z standard normal by the
    Box-Muller transform (Box & Muller, 1958) of two uniforms of the
    trajectory's Philox stream: draws 2j and 2j + 1 with
    j = step * n_sc + n give u1, u2 and z = sqrt(-2 ln u1) cos(2 pi u2);
  * recorded at every tlist time t_i: <psi|O|psi>/<psi|psi> and J_n of the
    last step that ended at or before t_i (at t_0: e_n(psi0));
  * ensemble outputs are arithmetic means over trajectories.
"""
import math

import numpy as np
import scipy.sparse as sp

from .integrate import LAND_ULPS
from .philox import uniform


def normal(seed, traj, j):
    """The j-th standard normal of trajectory traj (Box-Muller, cosine branch)."""
    u1 = uniform(seed, traj, 2 * j)
    u2 = uniform(seed, traj, 2 * j + 1)
    return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


def sse_trajectory(H, sc_ops, e_ops, psi0, tlist, dt, seed, traj):
    """One trajectory.  Returns (expect[k, t], measurement[n, t])."""
    H = sp.csr_matrix(H, dtype=np.complex128)
    S = [sp.csr_matrix(s, dtype=np.complex128) for s in sc_ops]
    A = -1j * H
    for s in S:
        A = A - 0.5 * (s.conj().T @ s)
    A = sp.csr_matrix(A)
    nsc = len(S)
    psi = np.asarray(psi0, dtype=np.complex128).copy()
    tlist = np.asarray(tlist, dtype=np.float64)
    expect = np.zeros((len(e_ops), len(tlist)), dtype=np.complex128)
    meas = np.zeros((nsc, len(tlist)))

    def save(idx, js):
        nrm = np.vdot(psi, psi)
        for k, O in enumerate(e_ops):
            expect[k, idx] = np.vdot(psi, O @ psi) / nrm
        meas[:, idx] = js

    e0 = [2.0 * float(np.vdot(psi, s @ psi).real) for s in S]
    save(0, e0)
    t = float(tlist[0])
    step = 0
    js = e0
    for idx in range(1, len(tlist)):
        t_target = float(tlist[idx])
        while t < t_target:
            land = dt >= (t_target - t) - LAND_ULPS * 2.0 ** -52 * max(1.0, abs(t_target))
            h = (t_target - t) if land else dt
            spsi = [s @ psi for s in S]
            e = [2.0 * float(np.vdot(psi, v).real) for v in spsi]
            dW = [math.sqrt(h) * normal(seed, traj, step * nsc + n) for n in range(nsc)]
            drift = A @ psi
            for n in range(nsc):
                drift = drift + (e[n] / 2.0) * spsi[n] - (e[n] ** 2 / 8.0) * psi
            new = psi + h * drift
            for n in range(nsc):
                new = new + dW[n] * (spsi[n] - (e[n] / 2.0) * psi)
            psi = new / math.sqrt(float(np.vdot(new, new).real))
            js = [e[n] + dW[n] / h for n in range(nsc)]
            t = t_target if land else t + h
            step += 1
        save(idx, js)
    return expect, meas


def ssesolve(H, sc_ops, e_ops, psi0, tlist, dt, ntraj, seed, keep_trajectories=False):
    """Ensemble of trajectories 0..ntraj-1.  Returns dict(expect, measurement
    (means over trajectories), traj_expect?, traj_measurement?)."""
    ex, ms = [], []
    for j in range(ntraj):
        a, b = sse_trajectory(H, sc_ops, e_ops, psi0, tlist, dt, seed, j)
        ex.append(a)
        ms.append(b)
    ex, ms = np.array(ex), np.array(ms)
    out = dict(expect=ex.mean(axis=0), measurement=ms.mean(axis=0))
    if keep_trajectories:
        out["traj_expect"] = ex
        out["traj_measurement"] = ms
    return out


def sme_trajectory(H, c_ops, sc_ops, e_ops, rho0, tlist, dt, seed, traj):
    """One trajectory of the stochastic master equation of Sec. 3.5,
        d rho = -i[H, rho] dt + sum_i D[C_i] rho dt + sum_n D[S_n] rho dt
                + sum_n H[S_n] rho dW_n,
        H[O] rho = O rho + rho O^dag - Tr(O rho + rho O^dag) rho,
    with J_n = Tr(S_n rho + rho S_n^dag) + dW_n/dt.  Euler-Maruyama with the
    steps, landing and Wiener increments of sse_trajectory; no
    renormalisation (the scheme keeps Tr rho = 1 up to rounding, since
    Tr H[S] rho = 0 at unit trace).  Returns (expect[k, t], measurement[n, t])."""
    from .lindblad import lindblad_rhs
    S = [np.asarray(sp.csr_matrix(s, dtype=np.complex128).todense()) for s in sc_ops]
    C = [sp.csr_matrix(c, dtype=np.complex128) for c in list(c_ops) + list(sc_ops)]
    Hm = sp.csr_matrix(H, dtype=np.complex128)
    nsc = len(S)
    rho = np.array(rho0, dtype=np.complex128)
    tlist = np.asarray(tlist, dtype=np.float64)
    expect = np.zeros((len(e_ops), len(tlist)), dtype=np.complex128)
    meas = np.zeros((nsc, len(tlist)))

    def hom(Sn, r):
        v = Sn @ r + r @ Sn.conj().T
        return v, float(np.trace(v).real)

    def save(idx, js):
        for k, O in enumerate(e_ops):
            expect[k, idx] = np.trace(np.asarray(O @ rho))
        meas[:, idx] = js

    js = [hom(s, rho)[1] for s in S]
    save(0, js)
    t = float(tlist[0])
    step = 0
    for idx in range(1, len(tlist)):
        t_target = float(tlist[idx])
        while t < t_target:
            land = dt >= (t_target - t) - LAND_ULPS * 2.0 ** -52 * max(1.0, abs(t_target))
            h = (t_target - t) if land else dt
            dW = [math.sqrt(h) * normal(seed, traj, step * nsc + n) for n in range(nsc)]
            new = rho + h * np.asarray(lindblad_rhs(Hm, C, rho))
            trs = []
            for n in range(nsc):
                v, tr = hom(S[n], rho)
                trs.append(tr)
                new = new + dW[n] * (v - tr * rho)
            rho = new
            js = [trs[n] + dW[n] / h for n in range(nsc)]
            t = t_target if land else t + h
            step += 1
        save(idx, js)
    return expect, meas


def smesolve(H, c_ops, sc_ops, e_ops, state0, tlist, dt, ntraj, seed, keep_trajectories=False):
    """Ensemble of SME trajectories 0..ntraj-1 from a ket or a density matrix.
    Returns dict(expect, measurement, traj_expect?, traj_measurement?)."""
    st = np.asarray(state0, dtype=np.complex128)
    rho0 = np.outer(st, st.conj()) if st.ndim == 1 else st
    ex, ms = [], []
    for j in range(ntraj):
        a, b = sme_trajectory(H, c_ops, sc_ops, e_ops, rho0, tlist, dt, seed, j)
        ex.append(a)
        ms.append(b)
    ex, ms = np.array(ex), np.array(ms)
    out = dict(expect=ex.mean(axis=0), measurement=ms.mean(axis=0))
    if keep_trajectories:
        out["traj_expect"] = ex
        out["traj_measurement"] = ms
    return out
