"""mcsolve: the Monte-Carlo wave-function method of Sec. 3.3.

Each trajectory evolves a ket under the non-Hermitian effective Hamiltonian
H_eff = H - (i/2) sum_k C_k^dag C_k, i.e. d psi/dt = -i H_eff psi, whose norm
decays.  A jump happens when the norm reaches a threshold drawn uniformly in
(0, 1); the channel k is drawn with probability
P_k = <psi|C_k^dag C_k|psi> / sum_j <psi|C_j^dag C_j|psi>;
the state becomes C_k psi / |C_k psi| and a new threshold is drawn.  The
ensemble average of the normalised expectation values estimates the master
equation solution.

Readings where the paper is silent (shared with the CUDA library):
  * the threshold compares the squared norm <psi|psi> with r;
  * the crossing time inside an accepted step [t, t+h] is located by the
    Illinois (modified regula falsi) method on g(tau) = ln|psi(t+tau)|^2 - ln r,
    psi(t+tau) being one RK step of size tau from the step's start; stop when
    the bracket is narrower than 1e-10 max(1, |t|) or after 30 evaluations;
    the jump is taken at the last evaluated point;
  * the channel is the smallest k with sum_{j<=k} p_j >= u sum_j p_j;
  * with no collapse operator the threshold is 0, so a trajectory never
    jumps (the Schroedinger equation);
  * draws per trajectory alternate: threshold, channel, threshold, ...
  * expectation values <psi|O|psi>/<psi|psi> are recorded at each tlist time
    and averaged arithmetically over trajectories.
"""
import math

import numpy as np

from .integrate import Stats, integrate, rk_step
from .lindblad import effective_hamiltonian
from .philox import uniform
from .tableau import TABLEAUS

ROOT_TOL = 1e-10
ROOT_MAX_ITERS = 30


def _norm2(psi):
    return float(np.vdot(psi, psi).real)


def trajectory(Heff, c_ops, e_ops, psi0, tlist, seed, traj_id, method="tsit5",
               rtol=1e-8, atol=1e-10, fixed_dt=None, dt0=0.0, stats=None,
               max_steps=10_000_000, resume=None, state_out=None):
    """One trajectory.  Returns (expect[k, t] complex, jump_times, jump_channels).

    resume: None, or dict(draws, r) to continue a trajectory whose random
    stream has already given `draws` numbers and whose current threshold is r
    (no new threshold is drawn at the start).  state_out: None, or a dict that
    receives psi (at the last time of tlist), draws and r, for resuming."""
    tab = TABLEAUS[method]
    st = stats if stats is not None else Stats()
    draws = [0 if resume is None else int(resume["draws"])]

    def draw():
        u = uniform(seed, traj_id, draws[0])
        draws[0] += 1
        return u

    if callable(Heff):       # time-dependent H_eff(t) applied to psi
        def f(t, psi):
            return -1j * Heff(t, psi)
    else:
        def f(t, psi):
            return -1j * (Heff @ psi)

    # without collapse operators there is no channel to jump to: the norm is
    # compared with a threshold of 0 (the first draw is still consumed)
    if resume is not None:
        r = [float(resume["r"])]
    else:
        r = [draw() if len(c_ops) > 0 else (draw(), 0.0)[1]]
    jump_times, jump_channels = [], []
    n_e = len(e_ops)
    expect = np.zeros((n_e, len(tlist)), dtype=np.complex128)

    def on_save(idx, t, psi):
        nrm = np.vdot(psi, psi)
        for k, O in enumerate(e_ops):
            expect[k, idx] = np.vdot(psi, O @ psi) / nrm
        if state_out is not None and idx == len(tlist) - 1:
            state_out["psi"] = np.array(psi, dtype=np.complex128)

    def after_accept(t, y, k1, h, t_new, y_new, k_last):
        if _norm2(y_new) >= r[0]:
            return None
        log_r = math.log(r[0])
        lo, g_lo = 0.0, math.log(_norm2(y)) - log_r
        hi, g_hi = h, math.log(_norm2(y_new)) - log_r
        tau, psi_tau = hi, y_new
        side = 0
        for _ in range(ROOT_MAX_ITERS):
            if hi - lo <= ROOT_TOL * max(1.0, abs(t)):
                break
            tau = (lo * g_hi - hi * g_lo) / (g_hi - g_lo)
            psi_tau, _ks = rk_step(f, t, y, tau, k1, tab)
            st.rhs_evals += tab.stages - 1
            g = math.log(_norm2(psi_tau)) - log_r
            if g > 0:
                lo, g_lo = tau, g
                if side == 1:
                    g_hi *= 0.5
                side = 1
            elif g < 0:
                hi, g_hi = tau, g
                if side == -1:
                    g_lo *= 0.5
                side = -1
            else:
                break
        t_star = t + tau
        weights = [_norm2(C @ psi_tau) for C in c_ops]
        total = sum(weights)
        u = draw()
        acc = 0.0
        k = len(weights) - 1
        for j, wj in enumerate(weights):
            acc += wj
            if acc >= u * total:
                k = j
                break
        psi_j = c_ops[k] @ psi_tau
        psi_j = psi_j / math.sqrt(weights[k])
        r[0] = draw()
        jump_times.append(t_star)
        jump_channels.append(k)
        st.jumps += 1
        st.rhs_evals += 1
        return t_star, psi_j, f(t_star, psi_j)

    integrate(f, np.asarray(psi0, dtype=np.complex128), tlist, tab, rtol, atol, on_save,
              dt0=dt0, fixed_dt=fixed_dt, max_steps=max_steps, after_accept=after_accept,
              stats=st)
    if state_out is not None:
        state_out["draws"] = draws[0]
        state_out["r"] = r[0]
    return expect, jump_times, jump_channels


def mcsolve(H, c_ops, e_ops, psi0, tlist, ntraj, seed, method="tsit5", rtol=1e-8,
            atol=1e-10, fixed_dt=None, dt0=0.0, traj_ids=None, keep_trajectories=False):
    """Ensemble of trajectories 0..ntraj-1 (or the given ids).  Returns
    dict(expect = mean over trajectories, traj_expect (optional), jump_times,
    jump_channels, stats)."""
    Heff = effective_hamiltonian(H, c_ops)
    tlist = np.asarray(tlist, dtype=np.float64)
    ids = list(range(ntraj)) if traj_ids is None else list(traj_ids)
    st = Stats()
    per = []
    jt, jc = [], []
    for j in ids:
        ex, times, chans = trajectory(Heff, c_ops, e_ops, psi0, tlist, seed, j, method, rtol,
                                      atol, fixed_dt, dt0, st)
        per.append(ex)
        jt.append(times)
        jc.append(chans)
    per = np.array(per)
    out = dict(expect=per.mean(axis=0), jump_times=jt, jump_channels=jc, stats=st.as_dict())
    if keep_trajectories:
        out["traj_expect"] = per
    return out
