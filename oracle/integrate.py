"""Adaptive embedded Runge-Kutta integration (the time stepping the paper
delegates to DifferentialEquations.jl, Sec. 2; memory independent of the
number of output times, Sec. 3.1).

The paper is silent on the method, the error norm, the step-size controller,
the starting step and how output times are met.  The readings used (the same
ones the CUDA library implements):
  * a 7-stage FSAL 5(4) pair (tableau.py);
  * error norm: RMS over complex entries of |e_i| / sc_i with
    e = h sum_j e_j k_j and sc_i = atol + rtol max(|y_i|, |y_new,i|);
  * PI controller: on accept fac = 0.9 err^-0.14 err_prev^0.08 clamped to
    [0.2, 10] (and at most 1 right after a reject), err_prev floored at 1e-4;
    on reject fac = max(0.2, 0.9 err^-1/5);
  * starting step: the Hairer-Norsett-Wanner heuristic (one extra RHS);
  * output times: each step is clamped so that it lands exactly on the next
    time of tlist (no interpolation); a step that would stop short of that
    time by no more than LAND_ULPS units of 2^-52 max(1, |t_target|) lands
    on it instead, so that rounding in t never leaves a vanishing remnant;
    with adaptive steps, a step that would cover more than half of the rest
    of the way, but not all of it, is shortened to half of it, so that two
    equal steps land rather than a full step and a short remainder.
"""
import math

import numpy as np

from .tableau import TABLEAUS as TABLEAUS_BY_NAME  # noqa: F401  (re-export)

SAFETY = 0.9
FAC_MIN = 0.2
FAC_MAX = 10.0
BETA1 = 0.7 / 5.0
BETA2 = 0.4 / 5.0
ERR_PREV_FLOOR = 1e-4
LAND_ULPS = 64.0


class StepLimitError(RuntimeError):
    pass


class Stats:
    def __init__(self):
        self.steps_acc = 0
        self.steps_rej = 0
        self.rhs_evals = 0
        self.jumps = 0

    def as_dict(self):
        return dict(steps_acc=self.steps_acc, steps_rej=self.steps_rej,
                    rhs_evals=self.rhs_evals, jumps=self.jumps)


def rk_step(f, t, y, h, k1, tab):
    """One step of size h from (t, y), with k1 = f(t, y) given (FSAL).
    Stage i has input y + h sum_{j<i} a_ij k_j evaluated at t + c_i h.
    The last stage's input is the new solution (its row of `a` equals b), so
    its derivative is the next step's k1.  Returns (y_new, [k1..k7])."""
    ks = [k1]
    yi = y
    for i in range(1, tab.stages):
        yi = y.copy()
        for j in range(i):
            yi = yi + (h * tab.a[i][j]) * ks[j]
        ks.append(f(t + tab.c[i] * h, yi))
    return yi, ks


def error_norm(y, y_new, ks, h, tab, rtol, atol):
    """sqrt(mean_i |e_i|^2 / sc_i^2) over all complex entries."""
    e = np.zeros_like(y)
    for j in range(tab.stages):
        e = e + (h * tab.e[j]) * ks[j]
    sc = atol + rtol * np.maximum(np.abs(y), np.abs(y_new))
    return math.sqrt(float(np.mean(np.abs(e) ** 2 / sc ** 2)))


class PIController:
    """beta1, beta2: the exponents of the accept factor.  The defaults are
    the PI reading; beta2 = 0 with beta1 = 1/5 is the plain (integral)
    controller of a 5(4) pair."""

    def __init__(self, beta1=BETA1, beta2=BETA2):
        self.beta1 = beta1
        self.beta2 = beta2
        self.err_prev = ERR_PREV_FLOOR
        self.last_rejected = False

    def on_accept(self, err):
        if err == 0.0:
            fac = FAC_MAX
        else:
            fac = SAFETY * err ** (-self.beta1) * self.err_prev ** self.beta2
        fac = min(FAC_MAX, max(FAC_MIN, fac))
        if self.last_rejected:
            fac = min(fac, 1.0)
        self.err_prev = max(err, ERR_PREV_FLOOR)
        self.last_rejected = False
        return fac

    def on_reject(self, err):
        self.last_rejected = True
        return max(FAC_MIN, SAFETY * err ** (-1.0 / 5.0))


def _rms(v):
    return math.sqrt(float(np.mean(np.abs(v) ** 2)))


def initial_step(f, t0, y0, f0, rtol, atol):
    """Starting step of Hairer, Norsett & Wanner, Solving ODEs I, Sec. II.4,
    for a method of order 5."""
    sc = atol + rtol * np.abs(y0)
    d0 = _rms(np.abs(y0) / sc)
    d1 = _rms(np.abs(f0) / sc)
    if d0 < 1e-5 or d1 < 1e-5:
        h0 = 1e-6
    else:
        h0 = 0.01 * d0 / d1
    y1 = y0 + h0 * f0
    f1 = f(t0 + h0, y1)
    d2 = _rms(np.abs(f1 - f0) / sc) / h0
    if max(d1, d2) <= 1e-15:
        h1 = max(1e-6, h0 * 1e-3)
    else:
        h1 = (0.01 / max(d1, d2)) ** (1.0 / 5.0)
    return min(100.0 * h0, h1)


def integrate(f, y0, tlist, tab, rtol, atol, on_save, dt0=0.0, fixed_dt=None,
              max_steps=10_000_000, dt_min=0.0, after_accept=None, stats=None,
              beta1=BETA1, beta2=BETA2, balance=True):
    """Integrate y' = f(t, y) from tlist[0], calling on_save(idx, t, y) at
    every tlist point (steps land on them exactly).

    fixed_dt: if given, every step has size min(fixed_dt, time to the next
    tlist point) and is accepted without error control.
    after_accept(t, y, k1, h, t_new, y_new, k_last) may return a replacement
    (t, y, k1) to restart from (used by the quantum-jump method).
    beta1, beta2: the step controller's exponents (PIController).
    balance: with adaptive steps, when the proposed step covers more than
    half of the way to the next tlist point without reaching it, the step
    is half of the way, so that two equal steps land (reading G7); False
    gives the plain clamp of the last step (the SciPy pin)."""
    st = stats if stats is not None else Stats()
    t = float(tlist[0])
    y = np.array(y0, dtype=np.complex128)
    k1 = f(t, y)
    st.rhs_evals += 1
    on_save(0, t, y)
    if fixed_dt is not None:
        h = float(fixed_dt)
    elif dt0 > 0:
        h = float(dt0)
    else:
        h = initial_step(f, t, y, k1, rtol, atol)
        st.rhs_evals += 1
    ctrl = PIController(beta1, beta2)
    nsteps = 0
    for idx in range(1, len(tlist)):
        t_target = float(tlist[idx])
        while t < t_target:
            if nsteps >= max_steps:
                raise StepLimitError("max_steps reached")
            nsteps += 1
            rem = t_target - t
            land = h >= rem - LAND_ULPS * 2.0 ** -52 * max(1.0, abs(t_target))
            if land:
                h_try = rem
            elif balance and fixed_dt is None and h >= 0.5 * rem:
                h_try = 0.5 * rem      # two equal steps land (reading G7)
            else:
                h_try = h
            y_new, ks = rk_step(f, t, y, h_try, k1, tab)
            st.rhs_evals += tab.stages - 1
            if fixed_dt is None:
                err = error_norm(y, y_new, ks, h_try, tab, rtol, atol)
                if not err <= 1.0:
                    st.steps_rej += 1
                    h = h_try * ctrl.on_reject(err)
                    if h < dt_min or not math.isfinite(err):
                        raise StepLimitError("step size underflow")
                    continue
                fac = ctrl.on_accept(err)
                h_next = h_try * fac
            else:
                h_next = float(fixed_dt)
            st.steps_acc += 1
            t_new = t_target if land else t + h_try
            restart = None
            if after_accept is not None:
                restart = after_accept(t, y, k1, h_try, t_new, y_new, ks[-1])
            if restart is None:
                t, y, k1 = t_new, y_new, ks[-1]
            else:
                t, y, k1 = restart
            h = h_next
        on_save(idx, t, y)
    return st
