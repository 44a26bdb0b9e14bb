"""Pins of the oracle's error norm, step controller and starting step
(oracle/integrate.py: error_norm, PIController, initial_step) against an
independent published implementation of the same pieces.

SciPy's RK45 integrates with the Dormand-Prince 5(4) pair and uses, as the
oracle does: the RMS norm of |e_i| / sc_i over complex entries with
sc_i = atol + rtol max(|y_i|, |y_new,i|); the starting-step heuristic of
Hairer, Norsett & Wanner (Solving ODEs I, Sec. II.4) with exponent 1/5; the
safety factor 0.9, the clamp [0.2, 10], the reject factor
max(0.2, 0.9 err^-1/5) and no growth on the step after a reject.  Its
controller is the plain integral one, which is the oracle's PI controller
with beta1 = 1/5 and beta2 = 0.  With those exponents the two must take the
same steps.  A mistake in any of the pinned pieces (a norm over 2n^2 real
components, a missing max() in sc, a wrong safety factor, exponent or clamp,
growth after a reject, a changed starting step) changes the step sequence by
far more than the bound used here.

The bound on the accepted times is 1e-9 of the span, not machine precision:
e = h sum_j e_j k_j cancels its terms to about |e| / (h |k|) ~ 1e-8 here, so
the rounding order of the sum alone moves err by ~1e-9 relative and each
step factor by a fifth of that; a norm off by sqrt(2) moves the factors by 7%.
"""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.integrate import RK45

from oracle.integrate import PIController, Stats, error_norm, initial_step, integrate, rk_step
from oracle.lindblad import liouvillian
from oracle.tableau import DP5


def _oracle_steps(f, y0, t0, t1, rtol, atol):
    times = []

    def after(t, y, k1, h, t_new, y_new, k_last):
        times.append(t_new)
        return None

    st = integrate(f, y0, np.array([t0, t1]), DP5, rtol, atol, lambda *a: None,
                   after_accept=after, beta1=0.2, beta2=0.0, balance=False)
    return np.array(times), st


def _scipy_steps(f, y0, t0, t1, rtol, atol):
    sol = RK45(f, t0, np.array(y0, dtype=complex), t1, rtol=rtol, atol=atol)
    h_first = sol.h_abs
    times = []
    while sol.status == "running":
        sol.step()
        times.append(sol.t)
    assert sol.status == "finished"
    return np.array(times), sol.nfev, h_first


def _complex_linear(seed=3, n=6):
    rng = np.random.default_rng(seed)
    M = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    M = M - (np.max(np.linalg.eigvals(M).real) + 0.3) * np.eye(n)   # stable
    y0 = rng.normal(size=n) + 1j * rng.normal(size=n)
    return (lambda t, y: M @ y), y0


def _pulsed(seed=7, n=4):
    """A rotating vector hit by a narrow pulse at t = 2: the controller grows
    the step before the pulse and must reject to get through it."""
    rng = np.random.default_rng(seed)
    M = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    M = -1j * (M + M.conj().T) / 2
    y0 = rng.normal(size=n) + 1j * rng.normal(size=n)
    return (lambda t, y: (1.0 + 30.0 * np.exp(-((t - 2.0) / 0.05) ** 2)) * (M @ y)), y0


def _lindblad4(seed=5):
    rng = np.random.default_rng(seed)
    n = 4
    H = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    H = sp.csr_matrix(H + H.conj().T)
    c_ops = [sp.csr_matrix(0.4 * (rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))))
             for _ in range(2)]
    L = liouvillian(H, c_ops)
    psi = rng.normal(size=n) + 1j * rng.normal(size=n)
    psi /= np.linalg.norm(psi)
    rho0 = np.outer(psi, psi.conj()).reshape(-1, order="F")
    return (lambda t, y: L @ y), rho0


@pytest.mark.parametrize("problem,t1,rtol,atol", [
    (_complex_linear, 4.0, 1e-6, 1e-9),
    (_complex_linear, 4.0, 1e-9, 1e-12),
    (_lindblad4, 6.0, 1e-7, 1e-10),
    (_pulsed, 4.0, 1e-7, 1e-10),
])
def test_integral_controller_matches_scipy_rk45(problem, t1, rtol, atol):
    f, y0 = problem()
    ours, st = _oracle_steps(f, y0, 0.0, t1, rtol, atol)
    ref, nfev, h_first = _scipy_steps(f, y0, 0.0, t1, rtol, atol)
    # the same starting step
    sc_h = initial_step(f, 0.0, np.asarray(y0, complex), f(0.0, np.asarray(y0, complex)), rtol, atol)
    assert abs(sc_h - h_first) <= 1e-14 * h_first
    # the same accepted steps ...
    assert len(ours) == len(ref) and len(ours) > 20
    assert np.max(np.abs(ours - ref)) <= 1e-9 * t1
    # ... and the same attempts: SciPy counts f(t0), the starting step's probe
    # and six evaluations per attempted step, as the oracle's rhs_evals does
    assert st.rhs_evals == nfev
    assert st.steps_rej == (nfev - 2) // 6 - len(ref)


def test_scipy_pin_sees_rejections():
    """The pulsed case above must exercise the reject branch, or the reject
    factor and the no-growth rule would go unpinned."""
    f, y0 = _pulsed()
    _, st = _oracle_steps(f, y0, 0.0, 4.0, 1e-7, 1e-10)
    assert st.steps_rej >= 2


def test_error_estimate_is_fifth_order_in_h():
    """The embedded estimate of a 5(4) pair is the local error of its
    order-4 member, O(h^5): halving h divides it by about 2^5 on y' = lam y."""
    lam = -1.0 + 2.0j
    f = lambda t, y: lam * y
    y0 = np.array([1.0 + 0.0j])
    errs = []
    for h in [0.08, 0.04, 0.02, 0.01]:
        y_new, ks = rk_step(f, 0.0, y0, h, f(0.0, y0), DP5)
        # atol dominates sc, so the norm is |e| / atol
        errs.append(error_norm(y0, y_new, ks, h, DP5, rtol=0.0, atol=1.0))
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(np.abs(ratios - 32.0) < 2.5)
    assert abs(ratios[-1] - 32.0) < 0.6


def test_pi_defaults_differ_from_the_integral_controller():
    """The default (PI) exponents are the reading used everywhere else; the
    integral controller is reached only by passing the exponents."""
    a, b = PIController(), PIController(0.2, 0.0)
    a.on_accept(0.3), b.on_accept(0.3)
    assert a.on_accept(0.5) != b.on_accept(0.5)
    assert isinstance(Stats(), Stats)


def _norm_over_real_components(y, y_new, ks, h, tab, rtol, atol):
    e = sum((h * tab.e[j]) * ks[j] for j in range(tab.stages))
    sc = atol + rtol * np.maximum(np.abs(y), np.abs(y_new))
    r = np.concatenate([e.real / sc, e.imag / sc])
    return float(np.sqrt(np.mean(r ** 2)))


def _norm_scaled_by_y_only(y, y_new, ks, h, tab, rtol, atol):
    e = sum((h * tab.e[j]) * ks[j] for j in range(tab.stages))
    sc = atol + rtol * np.abs(y)
    return float(np.sqrt(np.mean(np.abs(e) ** 2 / sc ** 2)))


class _GrowAfterReject(PIController):
    def on_accept(self, err):
        self.last_rejected = False
        return super().on_accept(err)


class _RejectSafety(PIController):
    def on_reject(self, err):
        self.last_rejected = True
        return max(0.2, 0.8 * err ** (-0.2))


@pytest.mark.parametrize("plant", ["real_components", "scale_y_only", "grow_after_reject",
                                   "reject_safety", "start_step"])
def test_planted_controller_mistakes_break_the_pin(plant, monkeypatch):
    import oracle.integrate as I
    if plant == "real_components":
        monkeypatch.setattr(I, "error_norm", _norm_over_real_components)
    elif plant == "scale_y_only":
        monkeypatch.setattr(I, "error_norm", _norm_scaled_by_y_only)
    elif plant == "grow_after_reject":
        monkeypatch.setattr(I, "PIController", _GrowAfterReject)
    elif plant == "reject_safety":
        monkeypatch.setattr(I, "PIController", _RejectSafety)
    else:
        real = I.initial_step
        monkeypatch.setattr(I, "initial_step", lambda *a: 1.5 * real(*a))
    broken = False
    for problem, t1, rtol, atol in [(_complex_linear, 4.0, 1e-6, 1e-9), (_pulsed, 4.0, 1e-7, 1e-10)]:
        f, y0 = problem()
        ours, st = _oracle_steps(f, y0, 0.0, t1, rtol, atol)
        ref, nfev, _ = _scipy_steps(f, y0, 0.0, t1, rtol, atol)
        if len(ours) != len(ref) or st.rhs_evals != nfev or np.max(np.abs(ours - ref)) > 1e-9 * t1:
            broken = True
    assert broken


def test_balanced_landing_takes_two_equal_steps():
    """With adaptive steps and output times denser than the free step size
    allows, a step that would cover more than half of the way to an output
    time without reaching it is cut to half of it, and the next step lands:
    every landing step equals the step before it whenever that step was
    balanced, no landing step is shorter than half the free step before it,
    and the balanced solve takes fewer steps than the plain clamp to the same
    accuracy (y' = (-0.3 + 2i) y, exact solution)."""
    lam = -0.3 + 2.0j
    f = lambda t, y: lam * y
    y0 = np.array([1.0 + 0.0j])
    tl = np.linspace(0.0, 10.0, 41)
    res = {}
    for bal in (False, True):
        steps, vals = [], {}

        def after(t, y, k1, h, t_new, y_new, k_last, steps=steps):
            steps.append((t, t_new))
            return None

        st = integrate(f, y0, tl, DP5, 1e-9, 1e-12, lambda i, t, y, vals=vals: vals.__setitem__(i, y[0]),
                       after_accept=after, balance=bal)
        got = np.array([vals[i] for i in range(len(tl))])
        assert np.max(np.abs(got - np.exp(lam * tl))) <= 1e-7
        res[bal] = (st, steps)
    (st0, s0), (st1, s1) = res[False], res[True]
    assert st1.steps_acc < st0.steps_acc
    grid = set(np.round(tl, 12))
    seen = 0
    for (ta, tb), (tc, td) in zip(s1, s1[1:]):
        if round(td, 12) in grid and round(tb, 12) not in grid:
            h_prev, h_land = tb - ta, td - tc
            assert h_land >= 0.5 * h_prev * (1 - 1e-12)
            if abs(h_land - h_prev) <= 1e-12 * h_prev:
                seen += 1
    assert seen > 5
