"""The grid mesolve kernel (product form A rho + rho B + sum C rho C^dag over a
cooperative grid, for density matrices too large for one cluster): parity
with the FP64 oracle at fixed steps and adaptively, mixed precision, and the
full-size Ising chain (n = 1024) against the oracle and a closed form."""
import numpy as np
import pytest

import workloads as W
from oracle.mesolve import mesolve as oracle_mesolve
from tests.gpu_util import maxabs, require_gpu

pytestmark = pytest.mark.gpu


def _gpu_state(s, state0, tlist, **kw):
    qtl = require_gpu()
    save = kw.pop("save_states", False)
    g = qtl.System(s.H, s.c_ops, s.e_ops)
    try:
        return g.mesolve(state0, tlist, save_states=save, engine="grid", **kw)
    finally:
        g.free()


def _gpu(s, tlist, **kw):
    qtl = require_gpu()
    save = kw.pop("save_states", False)
    g = qtl.System(s.H, s.c_ops, s.e_ops)
    try:
        return g.mesolve(s.psi0, tlist, save_states=save, engine="grid", **kw)
    finally:
        g.free()


@pytest.mark.parametrize("method", ["dp5", "tsit5"])
@pytest.mark.parametrize("mk,tl,dt", [
    (lambda: W.driven_cavity(), np.linspace(0, 2, 11), 0.01),
    (lambda: W.jaynes_cummings(), np.linspace(0, 20, 6), 0.05),
    (lambda: W.ising_chain(5, h=0.9), np.linspace(0, 1, 3), 0.01),
    (lambda: W.thermal_oscillator(N=7), np.linspace(0, 1, 5), 0.01),
], ids=["cavity20", "jc40x2", "ising5", "thermal7"])
def test_grid_fixed_step_parity_fp64(mk, tl, dt, method):
    s = mk()
    ref = oracle_mesolve(s.H, s.c_ops, s.e_ops, s.psi0, tl, method=method, fixed_dt=dt,
                         save_states=True, rhs="product")
    got = _gpu(s, tl, method=method, fixed_dt=dt, save_states=True)
    assert maxabs(got["expect"], ref["expect"]) <= 1e-10
    assert maxabs(got["states"], ref["states"]) <= 1e-10
    assert got["stats"]["steps_acc"] == ref["stats"]["steps_acc"]


def test_grid_adaptive_parity_cavity():
    s = W.driven_cavity()
    ref = oracle_mesolve(s.H, s.c_ops, s.e_ops, s.psi0, s.tlist, rtol=s.rtol, atol=s.atol)
    got = _gpu(s, s.tlist, rtol=s.rtol, atol=s.atol)
    assert maxabs(got["expect"], ref["expect"]) <= 1e-10


def test_grid_mixed_within_1e6():
    for s in [W.jaynes_cummings(nt=200), W.kerr_cavity(30, 0.5, 0.2, 1.0, 0.2, t_end=20.0, nt=41)]:
        ref = oracle_mesolve(s.H, s.c_ops, s.e_ops, s.psi0, s.tlist, rtol=1e-7, atol=1e-9)
        got = _gpu(s, s.tlist, precision="mixed", rtol=1e-7, atol=1e-9)
        assert maxabs(got["expect"], ref["expect"]) <= 1e-6


def test_grid_matches_cluster_kernel_fp64():
    qtl = require_gpu()
    s = W.jaynes_cummings(N=20, nt=11, t_end=30.0)
    g = qtl.System(s.H, s.c_ops, s.e_ops)
    a = g.mesolve(s.psi0, s.tlist, fixed_dt=0.05, engine="grid")
    b = g.mesolve(s.psi0, s.tlist, fixed_dt=0.05, engine="cluster")
    g.free()
    assert maxabs(a["expect"], b["expect"]) <= 1e-12


def test_ising10_full_size_fixed_steps_vs_oracle():
    """n = 1024 (rho with 1,048,576 entries), two FP64 steps against the oracle."""
    s = W.ising_chain(10)
    tl = np.array([0.0, 0.01, 0.02])
    ref = oracle_mesolve(s.H, s.c_ops, s.e_ops, s.psi0, tl, fixed_dt=0.01, rhs="product")
    got = _gpu(s, tl, fixed_dt=0.01)
    assert maxabs(got["expect"], ref["expect"]) <= 1e-10
    mix = _gpu(s, tl, fixed_dt=0.01, precision="mixed")
    assert maxabs(mix["expect"], ref["expect"]) <= 1e-5


def test_ising10_h0_closed_form_mixed_adaptive():
    """h = 0: each spin decays on its own, Sz(t) = N (2 e^{-g t} - 1), at full size."""
    s = W.ising_chain(10, h=0.0)
    got = _gpu(s, s.tlist, precision="mixed", rtol=1e-7, atol=1e-9)
    ref = 10 * (2 * np.exp(-0.1 * s.tlist) - 1)
    assert np.max(np.abs(got["expect"][2].real - ref)) <= 1e-5
    assert np.max(np.abs(got["expect"][0])) <= 1e-6   # Sx stays 0


@pytest.mark.parametrize("N", [37, 45, 66])
def test_grid_ragged_sizes_fixed_steps(N):
    """Dimensions that are not multiples of the 32-row slices or the 4-column
    work units (partial slices and column groups) against the oracle."""
    s = W.driven_cavity(N=N)
    tl = np.linspace(0, 0.5, 3)
    ref = oracle_mesolve(s.H, s.c_ops, s.e_ops, s.psi0, tl, fixed_dt=0.01, save_states=True,
                         rhs="product")
    got = _gpu(s, tl, fixed_dt=0.01, save_states=True)
    assert maxabs(got["expect"], ref["expect"]) <= 1e-10
    assert maxabs(got["states"], ref["states"]) <= 1e-10


def test_grid_non_hermitian_rho0_full_mode():
    """A non-Hermitian initial matrix (the kernel then integrates every entry,
    not the lower triangle) against the oracle, entry by entry."""
    s = W.jaynes_cummings(N=10)
    n = s.H.shape[0]
    rng = np.random.default_rng(11)
    rho0 = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    tl = np.linspace(0, 1.0, 3)
    ref = oracle_mesolve(s.H, s.c_ops, s.e_ops, rho0, tl, fixed_dt=0.02, save_states=True,
                         rhs="product")
    got = _gpu_state(s, rho0, tl, fixed_dt=0.02, save_states=True)
    assert maxabs(got["states"], ref["states"]) <= 1e-10
    assert maxabs(got["expect"], ref["expect"]) <= 1e-10


def test_grid_non_hermitian_h_full_mode():
    """H with an anti-Hermitian part keeps rho from staying Hermitian; the
    kernel detects it and integrates every entry."""
    s = W.jaynes_cummings(N=10)
    n = s.H.shape[0]
    Hn = np.asarray(s.H.todense() if hasattr(s.H, "todense") else s.H, dtype=complex)
    Hn = Hn - 0.05j * np.diag(np.arange(n) / n)
    tl = np.linspace(0, 1.0, 3)
    ref = oracle_mesolve(Hn, s.c_ops, s.e_ops, s.psi0, tl, fixed_dt=0.02, save_states=True,
                         rhs="product")
    qtl = require_gpu()
    g = qtl.System(Hn, s.c_ops, s.e_ops)
    try:
        got = g.mesolve(s.psi0, tl, fixed_dt=0.02, save_states=True, engine="grid")
    finally:
        g.free()
    assert maxabs(got["states"], ref["states"]) <= 1e-10


def test_grid_hermitian_mode_matches_full_mode():
    """The same Hermitian problem with and without a rounding-size
    anti-Hermitian part in rho0 (above the 1e-13 threshold: full mode) gives
    the same trajectory to well within the parity tolerance."""
    s = W.ising_chain(6, h=0.8)
    n = s.H.shape[0]
    psi = np.asarray(s.psi0)
    rho0 = np.outer(psi, psi.conj())
    rng = np.random.default_rng(5)
    pert = 1e-11 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    tl = np.linspace(0, 0.5, 3)
    a = _gpu_state(s, rho0, tl, fixed_dt=0.01, save_states=True)
    b = _gpu_state(s, rho0 + pert, tl, fixed_dt=0.01, save_states=True)
    ref = oracle_mesolve(s.H, s.c_ops, s.e_ops, rho0, tl, fixed_dt=0.01, save_states=True,
                         rhs="product")
    assert maxabs(a["states"], ref["states"]) <= 1e-10
    assert maxabs(b["states"], ref["states"]) <= 1e-9
