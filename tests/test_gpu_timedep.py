"""Time-dependent Hamiltonians H0 + sum_k f_k(t) H_k (QobjEvo form) and
sesolve through the C ABI: parity with the oracle (fixed steps and
adaptive, trajectory by trajectory for mcsolve), closed forms, the paper's
driven optomechanical example, and the paths that refuse such systems."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle.timedep import Coef, mcsolve_td, mesolve_td, sesolve as o_sesolve
from tests.gpu_util import maxabs, require_gpu

pytestmark = pytest.mark.gpu

SX = np.array([[0, 1], [1, 0]], dtype=complex)
SY = np.array([[0, -1j], [1j, 0]])
SZ = np.array([[1, 0], [0, -1]], dtype=complex)


def destroy(N):
    return sp.diags(np.sqrt(np.arange(1, N)), 1, format="csr", dtype=complex)


def both(spec):
    """[(Hk, dict)] -> (oracle terms, library terms)"""
    return [(h, Coef(**d)) for h, d in spec], [(h, d) for h, d in spec]


def test_sesolve_phase_drive_closed_form_and_oracle():
    qtl = require_gpu()
    A, w = 1.3, 2.1
    spec = [(SZ, dict(kind="cos", amp=A, omega=w))]
    ot, lt = both(spec)
    H0 = 0.3 * SZ
    psi0 = np.array([1, 1], dtype=complex) / math.sqrt(2)
    tl = np.linspace(0, 6, 25)
    g = qtl.System(H0, [], [SX, SY], td=lt)
    try:
        got = g.sesolve(psi0, tl, rtol=1e-10, atol=1e-12)
        fx = g.sesolve(psi0, tl, fixed_dt=0.01)
    finally:
        g.free()
    phi = 0.3 * tl + (A / w) * np.sin(w * tl)
    assert np.max(np.abs(got["expect"][0] - np.cos(2 * phi))) <= 1e-8
    assert np.max(np.abs(got["expect"][1] - np.sin(2 * phi))) <= 1e-8
    ref = o_sesolve(H0, ot, [SX, SY], psi0, tl, rtol=1e-10, atol=1e-12)
    assert maxabs(got["expect"], ref["expect"]) <= 1e-9
    reff = o_sesolve(H0, ot, [SX, SY], psi0, tl, fixed_dt=0.01)
    assert maxabs(fx["expect"], reff["expect"]) <= 1e-10
    assert fx["stats"]["steps_acc"] == reff["stats"]["steps_acc"]


def test_sesolve_gaussian_pulse_fixed_step():
    qtl = require_gpu()
    Om, t0, sig = 2.0, 3.0, 0.7
    spec = [(SX / 2, dict(kind="cos", amp=Om, omega=0.0, t0=t0, sigma=sig)),
            (SY / 2, dict(kind="exp", amp=0.0 + 0.0j, omega=1.0))]   # a zero-amplitude term
    ot, lt = both(spec)
    H0 = 0.0 * SZ + 1e-3 * SZ
    psi0 = np.array([1, 0], dtype=complex)
    tl = np.linspace(0, 6, 13)
    g = qtl.System(H0, [], [SZ, SY], td=lt)
    try:
        got = g.sesolve(psi0, tl, fixed_dt=0.005)
    finally:
        g.free()
    ref = o_sesolve(H0, ot, [SZ, SY], psi0, tl, fixed_dt=0.005)
    assert maxabs(got["expect"], ref["expect"]) <= 1e-10


def _pair_cavity(N=16, wc=1.0, gam=0.8, F=0.3 + 0.1j, w=1.2):
    a = destroy(N)
    spec = [(a, dict(kind="exp", amp=F, omega=w)), (a.conj().T.tocsr(), dict(kind="exp", amp=np.conj(F), omega=-w))]
    psi0 = np.zeros(N, dtype=complex)
    psi0[0] = 1
    z = 1j * wc + gam / 2

    def alpha(t):
        return -1j * np.conj(F) * (np.exp(-1j * w * t) - np.exp(-z * t)) / (z - 1j * w)
    return wc * (a.conj().T @ a), spec, [math.sqrt(gam) * a], [a, a.conj().T @ a], psi0, alpha


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_mcsolve_td_trajectories_coherent_closed_form(precision):
    """Every trajectory of the exp-pair-driven damped cavity stays coherent:
    <a> = alpha(t) on each one, jumps or not; FP64 trajectories also match the
    oracle's one by one."""
    qtl = require_gpu()
    H0, spec, c_ops, e_ops, psi0, alpha = _pair_cavity()
    ot, lt = both(spec)
    tl = np.linspace(0, 8, 17)
    g = qtl.System(H0, c_ops, e_ops, td=lt)
    try:
        got = g.mcsolve(psi0, tl, 8, 3, keep_trajectories=True, precision=precision, rtol=1e-9, atol=1e-11)
    finally:
        g.free()
    tol = 1e-7 if precision == "fp64" else 2e-5
    assert np.max(np.abs(got["traj_expect"][:, 0, :] - alpha(tl)[None, :])) <= tol
    assert got["stats"]["jumps"] > 0
    if precision == "fp64":
        ref = mcsolve_td(H0, ot, c_ops, e_ops, psi0, tl, 8, 3, rtol=1e-9, atol=1e-11, keep_trajectories=True)
        assert maxabs(got["traj_expect"], ref["traj_expect"]) <= 1e-8
        assert got["stats"]["jumps"] == ref["stats"]["jumps"]


def _cos_cavity(N=16, D=0.7, kap=0.5, F=0.4, w=1.1):
    a = destroy(N)
    spec = [((a + a.conj().T).tocsr(), dict(kind="cos", amp=F, omega=w))]
    psi0 = np.zeros(N, dtype=complex)
    psi0[0] = 1
    z = 1j * D + kap / 2

    def alpha(t):
        return -0.5j * F * ((np.exp(1j * w * t) - np.exp(-z * t)) / (z + 1j * w)
                            + (np.exp(-1j * w * t) - np.exp(-z * t)) / (z - 1j * w))
    return D * (a.conj().T @ a), spec, [math.sqrt(kap) * a], [a, a.conj().T @ a], psi0, alpha


@pytest.mark.parametrize("engine", ["cluster", "grid"])
@pytest.mark.parametrize("which", ["cos", "pair"])
def test_mesolve_td_parity_and_closed_form(which, engine):
    """FP64 mesolve on both kernels: the cos drive (real coefficient,
    Hermitian terms: the grid kernel's lower-triangle mode) and the complex
    pair (every entry) against the oracle at fixed steps, entry by entry, and
    adaptively against the closed form."""
    qtl = require_gpu()
    H0, spec, c_ops, e_ops, psi0, alpha = _cos_cavity() if which == "cos" else _pair_cavity()
    ot, lt = both(spec)
    tl = np.linspace(0, 4, 9)
    g = qtl.System(H0, c_ops, e_ops, td=lt)
    try:
        fx = g.mesolve(psi0, tl, fixed_dt=0.01, save_states=True, engine=engine)
        ad = g.mesolve(psi0, tl, rtol=1e-10, atol=1e-12, engine=engine)
    finally:
        g.free()
    ref = mesolve_td(H0, ot, c_ops, e_ops, psi0, tl, fixed_dt=0.01, save_states=True)
    assert maxabs(fx["expect"], ref["expect"]) <= 1e-10
    assert maxabs(fx["states"], ref["states"]) <= 1e-10
    assert np.max(np.abs(ad["expect"][0] - alpha(tl))) <= 1e-8


@pytest.mark.parametrize("engine", ["cluster", "grid"])
def test_paper_driven_optomechanics_short_time(engine):
    """Sec. 3.4's driven optomechanical system (Nc = 10, Nm = 7), drive
    F cos(w_d t)(a + a^dag), losses on both modes, from the vacuum: FP64 grid
    mesolve at fixed steps against the oracle."""
    qtl = require_gpu()
    Nc, Nm = 10, 7
    wc, wm, gc, kap, gam = 1.0, 2.0, 0.05, 0.01, 0.01
    F, wd = 10 * kap, wc
    a = sp.kron(destroy(Nc), sp.identity(Nm), format="csr")
    b = sp.kron(sp.identity(Nc), destroy(Nm), format="csr")
    ad, bd = a.conj().T, b.conj().T
    H0 = (wc * ad @ a + wm * bd @ b + gc / 2 * (a + ad) @ (a + ad) @ (b + bd)).tocsr()
    spec = [((a + ad).tocsr(), dict(kind="cos", amp=F, omega=wd))]
    ot, lt = both(spec)
    c_ops = [math.sqrt(kap) * a, math.sqrt(gam) * b]
    e_ops = [(ad @ a).tocsr()]
    psi0 = np.zeros(Nc * Nm, dtype=complex)
    psi0[0] = 1
    tl = np.linspace(0, 2, 5)
    g = qtl.System(H0, c_ops, e_ops, td=lt)
    try:
        got = g.mesolve(psi0, tl, fixed_dt=0.01, engine=engine)
    finally:
        g.free()
    ref = mesolve_td(H0, ot, c_ops, e_ops, psi0, tl, fixed_dt=0.01)
    assert maxabs(got["expect"], ref["expect"]) <= 1e-10


def test_time_dependent_systems_refuse_unsupported_paths():
    import torch
    qtl = require_gpu()
    H0, spec, c_ops, e_ops, psi0, _ = _cos_cavity(N=6)
    tl = np.linspace(0, 1, 3)
    g = qtl.System(H0, c_ops, e_ops, td=[(spec[0][0], spec[0][1])])
    with pytest.raises(qtl.QtlError) as e1:
        g.mesolve(psi0, tl, precision="mixed", engine="grid")   # mixed: cluster kernel only
    with pytest.raises(qtl.QtlError) as e3:
        g.sesolve(psi0, tl)                      # has collapse operators
    g.mesolve(psi0, tl, fixed_dt=0.01)          # a solve ran: no more terms
    with pytest.raises(qtl.QtlError) as e4:
        qtl.system_add_td(g.handle, spec[0][0], spec[0][1])
    g.free()
    for e in (e1, e3, e4):
        assert e.value.status == qtl.QTL_EINVAL


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_with_time_dependent_systems(precision):
    """qtl_mesolve_batch over driven cavities with different drives and
    detunings, mixed with time-independent Kerr cavities: each result
    against the same system solved alone (FP64 at fixed steps: only the
    cluster size differs, 1e-12; mixed adaptive against the FP64 solve,
    1e-6)."""
    qtl = require_gpu()
    systems = []
    for D, F, w in [(0.7, 0.4, 1.1), (0.3, 0.9, 0.8), (1.2, 0.2, 1.7)]:
        H0, spec, c_ops, e_ops, psi0, _ = _cos_cavity(D=D, F=F, w=w)
        systems.append((H0, both(spec)[1], c_ops, e_ops, psi0))
    for s in W.kerr_sweep(n_inst=2, seed=4, n_min=10, n_max=16, t_end=4.0, nt=9):
        systems.append((s.H, [], s.c_ops, s.e_ops, s.psi0))
    tl = np.linspace(0, 4, 9)
    gs = [qtl.System(H, c, e, td=td) for H, td, c, e, _ in systems]
    try:
        if precision == "fp64":
            kw = dict(fixed_dt=0.01)
            got = qtl.mesolve_batch([g.handle for g in gs], [g.n_e for g in gs], [x[4] for x in systems], tl,
                                    qtl.make_opts(**kw))
            for g, r, x in zip(gs, got, systems):
                alone = g.mesolve(x[4], tl, **kw)
                assert maxabs(r["expect"], alone["expect"]) <= 1e-12
        else:
            got = qtl.mesolve_batch([g.handle for g in gs], [g.n_e for g in gs], [x[4] for x in systems], tl,
                                    qtl.make_opts(precision="mixed", rtol=1e-7, atol=1e-9))
            for g, r, x in zip(gs, got, systems):
                ref = g.mesolve(x[4], tl, rtol=1e-10, atol=1e-12)
                assert maxabs(r["expect"], ref["expect"]) <= 1e-6
    finally:
        for g in gs:
            g.free()



@pytest.mark.parametrize("N", [300, 600], ids=["rows2", "rows4"])
def test_mcsolve_td_two_and_four_rows_per_thread(N):
    """Time-dependent trajectories above 256 rows (2 and 4 rows per thread)
    against the oracle at fixed steps, trajectory by trajectory."""
    qtl = require_gpu()
    a = destroy(N)
    H0 = (0.9 * (a.conj().T @ a)).tocsr()
    spec = [((a + a.conj().T).tocsr(), dict(kind="cos", amp=0.6, omega=1.1, sigma=0.5, t0=0.1))]
    ot, lt = both(spec)
    c_ops = [math.sqrt(0.3) * a]
    e_ops = [a, (a.conj().T @ a).tocsr()]
    psi0 = np.zeros(N, dtype=complex)
    psi0[3] = 1
    tl = np.linspace(0, 0.2, 3)
    g = qtl.System(H0, c_ops, e_ops, td=lt)
    try:
        got = g.mcsolve(psi0, tl, 3, 17, keep_trajectories=True, fixed_dt=0.01)
    finally:
        g.free()
    ref = mcsolve_td(H0, ot, c_ops, e_ops, psi0, tl, 3, 17, fixed_dt=0.01, keep_trajectories=True)
    assert maxabs(got["traj_expect"], ref["traj_expect"]) <= 1e-9


@pytest.mark.parametrize("which", ["cos", "pair", "optomech"])
def test_mesolve_td_mixed_precision_within_1e6_of_fp64(which):
    """Mixed-precision mesolve with time-dependent terms (cluster kernel: the
    increment form with one FP64 base product L_k y per term, the stage
    times' f_k entering through per-stage sums) against the FP64 solve of
    the same system on every expectation value, adaptively and at fixed
    steps; the cos and pair cavities also against their closed forms."""
    qtl = require_gpu()
    if which == "optomech":
        Nc, Nm = 10, 7
        wc, wm, gc, kap, gam = 1.0, 2.0, 0.05, 0.01, 0.01
        a = sp.kron(destroy(Nc), sp.identity(Nm), format="csr")
        b = sp.kron(sp.identity(Nc), destroy(Nm), format="csr")
        ad, bd = a.conj().T, b.conj().T
        H0 = (wc * ad @ a + wm * bd @ b + gc / 2 * (a + ad) @ (a + ad) @ (b + bd)).tocsr()
        spec = [((a + ad).tocsr(), dict(kind="cos", amp=10 * kap, omega=wc))]
        c_ops = [math.sqrt(kap) * a, math.sqrt(gam) * b]
        e_ops = [(ad @ a).tocsr(), a]
        psi0 = np.zeros(Nc * Nm, dtype=complex)
        psi0[0] = 1
        tl = np.linspace(0, 20, 11)
        alpha = None
    else:
        H0, spec, c_ops, e_ops, psi0, alpha = _cos_cavity() if which == "cos" else _pair_cavity()
        tl = np.linspace(0, 8, 17)
    _, lt = both(spec)
    g = qtl.System(H0, c_ops, e_ops, td=lt)
    try:
        ref = g.mesolve(psi0, tl, rtol=1e-10, atol=1e-12, engine="cluster")
        mix = g.mesolve(psi0, tl, precision="mixed", rtol=1e-7, atol=1e-9, engine="cluster")
        fx64 = g.mesolve(psi0, tl, fixed_dt=0.01, engine="cluster")
        fxm = g.mesolve(psi0, tl, fixed_dt=0.01, precision="mixed", engine="cluster")
    finally:
        g.free()
    assert mix["stats"]["steps_acc"] > 10
    assert maxabs(mix["expect"], ref["expect"]) <= 1e-6
    assert maxabs(fxm["expect"], fx64["expect"]) <= 1e-6
    if alpha is not None:
        assert np.max(np.abs(mix["expect"][0] - alpha(tl))) <= 1e-6


def test_td_beyond_n_1024_grid_mesolve_and_wide_trajectories():
    """A cos-driven damped cavity at N = 1100 (rho with 1.21M entries; kets
    above the register-resident size): the FP64 grid mesolve and every FP64
    trajectory of the wide kernel against the closed form of the coherent
    amplitude; mixed-precision trajectories of that size refuse the
    time-dependent system."""
    qtl = require_gpu()
    H0, spec, c_ops, e_ops, psi0, alpha = _cos_cavity(N=1100)
    _, lt = both(spec)
    tl = np.linspace(0, 4, 9)
    g = qtl.System(H0, c_ops, e_ops, td=lt)
    try:
        r = g.mesolve(psi0, tl, rtol=1e-10, atol=1e-12)
        assert np.max(np.abs(r["expect"][0] - alpha(tl))) <= 1e-8
        m = g.mcsolve(psi0, tl, 6, 2, keep_trajectories=True, rtol=1e-9, atol=1e-11)
        assert np.max(np.abs(m["traj_expect"][:, 0, :] - alpha(tl)[None, :])) <= 1e-7
        assert m["stats"]["jumps"] > 0
        with pytest.raises(qtl.QtlError) as e:
            g.mcsolve(psi0, tl, 4, 1, precision="mixed")
        assert e.value.status == qtl.QTL_EINVAL
    finally:
        g.free()


def test_td_wide_trajectory_kernel_equals_the_register_kernel():
    """The exp-pair-driven cavity (N = 16) on the wide trajectory kernel
    (engine="grid") and on the register-resident one, FP64 at fixed steps,
    trajectory by trajectory, and against the oracle."""
    qtl = require_gpu()
    H0, spec, c_ops, e_ops, psi0, alpha = _pair_cavity()
    ot, lt = both(spec)
    tl = np.linspace(0, 4, 9)
    g = qtl.System(H0, c_ops, e_ops, td=lt)
    try:
        wide = g.mcsolve(psi0, tl, 6, 5, keep_trajectories=True, fixed_dt=0.01, engine="grid")
        reg = g.mcsolve(psi0, tl, 6, 5, keep_trajectories=True, fixed_dt=0.01, engine="cluster")
    finally:
        g.free()
    ref = mcsolve_td(H0, ot, c_ops, e_ops, psi0, tl, 6, 5, fixed_dt=0.01, keep_trajectories=True)
    assert maxabs(wide["traj_expect"], reg["traj_expect"]) <= 1e-10
    assert maxabs(wide["traj_expect"], ref["traj_expect"]) <= 1e-9
    assert wide["stats"]["jumps"] == reg["stats"]["jumps"] == ref["stats"]["jumps"] > 0
