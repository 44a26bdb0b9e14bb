"""GPU parity of mcsolve (trajectory kernel, through the C ABI) against the
FP64 oracle, trajectory by trajectory, plus ensemble statistics."""
import math

import numpy as np
import pytest

import workloads as W
from oracle.mcsolve import mcsolve as oracle_mcsolve
from oracle.mesolve import mesolve as oracle_mesolve
from oracle.philox import uniform
from tests.gpu_util import maxabs, require_gpu

pytestmark = pytest.mark.gpu


def _gpu(s, tlist, ntraj, seed, **kw):
    qtl = require_gpu()
    keep = kw.pop("keep_trajectories", True)
    off = kw.pop("traj_offset", 0)
    g = qtl.System(s.H, s.c_ops, s.e_ops)
    try:
        return g.mcsolve(s.psi0, tlist, ntraj, seed, traj_offset=off, keep_trajectories=keep, **kw)
    finally:
        g.free()


def test_two_level_jump_times_closed_form():
    """H = 0: psi stays |e> (normalised) until t* = -ln(r)/g, then |g>."""
    g_ = 0.5
    s = W.two_level_decay(gamma=g_, t_end=8.0, nt=81)
    got = _gpu(s, s.tlist, 200, 11, rtol=1e-11, atol=1e-13)
    pe = got["traj_expect"][:, 0, :].real
    for j in range(200):
        t_star = -math.log(uniform(11, j, 0)) / g_
        expect = (s.tlist < t_star - 1e-7).astype(float)
        mask = np.abs(s.tlist - t_star) > 1e-7
        assert np.max(np.abs(pe[j][mask] - expect[mask])) < 1e-9


@pytest.mark.parametrize("precision", ["fp64"])
def test_trajectory_parity_jc(precision):
    s = W.jaynes_cummings(N=5, nt=41, t_end=80.0, kappa=0.1, gamma=0.05)
    ref = oracle_mcsolve(s.H, s.c_ops, s.e_ops, s.psi0, s.tlist, ntraj=24, seed=7,
                         keep_trajectories=True)
    got = _gpu(s, s.tlist, 24, 7, precision=precision)
    assert maxabs(got["traj_expect"], ref["traj_expect"]) <= 1e-8
    assert maxabs(got["expect"], ref["expect"]) <= 1e-8
    assert got["stats"]["jumps"] == ref["stats"]["jumps"]


def test_trajectory_parity_fixed_step_fock_cascade():
    s = W.damped_oscillator(N=6, omega=1.3, gamma=0.3, n0=3, t_end=12.0, nt=25)
    ref = oracle_mcsolve(s.H, s.c_ops, s.e_ops, s.psi0, s.tlist, ntraj=16, seed=2024,
                         fixed_dt=0.01, keep_trajectories=True)
    got = _gpu(s, s.tlist, 16, 2024, fixed_dt=0.01)
    assert maxabs(got["traj_expect"], ref["traj_expect"]) <= 1e-8


def test_traj_offset_selects_the_same_streams():
    s = W.jaynes_cummings(N=4, nt=11, t_end=40.0, kappa=0.2)
    a = _gpu(s, s.tlist, 40, 3)
    b = _gpu(s, s.tlist, 20, 3, traj_offset=20)
    assert maxabs(a["traj_expect"][20:], b["traj_expect"]) == 0.0


def test_ensemble_matches_mesolve_jc_config():
    """The configured JC cavity (N=40 x 2) with 1000 trajectories: the mean is
    within 3 sigma/sqrt(ntraj) of the master equation at every time."""
    s = W.jaynes_cummings(nt=200)
    me = oracle_mesolve(s.H, s.c_ops, s.e_ops, s.psi0, s.tlist)
    got = _gpu(s, s.tlist, 1000, 1)
    per = got["traj_expect"].real
    sd = per.std(axis=0)
    bound = 3 * np.maximum(sd, 1e-3) / math.sqrt(1000) + 1e-6
    assert np.all(np.abs(got["expect"].real - me["expect"].real) <= bound)


def test_mixed_precision_trajectories():
    s = W.jaynes_cummings(N=5, nt=41, t_end=80.0, kappa=0.1, gamma=0.05)
    ref = oracle_mcsolve(s.H, s.c_ops, s.e_ops, s.psi0, s.tlist, ntraj=24, seed=7,
                         keep_trajectories=True)
    got = _gpu(s, s.tlist, 24, 7, precision="mixed", rtol=1e-7, atol=1e-9)
    # a jump time moves by the FP32 rounding of the norm; compare trajectories
    # whose jump counts agree, at the 1e-6 bar
    same = [j for j in range(24) if np.allclose(got["traj_expect"][j, 0, -1].real,
                                                ref["traj_expect"][j, 0, -1].real, atol=1e-3)]
    assert len(same) >= 20
    for j in same:
        assert maxabs(got["traj_expect"][j], ref["traj_expect"][j]) <= 1e-5


def test_mixed_ensemble_within_sampling_error_of_fp64():
    """1000 trajectories of the JC system: the mixed ensemble mean is within
    3 sigma / sqrt(ntraj) of the FP64 ensemble with the same draws at every
    time (a jump moved by the FP32 rounding changes a trajectory, not the
    statistics)."""
    s = W.jaynes_cummings(N=10, nt=101, t_end=200.0, kappa=0.1, gamma=0.05)
    m = _gpu(s, s.tlist, 1000, 13, precision="mixed", rtol=1e-7, atol=1e-9, keep_trajectories=False)
    f = _gpu(s, s.tlist, 1000, 13, precision="fp64", rtol=1e-7, atol=1e-9)
    sd = f["traj_expect"].real.std(axis=0)
    bound = 3 * np.maximum(sd, 1e-3) / math.sqrt(1000) + 1e-6
    assert np.all(np.abs(m["expect"].real - f["expect"].real) <= bound)


def test_repeated_output_times():
    """A time listed twice is saved twice: the landing step saves the first
    copy and the repeat the second."""
    s = W.jaynes_cummings(N=4, nt=11, t_end=40.0, kappa=0.2)
    tl = np.array([0.0, 5.0, 5.0, 12.0, 12.0, 12.0, 20.0])
    ref = oracle_mcsolve(s.H, s.c_ops, s.e_ops, s.psi0, tl, ntraj=6, seed=8,
                         keep_trajectories=True)
    got = _gpu(s, tl, 6, 8)
    assert maxabs(got["traj_expect"], ref["traj_expect"]) <= 1e-8
    assert maxabs(got["traj_expect"][:, :, 1], got["traj_expect"][:, :, 2]) == 0.0


def test_mcsolve_edge_cases():
    qtl = require_gpu()
    s = W.two_level_decay()
    g = qtl.System(s.H, s.c_ops, s.e_ops)
    one = g.mcsolve(s.psi0, np.array([0.0]), 3, 1)
    assert maxabs(one["expect"][0], [1.0]) < 1e-15
    with pytest.raises(qtl.QtlError):
        g.mcsolve(s.psi0, np.array([0.0, 2.0, 1.0]), 3, 1)
    g.free()
    # no collapse operators: no jumps, the state evolves unitarily
    g2 = qtl.System(W.sigmax(), [], [W.sigmaz()])
    out = g2.mcsolve(W.fock(2, 0), np.linspace(0, 3, 7), 4, 1, rtol=1e-10, atol=1e-12)
    assert out["stats"]["jumps"] == 0
    assert maxabs(out["expect"][0].real, np.cos(2 * np.linspace(0, 3, 7))) < 1e-8
    g2.free()


def test_sharded_ranges_reproduce_the_full_ensemble():
    """Two trajectory shares (as two ranks would run them) combine to the
    single-call ensemble mean."""
    from paper_2504_21440_gb300.shard import trajectory_shard
    qtl = require_gpu()
    s = W.jaynes_cummings(N=5, nt=21, t_end=60.0, kappa=0.1)
    g = qtl.System(s.H, s.c_ops, s.e_ops)
    full = g.mcsolve(s.psi0, s.tlist, 101, 3)
    acc = 0
    for r in range(2):
        first, count = trajectory_shard(101, r, 2)
        part = g.mcsolve(s.psi0, s.tlist, count, 3, traj_offset=first)
        acc = acc + part["expect"] * count
    g.free()
    assert maxabs(acc / 101, full["expect"]) <= 1e-13


def _random_many_channel_system(n=20, n_c=40, n_e=20, seed=12):
    """A random n-level system with more collapse operators (n_c) and more
    observable slots (1 + 2 n_e) than a 32-thread trajectory CTA has threads."""
    import scipy.sparse as sp
    rng = np.random.default_rng(seed)

    def herm(density):
        m = sp.random(n, n, density=density, random_state=rng, dtype=np.float64)
        m = m + 1j * sp.random(n, n, density=density, random_state=rng, dtype=np.float64)
        return sp.csr_matrix((m + m.conj().T) * 0.5)

    H = herm(0.2)
    c_ops = []
    for _ in range(n_c):
        m = sp.random(n, n, density=0.05, random_state=rng, dtype=np.float64)
        c_ops.append(sp.csr_matrix(m * 0.15 + 0j))
    e_ops = [herm(0.15) for _ in range(n_e)]
    psi0 = np.zeros(n, complex)
    psi0[0] = 1.0
    return H, c_ops, e_ops, psi0


def test_many_observables_and_channels_in_a_32_thread_cta():
    """n = 20 runs in a 32-thread CTA; 20 general observables need 41
    reduction slots and 40 channels 40 jump weights.  Every slot must be
    reduced and every observable saved."""
    qtl = require_gpu()
    H, c_ops, e_ops, psi0 = _random_many_channel_system()
    tl = np.linspace(0.0, 6.0, 13)
    ref = oracle_mcsolve(H, c_ops, e_ops, psi0, tl, ntraj=12, seed=31, keep_trajectories=True)
    g = qtl.System(H, c_ops, e_ops)
    try:
        got = g.mcsolve(psi0, tl, 12, 31, keep_trajectories=True)
    finally:
        g.free()
    assert ref["stats"]["jumps"] > 0
    assert got["stats"]["jumps"] == ref["stats"]["jumps"]
    assert maxabs(got["traj_expect"], ref["traj_expect"]) <= 1e-8
    assert maxabs(got["expect"], ref["expect"]) <= 1e-8
