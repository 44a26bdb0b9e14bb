"""Pins for the quantum-trajectory oracle (Sec. 3.3): jump times that follow
in closed form from the drawn thresholds, channel statistics, and agreement
of the ensemble mean with the master equation."""
import math

import numpy as np
import pytest

import workloads as W
from oracle.mcsolve import mcsolve
from oracle.mesolve import mesolve
from oracle.philox import uniform


def test_two_level_first_jump_time():
    """H = 0, C = sqrt(g) sigma-, psi0 = |e>: |psi(t)|^2 = e^{-g t}, so the
    jump happens at t* = -ln(r)/g, r the trajectory's first draw."""
    g = 0.5
    s = W.two_level_decay(gamma=g, t_end=40.0, nt=5)
    res = mcsolve(s.H, s.c_ops, s.e_ops, s.psi0, s.tlist, ntraj=40, seed=11,
                  rtol=1e-11, atol=1e-13)
    for j in range(40):
        t_star = -math.log(uniform(11, j, 0)) / g
        if t_star < 40.0:
            assert len(res["jump_times"][j]) == 1
            assert abs(res["jump_times"][j][0] - t_star) < 1e-8
        else:
            assert res["jump_times"][j] == []


def test_fock_cascade_jump_times():
    """H = w a'a, C = sqrt(g) a, psi0 = |3>: between jumps |psi|^2 decays as
    e^{-g n (t - t_last)}; thresholds are draws 0, 2, 4, channel draws 1, 3, 5."""
    g = 0.3
    s = W.damped_oscillator(N=6, omega=1.3, gamma=g, n0=3, t_end=30.0, nt=7)
    res = mcsolve(s.H, s.c_ops, s.e_ops, s.psi0, s.tlist, ntraj=25, seed=2024,
                  rtol=1e-11, atol=1e-13)
    for j in range(25):
        t, ref = 0.0, []
        for k, n in enumerate((3, 2, 1)):
            t = t - math.log(uniform(2024, j, 2 * k)) / (g * n)
            if t < 30.0:
                ref.append(t)
        got = res["jump_times"][j]
        assert len(got) == len(ref)
        assert np.max(np.abs(np.array(got) - np.array(ref)), initial=0) < 1e-8
    # <a'a> of each trajectory is the Fock number at each saved time
    per = mcsolve(s.H, s.c_ops, s.e_ops, s.psi0, s.tlist, ntraj=3, seed=2024,
                  keep_trajectories=True)["traj_expect"]
    assert np.allclose(per.real, np.round(per.real), atol=1e-9)


def test_channel_choice_statistics():
    """Two channels producing the same jump with rates g1, g2: channel 0 is
    taken with probability g1/(g1+g2)."""
    s = W.two_level_decay(gamma=1.0, t_end=30.0, nt=3)
    g1, g2 = 0.3, 0.7
    c_ops = [math.sqrt(g1) * s.c_ops[0], math.sqrt(g2) * s.c_ops[0]]
    n = 400
    res = mcsolve(s.H, c_ops, s.e_ops, s.psi0, s.tlist, ntraj=n, seed=5, rtol=1e-6, atol=1e-8)
    ch = [c[0] for c in res["jump_channels"] if c]
    p = g1 / (g1 + g2)
    frac = ch.count(0) / len(ch)
    assert abs(frac - p) < 4 * math.sqrt(p * (1 - p) / len(ch))
    # and each choice is the cumulative rule applied to the channel draw
    for j in range(20):
        if res["jump_channels"][j]:
            u = uniform(5, j, 1)
            assert res["jump_channels"][j][0] == (0 if u * (g1 + g2) <= g1 else 1)


@pytest.mark.parametrize("mk", [lambda: W.jaynes_cummings(N=4, nt=31, t_end=60.0),
                                lambda: W.two_level_decay(gamma=0.2, t_end=10.0, nt=11)])
def test_ensemble_mean_matches_mesolve(mk):
    s = mk()
    ntraj = 300
    me = mesolve(s.H, s.c_ops, s.e_ops, s.psi0, s.tlist)
    mc = mcsolve(s.H, s.c_ops, s.e_ops, s.psi0, s.tlist, ntraj=ntraj, seed=1,
                 keep_trajectories=True)
    per = mc["traj_expect"].real
    sd = per.std(axis=0)
    bound = 3 * np.maximum(sd, 1e-3) / math.sqrt(ntraj) + 1e-6
    assert np.all(np.abs(mc["expect"].real - me["expect"].real) <= bound)
