"""GPU parity of mcsolve above the register-resident size (n > 1024): the
1024-thread trajectory kernel with its state in global memory, through the
C ABI, against the FP64 oracle trajectory by trajectory; the same kernel
forced at small n against the register-resident kernel; and the 14-spin
chain (n = 16,384) at 2000 trajectories, the configured size, on trajectories
sampled from the full launch and recomputed one by one by the oracle."""
import math

import numpy as np
import pytest

import workloads as W
from oracle.mcsolve import mcsolve as oracle_mcsolve
from tests.gpu_util import maxabs, require_gpu

pytestmark = pytest.mark.gpu


def _gpu(s, tlist, ntraj, seed, **kw):
    qtl = require_gpu()
    off = kw.pop("traj_offset", 0)
    g = qtl.System(s.H, s.c_ops, s.e_ops)
    try:
        return g.mcsolve(s.psi0, tlist, ntraj, seed, traj_offset=off, keep_trajectories=True, **kw)
    finally:
        g.free()


def test_wide_kernel_matches_register_kernel():
    """Forced onto the global-memory kernel at n = 10, trajectories equal the
    register-resident kernel's up to summation order."""
    s = W.jaynes_cummings(N=5, nt=41, t_end=80.0, kappa=0.1, gamma=0.05)
    a = _gpu(s, s.tlist, 24, 7, engine="cluster")
    b = _gpu(s, s.tlist, 24, 7, engine="grid")
    assert a["stats"]["jumps"] == b["stats"]["jumps"]
    assert maxabs(a["traj_expect"], b["traj_expect"]) <= 1e-9


def test_wide_fixed_step_parity_ising11():
    """11 spins (n = 2048, two rows per thread), fixed steps with jumps."""
    s = W.ising_chain(11, t_end=2.0, nt=11)
    ref = oracle_mcsolve(s.H, s.c_ops, s.e_ops, s.psi0, s.tlist, ntraj=6, seed=12,
                         fixed_dt=0.01, keep_trajectories=True)
    got = _gpu(s, s.tlist, 6, 12, fixed_dt=0.01)
    assert got["stats"]["jumps"] == ref["stats"]["jumps"] > 0
    assert maxabs(got["traj_expect"], ref["traj_expect"]) <= 1e-10


def test_wide_adaptive_parity_ragged():
    """n = 2200 (a ragged last row block of 152), adaptive steps."""
    s = W.jaynes_cummings(N=1100, nt=31, t_end=60.0, kappa=0.1, gamma=0.05)
    assert s.H.shape[0] == 2200
    ref = oracle_mcsolve(s.H, s.c_ops, s.e_ops, s.psi0, s.tlist, ntraj=8, seed=5,
                         keep_trajectories=True)
    got = _gpu(s, s.tlist, 8, 5)
    assert got["stats"]["jumps"] == ref["stats"]["jumps"] > 0
    assert maxabs(got["traj_expect"], ref["traj_expect"]) <= 1e-8
    assert maxabs(got["expect"], ref["expect"]) <= 1e-8


def test_wide_int32_columns_ising17():
    """17 spins (n = 131,072): column indices no longer fit in 16 bits and
    the stage inputs no longer fit in shared memory."""
    s = W.ising_chain(17, gamma=0.5, t_end=0.3, nt=4)
    ref = oracle_mcsolve(s.H, s.c_ops, s.e_ops, s.psi0, s.tlist, ntraj=3, seed=21,
                         fixed_dt=0.01, keep_trajectories=True)
    for prec, tol in (("fp64", 1e-10), ("mixed", 1e-6)):
        got = _gpu(s, s.tlist, 3, 21, fixed_dt=0.01, precision=prec)
        assert got["stats"]["jumps"] == ref["stats"]["jumps"] > 0
        assert maxabs(got["traj_expect"], ref["traj_expect"]) <= tol


MIXED = dict(precision="mixed", rtol=1e-7, atol=1e-9)


def test_wide_mixed_precision_ising11():
    """Mixed-precision trajectories against the oracle run at the same
    tolerances, trajectory by trajectory, at the 1e-6 bar."""
    s = W.ising_chain(11, t_end=4.0, nt=21)
    ref = oracle_mcsolve(s.H, s.c_ops, s.e_ops, s.psi0, s.tlist, ntraj=8, seed=3,
                         rtol=1e-7, atol=1e-9, keep_trajectories=True)
    got = _gpu(s, s.tlist, 8, 3, **MIXED)
    assert got["stats"]["jumps"] == ref["stats"]["jumps"] > 0
    assert maxabs(got["traj_expect"], ref["traj_expect"]) <= 1e-6


def test_wide_edge_cases():
    qtl = require_gpu()
    s = W.ising_chain(11)
    g = qtl.System(s.H, s.c_ops, s.e_ops)
    try:
        one = g.mcsolve(s.psi0, np.array([0.0]), 3, 1)
        assert maxabs(one["expect"][2], [11.0]) < 1e-12  # all spins excited: Sz = 11
        # repeated output times, a single trajectory
        tl = np.array([0.0, 0.5, 0.5, 1.0])
        rep = g.mcsolve(s.psi0, tl, 1, 4, keep_trajectories=True)
        assert maxabs(rep["traj_expect"][0][:, 1], rep["traj_expect"][0][:, 2]) == 0.0
        with pytest.raises(qtl.QtlError) as e:
            g.mcsolve(s.psi0, s.tlist, 2, 1, engine="cluster")
        assert e.value.status == qtl.QTL_ETOOBIG
    finally:
        g.free()


def test_ising14_full_size_sampled():
    """The 14-spin chain (n = 16,384) with 2000 trajectories in mixed
    precision, one launch as the benchmark runs it; trajectories 0 and 1999
    recomputed one by one by the FP64 oracle.  The FP64 kernel is checked on
    the same two trajectories (traj_offset selects their streams)."""
    s = W.ising_chain(14, t_end=2.0, nt=21)
    ids = [0, 1999]
    # the oracle at the mixed solve's tolerances (rtol 1e-7), and at the FP64
    # defaults (rtol 1e-8) for the FP64 kernel
    ref7 = oracle_mcsolve(s.H, s.c_ops, s.e_ops, s.psi0, s.tlist, ntraj=len(ids), seed=9,
                          traj_ids=ids, rtol=1e-7, atol=1e-9, keep_trajectories=True)
    ref = oracle_mcsolve(s.H, s.c_ops, s.e_ops, s.psi0, s.tlist, ntraj=len(ids), seed=9,
                         traj_ids=ids, keep_trajectories=True)
    mixed = _gpu(s, s.tlist, 2000, 9, **MIXED)
    for i, j in enumerate(ids):
        assert maxabs(mixed["traj_expect"][j], ref7["traj_expect"][i]) <= 1e-6
    # ensemble: Sz decays from 14; |Sx|, |Sy| <= 14 on every trajectory
    per = mixed["traj_expect"]
    assert np.all(np.abs(per.real) <= 14 + 1e-6)
    assert np.all(np.abs(per.imag) <= 1e-6)
    for i, j in enumerate(ids):
        f = _gpu(s, s.tlist, 1, 9, traj_offset=j)
        assert maxabs(f["traj_expect"][0], ref["traj_expect"][i]) <= 1e-8


def test_ising14_full_span_mixed_within_1e6_of_fp64():
    """The benchmark's 14-spin solve over its whole span (t in [0, 10], 100
    output times, seed 3), 152 trajectories (one per SM), mixed precision
    against the FP64 kernel with the same draws (itself checked against the
    oracle above).
    - Fixed steps of 0.0125 (the adaptive solve's typical step): both sides
      take the same steps, so the difference is the arithmetic alone; every
      trajectory and every Sx, Sy, Sz value is within 1e-6.
    - Adaptive (rtol 1e-7): the reported ensemble means are within 1e-6,
      and the library's err_vs_fp64 is that difference.  Single adaptive
      trajectories are not compared at 1e-6: two solves at rtol 1e-7 that
      take different steps already differ by the truncation error (FP64 at
      rtol 1e-7 against FP64 at rtol 1e-9: 1.4e-6 on Sz)."""
    qtl = require_gpu()
    s = W.ising_chain(14)
    g = qtl.System(s.H, s.c_ops, s.e_ops)
    try:
        fm = g.mcsolve(s.psi0, s.tlist, 152, 3, keep_trajectories=True, precision="mixed", fixed_dt=0.0125)
        ff = g.mcsolve(s.psi0, s.tlist, 152, 3, keep_trajectories=True, precision="fp64", fixed_dt=0.0125)
        m = g.mcsolve(s.psi0, s.tlist, 152, 3, **MIXED)
        f = g.mcsolve(s.psi0, s.tlist, 152, 3, **dict(MIXED, precision="fp64"))
        sh = g.mcsolve(s.psi0, s.tlist, 152, 3, shadow_fp64=True, **MIXED)
    finally:
        g.free()
    assert fm["stats"]["jumps"] == ff["stats"]["jumps"] > 0
    assert maxabs(fm["traj_expect"], ff["traj_expect"]) <= 1e-6
    assert maxabs(m["expect"], f["expect"]) <= 1e-6
    assert sh["stats"]["err_vs_fp64"] == maxabs(m["expect"], f["expect"])


def test_ising14_mixed_ensemble_within_sampling_error_of_fp64():
    """600 trajectories of the 14-spin chain: the mixed ensemble mean is
    within 3 sigma / sqrt(ntraj) of the FP64 ensemble at every time."""
    qtl = require_gpu()
    s = W.ising_chain(14)
    g = qtl.System(s.H, s.c_ops, s.e_ops)
    try:
        m = g.mcsolve(s.psi0, s.tlist, 600, 5, **MIXED)
        f = g.mcsolve(s.psi0, s.tlist, 600, 5, keep_trajectories=True, **dict(MIXED, precision="fp64"))
    finally:
        g.free()
    sd = f["traj_expect"].real.std(axis=0)
    bound = 3 * np.maximum(sd, 1e-3) / math.sqrt(600) + 1e-6
    assert np.all(np.abs(m["expect"].real - f["expect"].real) <= bound)
