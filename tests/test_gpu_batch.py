"""Batched mesolve (parameter sweeps of uneven Kerr cavities in one call):
every solve equals the same system solved alone with the same launch plan,
bit for bit, and agrees with the FP64 oracle."""
import numpy as np
import pytest

import workloads as W
from oracle.mesolve import mesolve as oracle_mesolve
from tests.gpu_util import maxabs, require_gpu

pytestmark = pytest.mark.gpu


def _sweep(k, seed=4, t_end=10.0, nt=21):
    return W.kerr_sweep(n_inst=k, seed=seed, n_min=3, n_max=60, t_end=t_end, nt=nt)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_equals_each_solve_alone(precision):
    qtl = require_gpu()
    sys_ = _sweep(14)
    tol = dict(rtol=1e-8, atol=1e-10) if precision == "fp64" else dict(rtol=1e-7, atol=1e-9)
    handles = [qtl.System(s.H, s.c_ops, s.e_ops) for s in sys_]
    opts = qtl.make_opts(precision=precision, **tol)
    batch = qtl.mesolve_batch([h.handle for h in handles], [h.n_e for h in handles],
                              [s.psi0 for s in sys_], sys_[0].tlist, opts)
    for s, h, b in zip(sys_, handles, batch):
        alone = h.mesolve(s.psi0, s.tlist, precision=precision,
                          cluster_size=qtl.batch_cluster_size(s.n), **tol)
        assert maxabs(alone["expect"], b["expect"]) == 0.0
        assert alone["stats"] == b["stats"]
    for h in handles:
        h.free()


def test_batch_matches_oracle_fixed_step_fp64():
    # dt inside the explicit stability region of the largest cavity
    # (spectral radius ~ K N^2 / 2 ~ 1e3 for N = 60)
    qtl = require_gpu()
    sys_ = _sweep(6, seed=11, t_end=0.2, nt=5)
    handles = [qtl.System(s.H, s.c_ops, s.e_ops) for s in sys_]
    opts = qtl.make_opts(fixed_dt=0.001)
    batch = qtl.mesolve_batch([h.handle for h in handles], [h.n_e for h in handles],
                              [s.psi0 for s in sys_], sys_[0].tlist, opts)
    for s, b in zip(sys_, batch):
        ref = oracle_mesolve(s.H, s.c_ops, s.e_ops, s.psi0, s.tlist, fixed_dt=0.001)
        assert maxabs(b["expect"], ref["expect"]) <= 1e-10
    for h in handles:
        h.free()


def test_batch_mixed_within_1e6_of_oracle():
    qtl = require_gpu()
    sys_ = _sweep(5, seed=21, t_end=20.0, nt=41)
    handles = [qtl.System(s.H, s.c_ops, s.e_ops) for s in sys_]
    opts = qtl.make_opts(precision="mixed", rtol=1e-7, atol=1e-9)
    batch = qtl.mesolve_batch([h.handle for h in handles], [h.n_e for h in handles],
                              [s.psi0 for s in sys_], sys_[0].tlist, opts)
    # against the FP64 oracle at the same tolerances: the difference is the
    # precision error plus two truncation errors of ~rtol each
    for s, b in zip(sys_, batch):
        ref = oracle_mesolve(s.H, s.c_ops, s.e_ops, s.psi0, s.tlist, rtol=1e-7, atol=1e-9)
        assert maxabs(b["expect"], ref["expect"]) <= 1e-6
    for h in handles:
        h.free()


def test_batch_rejects_bad_arguments():
    qtl = require_gpu()
    s = W.kerr_cavity(5, 0.1, 0.2, 0.3, 0.1)
    h = qtl.System(s.H, s.c_ops, s.e_ops)
    with pytest.raises(qtl.QtlError) as e:
        qtl.mesolve_batch([h.handle], [h.n_e], [s.psi0], np.array([0.0, 1.0, 0.5]), qtl.make_opts())
    assert e.value.status == qtl.QTL_EINVAL
    big = W.kerr_cavity(200, 0.1, 0.2, 0.3, 0.1)   # n^2 = 40000 > 16384
    hb = qtl.System(big.H, big.c_ops, big.e_ops)
    with pytest.raises(qtl.QtlError) as e:
        qtl.mesolve_batch([h.handle, hb.handle], [h.n_e, hb.n_e], [s.psi0, big.psi0],
                          np.array([0.0, 1.0]), qtl.make_opts())
    assert e.value.status == qtl.QTL_ETOOBIG
    h.free()
    hb.free()
