"""Batch plans (qtl_batch_*): the launch sequence of a parameter sweep is
captured once in a CUDA graph and replayed; the autotuner picks a cluster
size per group.  Every replay gives the same results, which equal the
one-shot batched call (untuned) or each system solved alone with its group's
cluster size (tuned), bit for bit."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_util import maxabs, require_gpu

pytestmark = pytest.mark.gpu


def _setup(qtl, k, seed, precision):
    import torch
    dev = torch.device("cuda", 0)
    sys_ = W.kerr_sweep(n_inst=k, seed=seed, n_min=3, n_max=60, t_end=10.0, nt=21)
    handles = [qtl.System(s.H, s.c_ops, s.e_ops) for s in sys_]
    states = [torch.from_numpy(s.psi0).to(dev) for s in sys_]
    tl = torch.from_numpy(sys_[0].tlist).to(dev)
    exps = [torch.zeros((2, len(sys_[0].tlist)), dtype=torch.complex128, device=dev) for _ in sys_]
    info = torch.zeros((k, 5), dtype=torch.int64, device=dev)
    tol = dict(rtol=1e-8, atol=1e-10) if precision == "fp64" else dict(rtol=1e-7, atol=1e-9)
    stream = torch.cuda.current_stream(dev)
    opts = qtl.make_opts(precision=precision, stream=stream.cuda_stream, **tol)
    return sys_, handles, states, tl, exps, info, opts, tol, stream


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_untuned_plan_replays_equal_the_batched_call(precision):
    import torch
    qtl = require_gpu()
    sys_, handles, states, tl, exps, info, opts, tol, stream = _setup(qtl, 16, 4, precision)
    hs = [h.handle for h in handles]
    qtl.mesolve_batch_async(hs, states, [1] * len(hs), tl, opts, exps, info)
    torch.cuda.synchronize()
    ref = [e.cpu().numpy().copy() for e in exps]
    ref_info = info.cpu().numpy().copy()
    plan = qtl.Batch(hs, states, [1] * len(hs), tl, opts, exps, info, autotune=False)
    for _ in range(2):
        for e in exps:
            e.zero_()
        info.zero_()
        plan.launch(stream.cuda_stream)
        torch.cuda.synchronize()
        assert all(maxabs(e.cpu().numpy(), r) == 0.0 for e, r in zip(exps, ref))
        assert np.array_equal(info.cpu().numpy(), ref_info)
    assert all(int(s) & 0xffffffff == 0 for s in ref_info[:, 0])
    plan.free()
    for h in handles:
        h.free()


def test_autotuned_plan_equals_each_solve_alone_at_its_cluster_size():
    import torch
    qtl = require_gpu()
    sys_, handles, states, tl, exps, info, opts, tol, stream = _setup(qtl, 24, 7, "mixed")
    hs = [h.handle for h in handles]
    plan = qtl.Batch(hs, states, [1] * len(hs), tl, opts, exps, info, autotune=True)
    groups = plan.groups()
    assert sum(g[1] for g in groups) == len(hs)
    tuned = [g for g in groups if len(g[2]) >= 2]
    assert tuned, groups          # at least one group had a choice
    for cs, _, cands in tuned:
        assert cs in [c for c, _ in cands]
        assert cs == min(cands, key=lambda x: x[1])[0]
        assert all(ms > 0 for _, ms in cands)
    outs = []
    for _ in range(2):
        plan.launch(stream.cuda_stream)
        torch.cuda.synchronize()
        outs.append([e.cpu().numpy().copy() for e in exps])
    assert all(maxabs(a, b) == 0.0 for a, b in zip(outs[0], outs[1]))
    for b, (s, h) in enumerate(zip(sys_, handles)):
        cs = groups[plan.group_of(b)][0]
        alone = h.mesolve(s.psi0, s.tlist, precision="mixed", cluster_size=cs, **tol)
        assert maxabs(alone["expect"], outs[1][b]) == 0.0
    plan.free()
    for h in handles:
        h.free()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_plan_with_time_dependent_systems_replays_equal_the_batched_call(precision):
    """Driven cavities (a cos drive term each) among time-independent Kerr
    cavities: the untuned plan's replays equal the one-shot batched call bit
    for bit."""
    import scipy.sparse as sp
    import torch
    qtl = require_gpu()
    dev = torch.device("cuda", 0)
    sys_ = W.kerr_sweep(n_inst=4, seed=4, n_min=6, n_max=20, t_end=4.0, nt=9)
    handles = [qtl.System(s.H, s.c_ops, s.e_ops) for s in sys_]
    kets = [s.psi0 for s in sys_]
    for N, D, F, w in [(12, 0.7, 0.4, 1.1), (16, 0.3, 0.9, 0.8)]:
        a = sp.diags(np.sqrt(np.arange(1, N)), 1, format="csr", dtype=complex)
        td = [((a + a.conj().T).tocsr(), dict(kind="cos", amp=F, omega=w))]
        handles.append(qtl.System(D * (a.conj().T @ a), [np.sqrt(0.5) * a], [a, a.conj().T @ a], td=td))
        kets.append(np.eye(N)[0].astype(complex))
    hs = [h.handle for h in handles]
    states = [torch.from_numpy(k).to(dev) for k in kets]
    tl = torch.from_numpy(sys_[0].tlist).to(dev)
    exps = [torch.zeros((2, len(sys_[0].tlist)), dtype=torch.complex128, device=dev) for _ in handles]
    info = torch.zeros((len(handles), 5), dtype=torch.int64, device=dev)
    tol = dict(rtol=1e-8, atol=1e-10) if precision == "fp64" else dict(rtol=1e-7, atol=1e-9)
    stream = torch.cuda.current_stream(dev)
    opts = qtl.make_opts(precision=precision, stream=stream.cuda_stream, **tol)
    qtl.mesolve_batch_async(hs, states, [1] * len(hs), tl, opts, exps, info)
    torch.cuda.synchronize()
    ref = [e.cpu().numpy().copy() for e in exps]
    ref_info = info.cpu().numpy().copy()
    assert all(int(s) & 0xffffffff == 0 for s in ref_info[:, 0])
    plan = qtl.Batch(hs, states, [1] * len(hs), tl, opts, exps, info, autotune=False)
    for _ in range(2):
        for e in exps:
            e.zero_()
        info.zero_()
        plan.launch(stream.cuda_stream)
        torch.cuda.synchronize()
        assert all(maxabs(e.cpu().numpy(), r) == 0.0 for e, r in zip(exps, ref))
    plan.free()
    for h in handles:
        h.free()
