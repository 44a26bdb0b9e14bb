"""The request server: requests submitted while others run are admitted as
memory frees, overlap on the GPU, and each result is bit for bit the result
of the same solve alone."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_util import maxabs, require_gpu

pytestmark = pytest.mark.gpu


def _requests(qtl):
    reqs = []
    for i, (n1, n2) in enumerate([(3, 4), (5, 5), (8, 6), (12, 13), (4, 9)]):
        s = W.coupled_cavities(n1, n2, J=0.3 + 0.1 * i, kappa1=0.05, kappa2=0.1, t_end=10.0, nt=21)
        reqs.append(("mesolve", s, dict(precision="mixed", rtol=1e-7, atol=1e-9), 0, 0))
    for i, ns in enumerate([4, 6, 8]):
        s = W.ising_chain(ns, seed=50 + i, t_end=4.0, nt=9)
        reqs.append(("mcsolve", s, dict(precision="mixed", rtol=1e-7, atol=1e-9), 40 + 20 * i, 7 + i))
    s = W.jaynes_cummings(N=6, nt=11, t_end=30.0)
    reqs.append(("mesolve", s, dict(rtol=1e-8, atol=1e-10), 0, 0))
    return reqs


def _batch_c(n):
    """The batch plan's cluster size: the smallest C in {1, 2, 4, 8, 16} with
    C * 1024 >= n^2 (cluster-kernel mesolve requests are served through the
    batched launch)."""
    for c in (1, 2, 4, 8, 16):
        if c * 1024 >= n * n:
            return c
    return 0


def _alone(qtl, kind, g, s, tol, ntraj, seed):
    if kind == "mesolve":
        c = _batch_c(s.H.shape[0])
        return g.mesolve(s.psi0, s.tlist, cluster_size=c, **tol)["expect"]
    return g.mcsolve(s.psi0, s.tlist, ntraj, seed, **tol)["expect"]


@pytest.mark.parametrize("budget,inflight", [(0, 8), (64 << 20, 2)])
def test_results_in_the_mix_equal_results_alone(budget, inflight):
    qtl = require_gpu()
    reqs = _requests(qtl)
    systems = [qtl.System(s.H, s.c_ops, s.e_ops) for _, s, _, _, _ in reqs]
    srv = qtl.Server(hbm_budget_bytes=budget, max_inflight=inflight)
    tickets = [srv.submit(k, g, s.psi0, s.tlist, qtl.make_opts(**tol), ntraj=nt, seed=sd)
               for (k, s, tol, nt, sd), g in zip(reqs, systems)]
    results = [srv.wait(t) for t in tickets]
    srv.free()
    for (k, s, tol, nt, sd), g, r in zip(reqs, systems, results):
        assert r["status"] == 0
        assert r["t_submit"] <= r["t_start"] <= r["t_end"]
        alone = _alone(qtl, k, g, s, tol, nt, sd)
        assert maxabs(r["expect"], alone) == 0.0
    for g in systems:
        g.free()


def test_continuous_batching_groups_queued_mesolve_requests():
    """Twelve small mesolve requests with one tlist and one set of options,
    submitted while a slow request holds the only slot: they share launches
    (fewer launches than requests), and each result is the solve alone."""
    qtl = require_gpu()
    slow = W.jaynes_cummings(N=6, nt=201, t_end=300.0)
    gs = qtl.System(slow.H, slow.c_ops, slow.e_ops)
    cav = [W.coupled_cavities(n1, n2, J=0.2 + 0.05 * i, kappa1=0.05, kappa2=0.1, t_end=10.0, nt=21)
           for i, (n1, n2) in enumerate([(3, 4), (4, 4), (5, 3), (6, 5), (3, 3), (4, 6)] * 2)]
    systems = [qtl.System(s.H, s.c_ops, s.e_ops) for s in cav]
    tol = dict(precision="mixed", rtol=1e-7, atol=1e-9)
    srv = qtl.Server(hbm_budget_bytes=0, max_inflight=1)
    t_slow = srv.submit("mcsolve", gs, slow.psi0, slow.tlist, qtl.make_opts(), ntraj=2000, seed=3)
    l0 = qtl.launch_count()
    tickets = [srv.submit("mesolve", g, s.psi0, s.tlist, qtl.make_opts(**tol)) for g, s in zip(systems, cav)]
    results = [srv.wait(t) for t in tickets]
    l1 = qtl.launch_count()
    assert srv.wait(t_slow)["status"] == 0
    srv.free()
    assert l1 - l0 < len(cav)
    for s, g, r in zip(cav, systems, results):
        assert r["status"] == 0
        assert maxabs(r["expect"], _alone(qtl, "mesolve", g, s, tol, 0, 0)) == 0.0
    for g in systems + [gs]:
        g.free()


def test_budget_refusal_and_cancel():
    qtl = require_gpu()
    s = W.jaynes_cummings(N=6, nt=201, t_end=300.0)
    g = qtl.System(s.H, s.c_ops, s.e_ops)
    srv = qtl.Server(hbm_budget_bytes=1 << 20, max_inflight=1)
    with pytest.raises(qtl.QtlError) as e:   # 2 x 201 x 4000 x 16 B > 1 MiB
        srv.submit("mcsolve", g, s.psi0, s.tlist, qtl.make_opts(), ntraj=4000, seed=1)
    assert e.value.status == qtl.QTL_ENOMEM
    t1 = srv.submit("mcsolve", g, s.psi0, s.tlist, qtl.make_opts(), ntraj=64, seed=1)
    t2 = srv.submit("mcsolve", g, s.psi0, s.tlist, qtl.make_opts(), ntraj=64, seed=2)
    c = srv.cancel(t2)   # queued behind t1 unless t1 already finished
    r1 = srv.wait(t1)
    r2 = srv.wait(t2)
    assert r1["status"] == 0
    if c == qtl.QTL_OK:
        assert r2["status"] == qtl.QTL_ECANCEL
    else:
        assert r2["status"] == 0
    srv.free()
    g.free()


def test_terms_are_frozen_once_a_request_is_submitted():
    """A submit builds the system's device structures from its terms as they
    are, so a time-dependent term added afterwards is refused and the served
    result is that of the system as submitted."""
    qtl = require_gpu()
    s = W.jaynes_cummings(N=6, nt=11, t_end=5.0)
    g = qtl.System(s.H, s.c_ops, s.e_ops)
    srv = qtl.Server(max_inflight=1)
    t = srv.submit("mesolve", g, s.psi0, s.tlist, qtl.make_opts())
    drive = s.c_ops[0] + s.c_ops[0].conj().T
    with pytest.raises(qtl.QtlError) as e:
        qtl.system_add_td(g.handle, drive, dict(kind="cos", amp=0.1, omega=1.0))
    assert e.value.status == qtl.QTL_EINVAL
    r = srv.wait(t)
    assert r["status"] == 0
    ref = g.mesolve(s.psi0, s.tlist, cluster_size=_batch_c(s.H.shape[0]))["expect"]
    assert np.array_equal(r["expect"], ref)
    srv.free()
    g.free()


def test_served_mixed_results_against_fp64_and_the_oracle():
    """Requests drawn from the serving mix (coupled-cavity mesolve and Ising
    mcsolve, mixed precision, each with its FP64 shadow): every mesolve
    result is within 1e-6 of the FP64 oracle, and of the FP64 solve the
    server ran beside it (err_vs_fp64); every mcsolve result is within
    3 sigma / sqrt(ntraj) of the FP64 ensemble with the same random draws,
    and its reported err_vs_fp64 is that difference."""
    from oracle.mesolve import mesolve as o_me
    qtl = require_gpu()
    mix = W.serving_mix(n_requests=12, seed=5, rate=1000.0, ising_spins=(5, 7),
                        ntraj=(100, 200), cav=(4, 9))
    systems = [qtl.System(r["system"].H, r["system"].c_ops, r["system"].e_ops) for r in mix]
    srv = qtl.Server(max_inflight=8)
    opts = qtl.make_opts(shadow_fp64=True, **dict(precision="mixed", rtol=1e-7, atol=1e-9))
    tickets = [srv.submit(r["kind"], g, r["system"].psi0, r["system"].tlist, opts,
                          ntraj=r.get("ntraj", 0), seed=r.get("seed", 0))
               for r, g in zip(mix, systems)]
    results = [srv.wait(t) for t in tickets]
    srv.free()
    kinds = set()
    for r, g, res in zip(mix, systems, results):
        s = r["system"]
        assert res["status"] == 0
        err = res["stats"]["err_vs_fp64"]
        assert err >= 0.0
        kinds.add(r["kind"])
        if r["kind"] == "mesolve":
            ref = o_me(s.H, s.c_ops, s.e_ops, s.psi0, s.tlist, rtol=1e-8, atol=1e-10)
            assert maxabs(res["expect"], ref["expect"]) <= 1e-6
            assert err <= 1e-6
        else:
            f = g.mcsolve(s.psi0, s.tlist, r["ntraj"], r["seed"], keep_trajectories=True,
                          precision="fp64", rtol=1e-7, atol=1e-9)
            assert err == maxabs(res["expect"], f["expect"])
            sd = f["traj_expect"].real.std(axis=0)
            bound = 3 * np.maximum(sd, 1e-3) / np.sqrt(r["ntraj"]) + 1e-6
            assert np.all(np.abs(res["expect"].real - f["expect"].real) <= bound)
    assert kinds == {"mesolve", "mcsolve"}
    for g in systems:
        g.free()
