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


def _alone(qtl, kind, g, s, tol, ntraj, seed):
    if kind == "mesolve":
        return g.mesolve(s.psi0, s.tlist, **tol)["expect"]
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
