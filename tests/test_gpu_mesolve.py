"""GPU parity of mesolve (cluster kernel, through the C ABI) against the FP64
oracle: element-wise on expectation values and states, fixed-step at 1e-10,
adaptive at the solver tolerance, mixed precision at 1e-6, plus edge cases."""
import numpy as np
import pytest

import workloads as W
from oracle.mesolve import mesolve as oracle_mesolve
from tests.gpu_util import maxabs, require_gpu

pytestmark = pytest.mark.gpu


def _gpu(s, tlist, **kw):
    qtl = require_gpu()
    save = kw.pop("save_states", False)
    sysg = qtl.System(s.H, s.c_ops, s.e_ops)
    try:
        return sysg.mesolve(s.psi0, tlist, save_states=save, **kw)
    finally:
        sysg.free()


@pytest.mark.parametrize("method", ["dp5", "tsit5"])
@pytest.mark.parametrize("mk,tl,dt", [
    (lambda: W.driven_cavity(), np.linspace(0, 2, 11), 0.01),
    (lambda: W.jaynes_cummings(), np.linspace(0, 20, 6), 0.05),
    (lambda: W.kerr_cavity(7, 0.3, 0.2, 0.8, 0.1), np.linspace(0, 3, 4), 0.02),
    (lambda: W.ising_chain(5, h=0.9), np.linspace(0, 1, 3), 0.01),
], ids=["cavity20", "jc40x2", "kerr7", "ising5"])
def test_fixed_step_parity_fp64(mk, tl, dt, method):
    s = mk()
    ref = oracle_mesolve(s.H, s.c_ops, s.e_ops, s.psi0, tl, method=method, fixed_dt=dt,
                         save_states=True)
    got = _gpu(s, tl, method=method, fixed_dt=dt, save_states=True)
    assert maxabs(got["expect"], ref["expect"]) <= 1e-10
    assert maxabs(got["states"], ref["states"]) <= 1e-10
    assert got["stats"]["steps_acc"] == ref["stats"]["steps_acc"]
    assert got["stats"]["rhs_evals"] == ref["stats"]["rhs_evals"]


@pytest.mark.parametrize("method", ["dp5", "tsit5"])
def test_adaptive_parity_cavity_full(method):
    s = W.driven_cavity()
    ref = oracle_mesolve(s.H, s.c_ops, s.e_ops, s.psi0, s.tlist, method=method, rtol=s.rtol,
                         atol=s.atol)
    got = _gpu(s, s.tlist, method=method, rtol=s.rtol, atol=s.atol)
    assert maxabs(got["expect"], ref["expect"]) <= 1e-10
    # Landing exactly on tlist makes the step count jump by a few steps when
    # err changes in its last bits (the oracle itself moves from 1590 to
    # 1540 steps under a 1e-15 relative change of err), so counts are
    # compared within 5% while the values are compared at 1e-10.
    assert abs(got["stats"]["steps_acc"] - ref["stats"]["steps_acc"]) <= 0.05 * ref["stats"]["steps_acc"]


def test_adaptive_parity_jc_full():
    s = W.jaynes_cummings()
    ref = oracle_mesolve(s.H, s.c_ops, s.e_ops, s.psi0, s.tlist, rtol=s.rtol, atol=s.atol)
    got = _gpu(s, s.tlist, rtol=s.rtol, atol=s.atol)
    assert maxabs(got["expect"], ref["expect"]) <= 1e-9
    assert abs(got["stats"]["steps_acc"] - ref["stats"]["steps_acc"]) <= 0.05 * ref["stats"]["steps_acc"]


def test_mixed_precision_within_1e6():
    s = W.jaynes_cummings()
    ref = oracle_mesolve(s.H, s.c_ops, s.e_ops, s.psi0, s.tlist, rtol=s.rtol, atol=s.atol)
    got = _gpu(s, s.tlist, rtol=1e-7, atol=1e-9, precision="mixed")
    assert maxabs(got["expect"], ref["expect"]) <= 1e-6
    s0 = W.driven_cavity()
    ref0 = oracle_mesolve(s0.H, s0.c_ops, s0.e_ops, s0.psi0, s0.tlist, rtol=s0.rtol, atol=s0.atol)
    got0 = _gpu(s0, s0.tlist, rtol=1e-7, atol=1e-9, precision="mixed")
    assert maxabs(got0["expect"], ref0["expect"]) <= 1e-6


@pytest.mark.parametrize("cs", [1, 2, 5, 8, 16])
def test_cluster_sizes_agree(cs):
    s = W.jaynes_cummings(N=12, nt=21, t_end=30.0)   # L = 576 fits every cluster size
    ref = oracle_mesolve(s.H, s.c_ops, s.e_ops, s.psi0, s.tlist, fixed_dt=0.05)
    got = _gpu(s, s.tlist, fixed_dt=0.05, cluster_size=cs)
    assert maxabs(got["expect"], ref["expect"]) <= 1e-10


def test_ket_and_density_matrix_inputs_agree():
    qtl = require_gpu()
    s = W.driven_cavity(N=9)
    rho0 = np.outer(s.psi0, s.psi0.conj())
    g = qtl.System(s.H, s.c_ops, s.e_ops)
    a = g.mesolve(s.psi0, s.tlist[:11], fixed_dt=0.02)
    b = g.mesolve(rho0, s.tlist[:11], fixed_dt=0.02)
    g.free()
    assert maxabs(a["expect"], b["expect"]) <= 1e-13


def test_edge_cases():
    qtl = require_gpu()
    s = W.driven_cavity(N=5)
    g = qtl.System(s.H, s.c_ops, s.e_ops)
    # a single output time: only the initial expectation values
    one = g.mesolve(s.psi0, np.array([0.0]))
    ref = oracle_mesolve(s.H, s.c_ops, s.e_ops, s.psi0, np.array([0.0]))
    assert maxabs(one["expect"], ref["expect"]) <= 1e-14
    # repeated output times
    tl = np.array([0.0, 0.5, 0.5, 1.0])
    r1 = g.mesolve(s.psi0, tl, fixed_dt=0.1)
    r2 = oracle_mesolve(s.H, s.c_ops, s.e_ops, s.psi0, tl, fixed_dt=0.1)
    assert maxabs(r1["expect"], r2["expect"]) <= 1e-12
    # invalid arguments are refused with a status, not a fault
    with pytest.raises(qtl.QtlError) as e:
        g.mesolve(s.psi0, np.array([0.0, 1.0, 0.5]))
    assert e.value.status == qtl.QTL_EINVAL
    bad = s.psi0.copy()
    bad[0] = np.nan
    with pytest.raises(qtl.QtlError) as e:
        g.mesolve(bad, s.tlist[:3])
    assert e.value.status == qtl.QTL_EINVAL
    with pytest.raises(qtl.QtlError) as e:
        g.mesolve(s.psi0, s.tlist, max_steps=5)
    assert e.value.status == qtl.QTL_ESTEP
    with pytest.raises(qtl.QtlError) as e:
        g.mesolve(s.psi0, s.tlist[:3], rtol=-1.0)
    assert e.value.status == qtl.QTL_EINVAL
    g.free()
    # no observables
    g2 = qtl.System(s.H, s.c_ops, [])
    out = g2.mesolve(s.psi0, s.tlist[:5], save_states=True, fixed_dt=0.05)
    ref = oracle_mesolve(s.H, s.c_ops, [], s.psi0, s.tlist[:5], fixed_dt=0.05, save_states=True)
    assert maxabs(out["states"], ref["states"]) <= 1e-12
    g2.free()
    # no collapse operators (unitary): trace and purity are conserved
    g3 = qtl.System(s.H, [], s.e_ops)
    u = g3.mesolve(s.psi0, s.tlist[:21], save_states=True)
    for rho in u["states"]:
        assert abs(np.trace(rho) - 1) < 1e-9
        assert abs(np.trace(rho @ rho) - 1) < 1e-8
    g3.free()


def test_too_big_for_a_cluster():
    """n*n = 262144 is beyond one cluster: forcing the cluster kernel is refused
    with a status, the automatic choice runs it on the grid kernel."""
    qtl = require_gpu()
    s = W.ising_chain(9, h=1.0)
    g = qtl.System(s.H, s.c_ops, s.e_ops)
    with pytest.raises(qtl.QtlError) as e:
        g.mesolve(s.psi0, np.array([0.0, 0.1]), engine="cluster")
    assert e.value.status == qtl.QTL_ETOOBIG
    out = g.mesolve(s.psi0, np.array([0.0, 0.05, 0.1]), precision="mixed", rtol=1e-7, atol=1e-9)
    g.free()
    assert np.all(np.isfinite(out["expect"]))
    assert abs(out["expect"][2, 0].real - 9.0) < 1e-12   # all spins up at t = 0


def test_async_device_path_matches_host_path():
    qtl = require_gpu()
    import torch
    s = W.jaynes_cummings(N=10, nt=11, t_end=10.0)
    g = qtl.System(s.H, s.c_ops, s.e_ops)
    host = g.mesolve(s.psi0, s.tlist)
    dev = torch.device("cuda:0")
    psi = torch.from_numpy(s.psi0).to(dev)
    tl = torch.from_numpy(s.tlist).to(dev)
    ex = torch.zeros((len(s.e_ops), len(s.tlist)), dtype=torch.complex128, device=dev)
    info = torch.zeros(qtl.DEVICE_INFO_BYTES // 8, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    qtl.mesolve_async(g.handle, psi, 1, tl, qtl.make_opts(stream=stream.cuda_stream), ex, None,
                      info)
    torch.cuda.synchronize()
    assert int(info[0].item() & 0xffffffff) == 0
    assert maxabs(ex.cpu().numpy(), host["expect"]) == 0.0
    g.free()


def test_entry_type_counts_of_a_and_the_liouvillian():
    """qtl_system_nnz's counts of entries with a zero real or imaginary part
    (the products that take 4 flops, not 8), against their closed forms for
    a driven damped cavity H = D a^dag a + F (a + a^dag), C = sqrt(k) a with
    dyadic D, F, k, where every entry's real and imaginary parts are exact:
    A = -i H - (k/2) a^dag a has N - 1 complex diagonal entries (n = 0 is
    zero) and 2 (N - 1) imaginary off-diagonal ones; the Liouvillian has
    N^2 - 1 diagonal entries -i D (i - j) - (k/2)(i + j), real for the N - 1
    with i = j, (N - 1)^2 real jump entries k sqrt((i+1)(j+1)) and 4 N (N - 1)
    imaginary drive entries."""
    import scipy.sparse as sp
    qtl = require_gpu()
    N, D, F, k = 6, 0.5, 0.25, 1.0
    a = sp.diags(np.sqrt(np.arange(1, N)), 1, format="csr", dtype=complex)
    H = D * (a.conj().T @ a) + F * (a + a.conj().T)
    g = qtl.System(H, [np.sqrt(k) * a], [a.conj().T @ a])
    try:
        assert qtl.system_nnz(g.handle, 1) == 3 * (N - 1)
        assert qtl.system_nnz(g.handle, 3) == 2 * (N - 1)
        psi0 = np.zeros(N, complex)
        psi0[0] = 1.0
        g.mesolve(psi0, np.linspace(0.0, 0.5, 3))
        assert qtl.system_nnz(g.handle, 2) == (N * N - 1) + (N - 1) ** 2 + 4 * N * (N - 1)
        assert qtl.system_nnz(g.handle, 4) == (N - 1) + (N - 1) ** 2 + 4 * N * (N - 1)
    finally:
        g.free()
