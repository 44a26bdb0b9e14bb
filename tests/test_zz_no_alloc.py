"""qtl_mcsolve_noalloc: the mcsolve entry point for callers that cannot
allocate device memory while they solve (during stream capture, under
another allocator's budget, in latency-critical loops).  It must return what
the allocating entry point returns, call after call, although every call
reuses the same fixed device scratch array.  This file is collected last."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle.lindblad import effective_hamiltonian
from tests.gpu_util import maxabs, require_gpu

pytestmark = pytest.mark.gpu


def _dev_csr(m, dev):
    import torch
    m = sp.csr_matrix(m)
    return (torch.from_numpy(np.ascontiguousarray(m.indptr, dtype=np.int32)).to(dev),
            torch.from_numpy(np.ascontiguousarray(m.indices, dtype=np.int32)).to(dev),
            torch.from_numpy(np.ascontiguousarray(m.data, dtype=np.complex128)).to(dev))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_matches_allocating_entry_point_twice(precision):
    qtl = require_gpu()
    import torch
    dev = torch.device("cuda:0")
    s = W.jaynes_cummings(N=10, nt=41, t_end=60.0, kappa=0.1, gamma=0.05)
    ntraj, seed = 64, 9
    tol = dict(precision=precision, rtol=1e-8 if precision == "fp64" else 1e-7,
               atol=1e-10 if precision == "fp64" else 1e-9)
    g = qtl.System(s.H, s.c_ops, s.e_ops)
    ref = g.mcsolve(s.psi0, s.tlist, ntraj, seed, **tol)
    g.free()

    A = (-1j * effective_hamiltonian(s.H, s.c_ops)).tocsr()
    a = _dev_csr(A, dev)
    c = _dev_csr(sp.vstack(s.c_ops), dev)
    o = _dev_csr(sp.vstack(s.e_ops), dev)
    psi = torch.from_numpy(s.psi0).to(dev)
    tl = torch.from_numpy(s.tlist).to(dev)
    stream = torch.cuda.current_stream(dev)
    opts = qtl.make_opts(stream=stream.cuda_stream, **tol)
    bound = 1e-8 if precision == "fp64" else 1e-6
    for _ in range(2):
        ex = torch.full((len(s.e_ops), len(s.tlist)), float("nan"), dtype=torch.complex128, device=dev)
        info = torch.full((5,), -1, dtype=torch.int64, device=dev)
        qtl.mcsolve_noalloc(s.n, a, c, len(s.c_ops), o, len(s.e_ops), psi, tl, ntraj, seed,
                            opts, ex, info)
        torch.cuda.synchronize(dev)
        inf = info.cpu().numpy()
        assert int(inf[0]) & 0xffffffff == 0
        assert int(inf[4]) > 0                      # jumps happened
        assert maxabs(ex.cpu().numpy(), ref["expect"]) <= bound


def test_noalloc_rejects_requests_beyond_its_scratch():
    qtl = require_gpu()
    import torch
    dev = torch.device("cuda:0")
    s = W.two_level_decay()
    a = _dev_csr((-1j * effective_hamiltonian(s.H, s.c_ops)).tocsr(), dev)
    c = _dev_csr(sp.vstack(s.c_ops), dev)
    o = _dev_csr(sp.vstack(s.e_ops), dev)
    psi = torch.from_numpy(s.psi0).to(dev)
    tl = torch.linspace(0, 1, 1000, dtype=torch.float64, device=dev)
    ex = torch.zeros((2, 1000), dtype=torch.complex128, device=dev)
    info = torch.zeros(5, dtype=torch.int64, device=dev)
    opts = qtl.make_opts(stream=torch.cuda.current_stream(dev).cuda_stream)
    # 2 observables x 1000 times x 2000 trajectories x 16 B = 64 MB > 32 MiB
    with pytest.raises(qtl.QtlError) as e:
        qtl.mcsolve_noalloc(2, a, c, 1, o, 2, psi, tl, 2000, 1, opts, ex, info)
    assert e.value.status == qtl.QTL_ETOOBIG


def test_noalloc_reports_a_malformed_operator_in_its_status():
    """A whose row pointers do not end at its entry count, or whose columns
    leave [0, n), is refused by the device-side check with QTL_EINVAL in
    info->status (the trajectory kernel then sees empty rows and reads
    nothing outside the caller's arrays)."""
    qtl = require_gpu()
    import torch
    dev = torch.device("cuda:0")
    s = W.jaynes_cummings(N=4, nt=5, t_end=4.0, kappa=0.1)
    rp, ci, v = _dev_csr((-1j * effective_hamiltonian(s.H, s.c_ops)).tocsr(), dev)
    c = _dev_csr(sp.vstack(s.c_ops), dev)
    o = _dev_csr(sp.vstack(s.e_ops), dev)
    psi = torch.from_numpy(s.psi0).to(dev)
    tl = torch.from_numpy(s.tlist).to(dev)
    opts = qtl.make_opts(stream=torch.cuda.current_stream(dev).cuda_stream)
    bad_col = ci.clone()
    bad_col[-1] = s.n + 5
    for a in [(rp, ci[:-2].clone(), v[:-2].clone()), (rp, bad_col, v)]:
        ex = torch.zeros((len(s.e_ops), len(s.tlist)), dtype=torch.complex128, device=dev)
        info = torch.zeros(5, dtype=torch.int64, device=dev)
        qtl.mcsolve_noalloc(s.n, a, c, len(s.c_ops), o, len(s.e_ops), psi, tl, 4, 1, opts, ex, info)
        torch.cuda.synchronize(dev)
        assert int(info.cpu().numpy()[0]) & 0xffffffff == qtl.QTL_EINVAL


def test_noalloc_call_captured_in_a_cuda_graph():
    """One warm call, then a call captured into a CUDA graph on a side stream
    (global capture mode) and replayed twice: each replay gives the
    allocating entry point's ensemble (the captured host steps set function
    attributes and query occupancy, which capture allows, and allocate
    nothing)."""
    qtl = require_gpu()
    import torch
    dev = torch.device("cuda:0")
    s = W.jaynes_cummings(N=10, nt=41, t_end=60.0, kappa=0.1, gamma=0.05)
    ntraj, seed = 64, 11
    tol = dict(precision="fp64", rtol=1e-8, atol=1e-10)
    g = qtl.System(s.H, s.c_ops, s.e_ops)
    ref = g.mcsolve(s.psi0, s.tlist, ntraj, seed, **tol)
    g.free()
    a = _dev_csr((-1j * effective_hamiltonian(s.H, s.c_ops)).tocsr(), dev)
    c = _dev_csr(sp.vstack(s.c_ops), dev)
    o = _dev_csr(sp.vstack(s.e_ops), dev)
    psi = torch.from_numpy(s.psi0).to(dev)
    tl = torch.from_numpy(s.tlist).to(dev)
    ex = torch.zeros((len(s.e_ops), len(s.tlist)), dtype=torch.complex128, device=dev)
    info = torch.zeros(5, dtype=torch.int64, device=dev)

    def call(stream):
        qtl.mcsolve_noalloc(s.n, a, c, len(s.c_ops), o, len(s.e_ops), psi, tl, ntraj, seed,
                            qtl.make_opts(stream=stream.cuda_stream, **tol), ex, info)

    call(torch.cuda.current_stream(dev))
    torch.cuda.synchronize(dev)
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        call(side)
    for _ in range(2):
        ex.fill_(float("nan"))
        info.fill_(-1)
        graph.replay()
        torch.cuda.synchronize(dev)
        inf = info.cpu().numpy()
        assert int(inf[0]) & 0xffffffff == 0
        assert int(inf[4]) > 0
        assert maxabs(ex.cpu().numpy(), ref["expect"]) <= 1e-8
