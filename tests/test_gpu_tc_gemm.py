"""Dense complex products (qtl_zgemm_async): the FP64 path and the
split-BF16 tensor-core path (tcgen05) against NumPy, and the stationary-state
solve with the tensor-core preconditioner against the oracle's direct solve."""
import numpy as np
import pytest

import workloads as W
from oracle.steadystate import steadystate as o_ss
from tests.gpu_util import maxabs, require_gpu

pytestmark = pytest.mark.gpu


def _dev(qtl, M):
    import torch
    # column-major storage: the transpose's C-order buffer
    return torch.from_numpy(np.ascontiguousarray(M.T)).to("cuda:0")


def _op(M, op):
    return M.conj().T if op else M


@pytest.mark.parametrize("n", [16, 40, 130, 300])
@pytest.mark.parametrize("ops", [(0, 0), (0, 1), (1, 0)])
def test_zgemm_fp64_and_tensor_core(n, ops):
    qtl = require_gpu()
    import torch
    rng = np.random.default_rng(n + 7 * ops[0] + 3 * ops[1])
    A = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    B = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    ref = _op(A, ops[0]) @ _op(B, ops[1])
    scale = np.abs(_op(A, ops[0])) @ np.abs(_op(B, ops[1]))
    Ad, Bd = _dev(qtl, A), _dev(qtl, B)
    err = torch.zeros(1, dtype=torch.int32, device="cuda:0")
    for prec, tol in (("fp64", 1e-13), ("mixed", 4e-5)):
        Cd = torch.full((n, n), complex("nan"), dtype=torch.complex128, device="cuda:0")
        qtl.zgemm_async(Ad, Bd, Cd, ops[0], ops[1], precision=prec,
                        stream=torch.cuda.current_stream().cuda_stream, err=err)
        torch.cuda.synchronize()
        C = Cd.cpu().numpy().T
        assert np.all(np.abs(C - ref) <= tol * scale), prec
    assert int(err.item()) == 0


@pytest.mark.parametrize("name", ["cavity40", "jc40x2", "kerr30"])
def test_steadystate_with_the_tensor_core_preconditioner(name):
    """The preconditioner is applied in split BF16 on the tensor cores; the
    Krylov vectors, the products with L and the residual stay FP64, so the
    result is the direct solve's to 1e-10, in a few more iterations."""
    qtl = require_gpu()
    if name == "cavity40":
        s = W.driven_cavity(N=40)
    elif name == "jc40x2":
        s = W.jaynes_cummings(N=40)
    else:
        s = W.kerr_cavity(30, 0.5, 0.2, 1.0, 0.1)
    ref = o_ss(s.H, s.c_ops)
    g = qtl.System(s.H, s.c_ops, [])
    try:
        f = g.steadystate()
        m = g.steadystate(precision="mixed")
    finally:
        g.free()
    assert maxabs(m["rho"], ref) <= 1e-10
    assert m["stats"]["residual"] <= 1e-11
    assert m["stats"]["iterations"] <= f["stats"]["iterations"] + 20
