"""The reduced-precision form's error against FP64, reported per result by
the library (qtl_stats.err_vs_fp64 with opts.shadow_fp64), and held to the
1e-6 bar on every expectation value, up to the full 10-spin chain (a density
matrix with 2^20 entries)."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_util import maxabs, require_gpu

pytestmark = pytest.mark.gpu

MIXED = dict(precision="mixed", rtol=1e-7, atol=1e-9)


def test_mesolve_reports_its_error_against_fp64():
    qtl = require_gpu()
    s = W.jaynes_cummings(N=10, nt=101, t_end=200.0, kappa=0.1, gamma=0.05)
    g = qtl.System(s.H, s.c_ops, s.e_ops)
    try:
        mixed = g.mesolve(s.psi0, s.tlist, shadow_fp64=True, **MIXED)
        plain = g.mesolve(s.psi0, s.tlist, **MIXED)
        fp64 = g.mesolve(s.psi0, s.tlist, **dict(MIXED, precision="fp64"))
    finally:
        g.free()
    err = mixed["stats"]["err_vs_fp64"]
    assert err == maxabs(mixed["expect"], fp64["expect"])   # the shadow is that FP64 solve
    assert 0.0 < err <= 1e-6
    assert maxabs(mixed["expect"], plain["expect"]) == 0.0   # the shadow does not touch the result
    assert plain["stats"]["err_vs_fp64"] == -1.0
    assert fp64["stats"]["err_vs_fp64"] == 0.0


def test_mcsolve_reports_its_error_against_fp64():
    qtl = require_gpu()
    s = W.jaynes_cummings(N=8, nt=41, t_end=80.0, kappa=0.1, gamma=0.05)
    g = qtl.System(s.H, s.c_ops, s.e_ops)
    try:
        mixed = g.mcsolve(s.psi0, s.tlist, 200, 3, shadow_fp64=True, **MIXED)
        fp64 = g.mcsolve(s.psi0, s.tlist, 200, 3, **dict(MIXED, precision="fp64"))
    finally:
        g.free()
    assert mixed["stats"]["err_vs_fp64"] == maxabs(mixed["expect"], fp64["expect"])
    assert fp64["stats"]["err_vs_fp64"] == 0.0


def test_ising10_full_span_mixed_within_1e6_of_fp64():
    """The 10-spin chain over its whole span (t in [0, 10], 100 output
    times, adaptive): the mixed solve against the FP64 grid solve of the same
    system at the same tolerances (the FP64 grid kernel is checked against
    the oracle entry by entry elsewhere) and against a tighter FP64 solve, on
    every Sx, Sy, Sz value."""
    qtl = require_gpu()
    s = W.ising_chain(10)
    g = qtl.System(s.H, s.c_ops, s.e_ops)
    try:
        mixed = g.mesolve(s.psi0, s.tlist, shadow_fp64=True, **MIXED)
        tight = g.mesolve(s.psi0, s.tlist, precision="fp64", rtol=1e-10, atol=1e-12)
    finally:
        g.free()
    assert mixed["stats"]["err_vs_fp64"] <= 1e-6
    assert maxabs(mixed["expect"], tight["expect"]) <= 1e-6
