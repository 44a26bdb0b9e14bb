"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package builds the *inputs* of a solve: operator matrices (H, collapse
operators C_k, observables O_k), the initial state and the time grid, with
random parameters drawn from fixed seeds.  It contains none of the solver's
arithmetic (no Liouvillian, no effective Hamiltonian, no integrator), so that
the FP64 oracle and the CUDA library can both consume it without sharing any
part of the method.
"""
from .operators import (dag, destroy, qeye, sigmaz, sigmax, sigmay, sigmam, sigmap,
                        tensor, fock, coherent, site_operator)
from .systems import (System, driven_cavity, jaynes_cummings, ising_chain,
                      kerr_cavity, kerr_sweep, coupled_cavities, damped_oscillator,
                      thermal_oscillator, two_level_decay, serving_mix, CONFIGS)

__all__ = [
    "dag", "destroy", "qeye", "sigmaz", "sigmax", "sigmay", "sigmam", "sigmap", "tensor",
    "fock", "coherent", "site_operator", "System", "driven_cavity", "jaynes_cummings",
    "ising_chain", "kerr_cavity", "kerr_sweep", "coupled_cavities", "damped_oscillator",
    "thermal_oscillator", "two_level_decay", "serving_mix", "CONFIGS",
]
