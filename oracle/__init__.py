"""FP64 CPU oracle for the Lindblad / quantum-trajectory hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may import
or call this package; only the tests, `__graft_entry__.smoke()` and the
benchmark's CPU-baseline leg use it.  It shares no code with the CUDA path;
the only code both sides consume is the `workloads` input generator.

Everything is plain NumPy / SciPy in float64 / complex128, written step by
step after the paper:
  lindblad.py  the master equation (Sec. 3.2, eq. for d rho/dt and the
               Lindblad dissipator) as a Liouvillian superoperator and as a
               plain matrix product; the effective Hamiltonian (Sec. 3.3)
  tableau.py   Dormand-Prince 5(4) and Tsitouras 5(4) coefficients
  integrate.py embedded RK step, error norm, PI controller, starting step,
               tlist landing (the paper names no integrator; integrate.py
               states each reading it uses)
  mesolve.py   mesolve with expectation values Tr(O rho) (Sec. 3.2)
  philox.py    Philox4x32-10 counter-based generator (Salmon et al. 2011)
  mcsolve.py   Monte-Carlo wave-function method (Sec. 3.3)
  timedep.py   time-dependent Hamiltonians H0 + sum_k f_k(t) H_k (Sec. 2,
               Sec. 3.2) for mesolve and mcsolve; sesolve (Sec. 3.1)
  stochastic.py  the stochastic Schroedinger and master equations under
               homodyne detection (Sec. 3.4), Euler-Maruyama
  steadystate.py stationary states: direct solve with the trace condition
               (Sec. 3.2) and the Fourier-component system of Appendix A
  dsf.py       the dynamical shifted Fock master equation (Sec. 3.6,
               Appendix B, Algorithm 1)

Parity status: every function here is pinned by tests/test_oracle_*.py to
closed forms, brute-force matrix exponentials, invariants, order conditions
or published known-answer vectors, except where a docstring says
"parity unpinned".
"""
