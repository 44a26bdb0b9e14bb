"""Stationary states (Sec. 3.2, steadystate; Appendix A, steadystate_fourier).

TEST INFRASTRUCTURE ONLY (see the package docstring).

steadystate: the density matrix with L vec(rho) = 0 and Tr rho = 1, solved
directly (one equation of L vec(rho) = 0 is redundant, since Tr(L rho) = 0 for
every rho; it is replaced by the trace condition).

steadystate_fourier: for d rho/dt = [L0 + L1 e^{i w t} + L_{-1} e^{-i w t}] rho,
the periodic long-time solution rho(t) = sum_n rho_n e^{i n w t} satisfies
    (L0 - i n w) rho_n + L1 rho_{n-1} + L_{-1} rho_{n+1} = 0,
a block-tridiagonal system over n = -nmax..nmax (components beyond the cutoff
set to zero), solved directly with Tr rho_0 = 1 replacing one equation of
the n = 0 block.  A drive F cos(w t) X gives L_{+1} = L_{-1} = -i[(F/2) X, .].
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .lindblad import liouvillian


def _trace_row(n):
    """Row vector w with w . vec(rho) = Tr rho (column stacking)."""
    w = np.zeros(n * n, dtype=np.complex128)
    w[np.arange(n) * (n + 1)] = 1.0
    return w


def steadystate(H, c_ops):
    """rho_ss with L vec(rho_ss) = 0, Tr rho_ss = 1 (direct sparse solve)."""
    n = H.shape[0]
    L = sp.lil_matrix(liouvillian(H, c_ops))
    L[0, :] = _trace_row(n)
    b = np.zeros(n * n, dtype=np.complex128)
    b[0] = 1.0
    v = spla.spsolve(sp.csc_matrix(L), b)
    return v.reshape((n, n), order="F")


def steadystate_fourier(H0, c_ops, X, F, w, nmax):
    """Fourier components rho_n (n = -nmax..nmax) of the periodic steady state
    under H0 + F cos(w t) X.  Returns dict n -> rho_n (n x n)."""
    n = H0.shape[0]
    N2 = n * n
    L0 = sp.csr_matrix(liouvillian(H0, c_ops))
    L1 = sp.csr_matrix(liouvillian((F / 2.0) * sp.csr_matrix(X, dtype=np.complex128), []))
    I = sp.identity(N2, dtype=np.complex128, format="csr")
    ks = list(range(-nmax, nmax + 1))
    blocks = [[None] * len(ks) for _ in ks]
    for a, k in enumerate(ks):
        blocks[a][a] = L0 - 1j * k * w * I
        if a > 0:
            blocks[a][a - 1] = L1          # L_{+1} rho_{k-1}
        if a + 1 < len(ks):
            blocks[a][a + 1] = L1          # L_{-1} rho_{k+1}
    A = sp.lil_matrix(sp.bmat(blocks, format="csr"))
    r0 = nmax * N2                         # first equation of the n = 0 block
    A[r0, :] = 0.0
    A[r0, r0:r0 + N2] = _trace_row(n)
    b = np.zeros(len(ks) * N2, dtype=np.complex128)
    b[r0] = 1.0
    v = spla.spsolve(sp.csc_matrix(A), b)
    return {k: v[a * N2:(a + 1) * N2].reshape((n, n), order="F") for a, k in enumerate(ks)}
