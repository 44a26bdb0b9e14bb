"""Lindblad master equation, Sec. 3.2 and Sec. 3.3 of the paper.

    d rho / dt = L rho = -i [H, rho] + sum_k D[C_k] rho,
    D[C] rho   = C rho C^dag - 1/2 (C^dag C rho + rho C^dag C).

The dissipator is printed in the paper with a minus sign inside the bracket,
which would make it a commutator and break trace preservation; the
anticommutator is the Lindblad form (and the one consistent with the
effective Hamiltonian of Sec. 3.3), so it is used here.

Vectorisation is column stacking: vec(rho)[i + n*j] = rho[i, j], for which
vec(A rho B) = (B^T kron A) vec(rho).
"""
import numpy as np
import scipy.sparse as sp


def dag(m):
    return m.conj().T


def effective_hamiltonian(H, c_ops):
    """H_eff = H - (i/2) sum_k C_k^dag C_k  (Sec. 3.3)."""
    Heff = sp.csr_matrix(H, dtype=np.complex128).copy()
    for C in c_ops:
        Heff = Heff - 0.5j * (dag(C) @ C)
    Heff = sp.csr_matrix(Heff)
    Heff.eliminate_zeros()
    Heff.sort_indices()
    return Heff


def liouvillian(H, c_ops):
    """The Liouvillian superoperator as an n^2 x n^2 CSR matrix acting on the
    column-stacked vec(rho):
        -i (I kron H - H^T kron I)
        + sum_k [ conj(C_k) kron C_k - 1/2 I kron C_k^dag C_k - 1/2 (C_k^dag C_k)^T kron I ].
    """
    n = H.shape[0]
    I = sp.identity(n, dtype=np.complex128, format="csr")
    H = sp.csr_matrix(H, dtype=np.complex128)
    L = -1j * (sp.kron(I, H) - sp.kron(H.T, I))
    for C in c_ops:
        C = sp.csr_matrix(C, dtype=np.complex128)
        CdC = dag(C) @ C
        L = L + sp.kron(C.conj(), C) - 0.5 * sp.kron(I, CdC) - 0.5 * sp.kron(CdC.T, I)
    L = sp.csr_matrix(L)
    L.sum_duplicates()
    L.eliminate_zeros()
    L.sort_indices()
    return L


def lindblad_rhs(H, c_ops, rho):
    """The right-hand side written as plain matrix products on a dense rho:
    -i (H rho - rho H) + sum_k (C rho C^dag - 1/2 C^dag C rho - 1/2 rho C^dag C)."""
    rho = np.asarray(rho)
    out = -1j * (H @ rho - (rho @ H))
    for C in c_ops:
        CdC = dag(C) @ C
        out = out + C @ (rho @ dag(C)) - 0.5 * (CdC @ rho) - 0.5 * (rho @ CdC)
    return np.asarray(out)


def vec(rho):
    """Column stacking."""
    return np.asarray(rho).reshape(-1, order="F")


def unvec(v, n):
    return np.asarray(v).reshape((n, n), order="F")


def expect_dm(O, rho):
    """Tr(O rho) (Sec. 3.1, sol.expect)."""
    return complex(np.trace(np.asarray(O @ rho)))


def expect_ket(O, psi):
    """<psi|O|psi> / <psi|psi> (normalised trajectory expectation)."""
    psi = np.asarray(psi)
    return complex(np.vdot(psi, O @ psi) / np.vdot(psi, psi))
