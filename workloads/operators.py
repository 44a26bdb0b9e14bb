"""Elementary operators and states (the paper's Table of Qobj constructors).

Conventions, stated once and used everywhere:
  * two-level basis: index 0 = excited |e>, index 1 = ground |g>, so that
    sigmaz = diag(+1, -1) as printed in Sec. 2 (Pauli matrices) and
    sigmam = |g><e| lowers the excitation;
  * tensor(A, B) = kron(A, B): the first factor is the most significant index;
  * all matrices are scipy CSR, complex128, explicit zeros removed.
"""
import math

import numpy as np
import scipy.sparse as sp


def _csr(m):
    m = sp.csr_matrix(m, dtype=np.complex128)
    m.eliminate_zeros()
    m.sort_indices()
    return m


def dag(m):
    """Hermitian adjoint of a sparse matrix."""
    return _csr(m.conj().T)


def destroy(n):
    """Annihilation operator a|k> = sqrt(k)|k-1> on a Fock space cut at n."""
    k = np.arange(1, n)
    return _csr(sp.diags(np.sqrt(k).astype(np.complex128), offsets=1, shape=(n, n)))


def qeye(n):
    return _csr(sp.identity(n, dtype=np.complex128))


def sigmaz():
    return _csr(np.array([[1, 0], [0, -1]]))


def sigmax():
    return _csr(np.array([[0, 1], [1, 0]]))


def sigmay():
    return _csr(np.array([[0, -1j], [1j, 0]]))


def sigmam():
    """|g><e| with e = index 0, g = index 1."""
    return _csr(np.array([[0, 0], [1, 0]]))


def sigmap():
    """|e><g|, the adjoint of sigmam."""
    return _csr(np.array([[0, 1], [0, 0]]))


def tensor(*ops):
    out = ops[0]
    for o in ops[1:]:
        out = sp.kron(out, o, format="csr")
    return _csr(out)


def site_operator(op, site, n_sites, local_dim=2):
    """op acting on `site` (0-based, site 0 most significant) of a chain."""
    mats = [qeye(local_dim)] * n_sites
    mats = list(mats)
    mats[site] = op
    return tensor(*mats)


def fock(n, k):
    """Basis ket |k> of dimension n (dense complex128 vector)."""
    v = np.zeros(n, dtype=np.complex128)
    v[k] = 1.0
    return v


def coherent(n, alpha):
    """Truncated coherent state: c_k = exp(-|a|^2/2) a^k / sqrt(k!), k < n, then
    renormalised (App. B, coherent-state series)."""
    c = np.zeros(n, dtype=np.complex128)
    for k in range(n):
        c[k] = math.exp(-abs(alpha) ** 2 / 2) * alpha ** k / math.sqrt(math.factorial(k))
    return c / np.linalg.norm(c)
