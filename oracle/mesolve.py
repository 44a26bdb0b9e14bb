"""mesolve: the Lindblad master equation integrated in time with
expectation values Tr(O_k rho(t)) at each time of tlist (Sec. 3.2; the GPU
example of Sec. 4 runs the same call)."""
import numpy as np

from .integrate import TABLEAUS_BY_NAME, integrate
from .lindblad import liouvillian, lindblad_rhs, unvec, vec


def initial_density_matrix(state):
    """rho0 = |psi0><psi0| for a ket (ket2dm), or the matrix itself."""
    state = np.asarray(state, dtype=np.complex128)
    if state.ndim == 1:
        return np.outer(state, state.conj())
    return state


def mesolve(H, c_ops, e_ops, state0, tlist, method="tsit5", rtol=1e-8, atol=1e-10,
            rhs="liouvillian", fixed_dt=None, dt0=0.0, save_states=False,
            max_steps=10_000_000):
    """Returns dict(expect[k, t] complex, states[t] (n x n) or None, stats).

    rhs = "liouvillian": k = L vec(rho) with the CSR superoperator;
    rhs = "product":     k = -i[H, rho] + sum D[C] rho by dense matrix products.
    Both are the same mathematical map (tested against each other)."""
    tab = TABLEAUS_BY_NAME[method]
    rho0 = initial_density_matrix(state0)
    n = rho0.shape[0]
    tlist = np.asarray(tlist, dtype=np.float64)
    if rhs == "liouvillian":
        L = liouvillian(H, c_ops)

        def f(t, y):
            return L @ y
    else:
        def f(t, y):
            return vec(lindblad_rhs(H, c_ops, unvec(y, n)))

    n_e = len(e_ops)
    expect = np.zeros((n_e, len(tlist)), dtype=np.complex128)
    states = np.zeros((len(tlist), n, n), dtype=np.complex128) if save_states else None
    e_dense = [np.asarray(O.todense()) if hasattr(O, "todense") else np.asarray(O) for O in e_ops]

    def on_save(idx, t, y):
        rho = unvec(y, n)
        for k, O in enumerate(e_dense):
            expect[k, idx] = np.trace(O @ rho)
        if states is not None:
            states[idx] = rho

    st = integrate(f, vec(rho0), tlist, tab, rtol, atol, on_save, dt0=dt0,
                   fixed_dt=fixed_dt, max_steps=max_steps)
    return dict(expect=expect, states=states, stats=st.as_dict())
