"""ctypes binding of the C ABI declared in include/qtl.h.

Argument marshalling only: every step of the solve runs in the library's
CUDA kernels.  The names mirror the C entry points without the `qtl_` prefix
(system_create, system_free, mesolve, mesolve_async, mcsolve, mcsolve_async,
opts_default, strerror, launch_count).  There is no CPU fallback: if the
library is missing or cannot be loaded, `load()` raises.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libqtl.so")

QTL_OK, QTL_EINVAL, QTL_ENOMEM, QTL_ESTEP, QTL_ECUDA, QTL_ECANCEL, QTL_EBUSY, QTL_ETOOBIG = range(8)
METHODS = {"dp5": 0, "tsit5": 1}
PRECISIONS = {"fp64": 0, "mixed": 1}
ENGINES = {"auto": 0, "cluster": 1, "grid": 2}


class QtlError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__(f"{what}: {strerror(status)} (status {status})"
                         + (f" [{last_cuda_error()}]" if status == QTL_ECUDA else ""))


class Op(C.Structure):
    _fields_ = [("n", C.c_int32), ("is_csr", C.c_int32), ("nnz", C.c_int64),
                ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p), ("vals", C.c_void_p)]


class Opts(C.Structure):
    _fields_ = [("method", C.c_int32), ("precision", C.c_int32), ("rtol", C.c_double),
                ("atol", C.c_double), ("dt0", C.c_double), ("dt_min", C.c_double),
                ("max_steps", C.c_int64), ("fixed_step", C.c_int32), ("cluster_size", C.c_int32),
                ("dt_fixed", C.c_double), ("cuda_stream", C.c_void_p), ("engine", C.c_int32),
                ("shadow_fp64", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("steps_acc", C.c_int64), ("steps_rej", C.c_int64), ("rhs_evals", C.c_int64),
                ("jumps", C.c_int64), ("err_vs_fp64", C.c_double)]

    def as_dict(self):
        d = {k: int(getattr(self, k)) for k, _ in self._fields_[:4]}
        d["err_vs_fp64"] = float(self.err_vs_fp64)
        return d


class Request(C.Structure):
    _fields_ = [("kind", C.c_int32), ("sys", C.c_void_p), ("state0", C.c_void_p), ("is_ket", C.c_int32),
                ("tlist", C.c_void_p), ("nt", C.c_int32), ("ntraj", C.c_int32), ("seed", C.c_uint64),
                ("opts", Opts)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("pad", C.c_int32), ("stats", Stats), ("t_submit", C.c_double),
                ("t_start", C.c_double), ("t_end", C.c_double)]


class SsOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("restart", C.c_int32), ("max_iter", C.c_int32),
                ("cuda_stream", C.c_void_p), ("precision", C.c_int32), ("pad", C.c_int32)]


class SsStats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("pad", C.c_int32), ("residual", C.c_double),
                ("cond_v", C.c_double), ("gmres_residual", C.c_double)]

    def as_dict(self):
        return dict(iterations=int(self.iterations), residual=float(self.residual),
                    cond_v=float(self.cond_v), gmres_residual=float(self.gmres_residual))


class C128(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double)]


DSF_BUILD = C.CFUNCTYPE(C.c_int, C.POINTER(C128), C.c_int32, C.c_void_p, C.POINTER(C.c_void_p))


class DeviceInfo(C.Structure):
    _fields_ = [("status", C.c_int32), ("pad", C.c_int32), ("steps_acc", C.c_int64),
                ("steps_rej", C.c_int64), ("rhs_evals", C.c_int64), ("jumps", C.c_int64)]


DEVICE_INFO_BYTES = C.sizeof(DeviceInfo)
_lib = None


def load():
    """Loads libqtl.so (built in-tree by build.py); raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libqtl.so not built ({LIB_PATH}); run paper_2504_21440_gb300/build.py")
    lib = C.CDLL(LIB_PATH)
    P = C.c_void_p
    lib.qtl_opts_default.argtypes = [C.POINTER(Opts)]
    lib.qtl_opts_default.restype = None
    lib.qtl_system_create.argtypes = [C.POINTER(Op), C.POINTER(Op), C.c_int32, C.POINTER(Op),
                                      C.c_int32, C.POINTER(P)]
    lib.qtl_system_create.restype = C.c_int
    lib.qtl_system_free.argtypes = [P]
    lib.qtl_system_free.restype = None
    lib.qtl_system_dim.argtypes = [P]
    lib.qtl_system_dim.restype = C.c_int32
    lib.qtl_system_liouvillian_nnz.argtypes = [P]
    lib.qtl_system_liouvillian_nnz.restype = C.c_int64
    lib.qtl_system_nnz.argtypes = [P, C.c_int32]
    lib.qtl_system_nnz.restype = C.c_int64
    lib.qtl_mesolve.argtypes = [P, P, C.c_int32, P, C.c_int32, C.POINTER(Opts), P, P,
                                C.POINTER(Stats)]
    lib.qtl_mesolve.restype = C.c_int
    lib.qtl_mesolve_async.argtypes = [P, P, C.c_int32, P, C.c_int32, C.POINTER(Opts), P, P, P]
    lib.qtl_mesolve_async.restype = C.c_int
    lib.qtl_mcsolve.argtypes = [P, P, P, C.c_int32, C.c_int32, C.c_uint64, C.c_int64,
                                C.POINTER(Opts), P, P, C.POINTER(Stats)]
    lib.qtl_mcsolve.restype = C.c_int
    lib.qtl_mcsolve_async.argtypes = [P, P, P, C.c_int32, C.c_int32, C.c_uint64, C.c_int64,
                                      C.POINTER(Opts), P, P, P]
    lib.qtl_mcsolve_async.restype = C.c_int
    lib.qtl_mesolve_batch.argtypes = [P, C.c_int32, P, P, P, C.c_int32, C.POINTER(Opts), P,
                                      C.POINTER(Stats)]
    lib.qtl_mesolve_batch.restype = C.c_int
    lib.qtl_mesolve_batch_async.argtypes = [P, C.c_int32, P, P, P, C.c_int32, C.POINTER(Opts), P, P]
    lib.qtl_mesolve_batch_async.restype = C.c_int
    lib.qtl_system_add_td.argtypes = [P, C.POINTER(Op), C.POINTER(Coef)]
    lib.qtl_system_add_td.restype = C.c_int
    lib.qtl_sesolve.argtypes = [P, P, P, C.c_int32, C.POINTER(Opts), P, C.POINTER(Stats)]
    lib.qtl_sesolve.restype = C.c_int
    lib.qtl_ssesolve.argtypes = [P, P, P, C.c_int32, C.c_int32, C.c_uint64, C.POINTER(Opts), P, P,
                                 C.POINTER(Stats), P, P]
    lib.qtl_ssesolve.restype = C.c_int
    lib.qtl_smesolve.argtypes = [P, C.c_int32, P, P, C.c_int32, C.c_int32, C.c_uint64, C.POINTER(Opts), P, P,
                                 C.POINTER(Stats), P, P]
    lib.qtl_smesolve.restype = C.c_int
    lib.qtl_batch_create.argtypes = [P, C.c_int32, P, P, P, C.c_int32, C.POINTER(Opts), P, P, C.c_int32,
                                     C.POINTER(P)]
    lib.qtl_batch_create.restype = C.c_int
    lib.qtl_batch_launch.argtypes = [P, P]
    lib.qtl_batch_launch.restype = C.c_int
    lib.qtl_batch_groups.argtypes = [P]
    lib.qtl_batch_groups.restype = C.c_int32
    lib.qtl_batch_group_info.argtypes = [P, C.c_int32, P, P, P, P, P]
    lib.qtl_batch_group_info.restype = C.c_int
    lib.qtl_batch_group_of.argtypes = [P, C.c_int32]
    lib.qtl_batch_group_of.restype = C.c_int32
    lib.qtl_batch_free.argtypes = [P]
    lib.qtl_batch_free.restype = None
    lib.qtl_mcsolve_noalloc.argtypes = [C.c_int32, P, P, P, C.c_int64, C.c_int32, P, P, P,
                                        C.c_int32, P, P, P, P, P, C.c_int32, C.c_int32,
                                        C.c_uint64, C.c_int64, C.POINTER(Opts), P, P]
    lib.qtl_mcsolve_noalloc.restype = C.c_int
    lib.qtl_ss_opts_default.argtypes = [C.POINTER(SsOpts)]
    lib.qtl_ss_opts_default.restype = None
    lib.qtl_steadystate.argtypes = [P, C.POINTER(SsOpts), P, C.POINTER(SsStats)]
    lib.qtl_steadystate.restype = C.c_int
    lib.qtl_steadystate_fourier.argtypes = [P, C.POINTER(Op), C.c_double, C.c_double, C.c_int32,
                                            C.POINTER(SsOpts), P, C.POINTER(SsStats)]
    lib.qtl_steadystate_fourier.restype = C.c_int
    lib.qtl_zgemm_async.argtypes = [C.c_int32, P, C.c_int32, P, C.c_int32, P, C.c_int32, P, P]
    lib.qtl_zgemm_async.restype = C.c_int
    lib.qtl_dsf_mesolve.argtypes = [DSF_BUILD, P, C.c_int32, C.POINTER(Op), P, P, C.c_int32, P, C.c_int32,
                                    C.c_double, C.POINTER(Opts), C.c_int32, P, P, C.POINTER(C.c_int32),
                                    C.POINTER(Stats)]
    lib.qtl_dsf_mesolve.restype = C.c_int
    lib.qtl_dsf_mcsolve.argtypes = [DSF_BUILD, P, C.c_int32, C.POINTER(Op), P, P, P, C.c_int32, C.c_double,
                                    C.c_int32, C.c_uint64, C.POINTER(Opts), C.c_int32, P, P,
                                    C.POINTER(C.c_int64), C.POINTER(Stats)]
    lib.qtl_dsf_mcsolve.restype = C.c_int
    lib.qtl_server_create.argtypes = [C.c_size_t, C.c_int32, C.POINTER(P)]
    lib.qtl_server_create.restype = C.c_int
    lib.qtl_server_submit.argtypes = [P, C.POINTER(Request), P, C.POINTER(C.c_uint64)]
    lib.qtl_server_submit.restype = C.c_int
    lib.qtl_server_poll.argtypes = [P, C.c_uint64, C.POINTER(Result)]
    lib.qtl_server_poll.restype = C.c_int
    lib.qtl_server_wait.argtypes = [P, C.c_uint64, C.POINTER(Result)]
    lib.qtl_server_wait.restype = C.c_int
    lib.qtl_server_cancel.argtypes = [P, C.c_uint64]
    lib.qtl_server_cancel.restype = C.c_int
    lib.qtl_server_usage.argtypes = [P, C.POINTER(C.c_size_t), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    lib.qtl_server_usage.restype = C.c_int
    lib.qtl_server_free.argtypes = [P]
    lib.qtl_server_free.restype = None
    lib.qtl_strerror.argtypes = [C.c_int]
    lib.qtl_strerror.restype = C.c_char_p
    lib.qtl_last_cuda_error.argtypes = []
    lib.qtl_last_cuda_error.restype = C.c_char_p
    lib.qtl_launch_count.argtypes = []
    lib.qtl_launch_count.restype = C.c_int64
    _lib = lib
    return lib


def strerror(status):
    return load().qtl_strerror(int(status)).decode()


def last_cuda_error():
    return load().qtl_last_cuda_error().decode()


def launch_count():
    return int(load().qtl_launch_count())


def opts_default():
    o = Opts()
    load().qtl_opts_default(C.byref(o))
    return o


def make_opts(method="tsit5", precision="fp64", rtol=1e-8, atol=1e-10, dt0=0.0, dt_min=0.0,
              max_steps=10_000_000, fixed_dt=None, cluster_size=0, stream=None, engine="auto",
              shadow_fp64=False):
    o = opts_default()
    o.method = METHODS[method]
    o.precision = PRECISIONS[precision]
    o.rtol, o.atol, o.dt0, o.dt_min = float(rtol), float(atol), float(dt0), float(dt_min)
    o.max_steps = int(max_steps)
    o.fixed_step = 1 if fixed_dt is not None else 0
    o.dt_fixed = float(fixed_dt) if fixed_dt is not None else 0.0
    o.cluster_size = int(cluster_size)
    o.cuda_stream = stream
    o.engine = ENGINES[engine]
    o.shadow_fp64 = 1 if shadow_fp64 else 0
    return o


def _check(status, what):
    if status != QTL_OK:
        raise QtlError(status, what)


class Coef(C.Structure):
    """qtl_coef: f(t) = (amp_re + i amp_im) env(t) g(omega t + phi), g = cos
    (kind 0) or exp(i .) (kind 1), env a Gaussian around t0 when sigma > 0."""
    _fields_ = [("kind", C.c_int32), ("amp_re", C.c_double), ("amp_im", C.c_double),
                ("omega", C.c_double), ("phi", C.c_double), ("t0", C.c_double), ("sigma", C.c_double)]


def coef(kind="cos", amp=1.0, omega=0.0, phi=0.0, t0=0.0, sigma=0.0):
    a = complex(amp)
    return Coef({"cos": 0, "exp": 1}[kind], a.real, a.imag, float(omega), float(phi), float(t0), float(sigma))


class _OpHolder:
    """Keeps the arrays behind a qtl_op alive for the duration of a call."""

    def __init__(self, m):
        if hasattr(m, "tocsr"):
            m = m.tocsr()
            self.rp = np.ascontiguousarray(m.indptr, dtype=np.int32)
            self.ci = np.ascontiguousarray(m.indices, dtype=np.int32)
            self.v = np.ascontiguousarray(m.data, dtype=np.complex128)
            self.op = Op(m.shape[0], 1, len(self.v), self.rp.ctypes.data, self.ci.ctypes.data,
                         self.v.ctypes.data)
        else:
            a = np.asarray(m, dtype=np.complex128)
            self.v = np.asfortranarray(a)
            self.op = Op(a.shape[0], 0, 0, None, None, self.v.ctypes.data)


def _ptr(x):
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return C.c_void_p(x.data_ptr())
    return C.c_void_p(x.ctypes.data)


def system_create(H, c_ops=(), e_ops=()):
    """qtl_system_create: H, c_ops, e_ops as scipy sparse or dense arrays."""
    lib = load()
    hold = [_OpHolder(H)] + [_OpHolder(c) for c in c_ops] + [_OpHolder(e) for e in e_ops]
    nc, ne = len(c_ops), len(e_ops)
    ca = (Op * max(nc, 1))(*[h.op for h in hold[1:1 + nc]])
    ea = (Op * max(ne, 1))(*[h.op for h in hold[1 + nc:]])
    out = C.c_void_p()
    _check(lib.qtl_system_create(C.byref(hold[0].op), ca, nc, ea, ne, C.byref(out)),
           "qtl_system_create")
    return out


def system_add_td(sys, Hk, f):
    """qtl_system_add_td: adds f(t) Hk (f a Coef, or a dict of coef() arguments)."""
    h = _OpHolder(Hk)
    c = f if isinstance(f, Coef) else coef(**f)
    _check(load().qtl_system_add_td(sys, C.byref(h.op), C.byref(c)), "qtl_system_add_td")


def sesolve(sys, n_e, psi0, tlist, opts):
    """qtl_sesolve with host arrays.  Returns dict(expect[n_e, nt], stats)."""
    lib = load()
    p0 = np.ascontiguousarray(psi0, dtype=np.complex128)
    tl = np.ascontiguousarray(tlist, dtype=np.float64)
    ex = np.zeros((max(n_e, 1), len(tl)), dtype=np.complex128)
    st = Stats()
    _check(lib.qtl_sesolve(sys, _ptr(p0), _ptr(tl), len(tl), C.byref(opts), _ptr(ex), C.byref(st)),
           "qtl_sesolve")
    return dict(expect=ex[:n_e], stats=st.as_dict())


def _traj_buffers(n_e, n_sc, nt, ntraj, keep):
    if not keep:
        return None, None
    return (np.zeros((max(n_e, 1), nt, ntraj), dtype=np.complex128),
            np.zeros((max(n_sc, 1), nt, ntraj), dtype=np.float64))


def _with_traj(out, n_e, n_sc, te, tm):
    if te is not None:
        out["traj_expect"] = np.moveaxis(te[:n_e], 2, 0)        # [traj, e, t]
        out["traj_measurement"] = np.moveaxis(tm[:n_sc], 2, 0)   # [traj, n, t]
    return out


def ssesolve(sys, n_e, n_sc, psi0, tlist, ntraj, seed, opts, keep_trajectories=False):
    """qtl_ssesolve with host arrays.  Returns dict(expect[n_e, nt],
    measurement[n_sc, nt], stats) and, with keep_trajectories, the
    per-trajectory traj_expect[traj, e, t] and traj_measurement[traj, n, t]."""
    lib = load()
    p0 = np.ascontiguousarray(psi0, dtype=np.complex128)
    tl = np.ascontiguousarray(tlist, dtype=np.float64)
    ex = np.zeros((max(n_e, 1), len(tl)), dtype=np.complex128)
    ms = np.zeros((max(n_sc, 1), len(tl)), dtype=np.float64)
    te, tm = _traj_buffers(n_e, n_sc, len(tl), int(ntraj), keep_trajectories)
    st = Stats()
    _check(lib.qtl_ssesolve(sys, _ptr(p0), _ptr(tl), len(tl), int(ntraj), C.c_uint64(int(seed) & (2**64 - 1)),
                            C.byref(opts), _ptr(ex), _ptr(ms), C.byref(st), _ptr(te), _ptr(tm)), "qtl_ssesolve")
    return _with_traj(dict(expect=ex[:n_e], measurement=ms[:n_sc], stats=st.as_dict()), n_e, n_sc, te, tm)


def smesolve(sys, n_e, n_sc, psi0, tlist, ntraj, seed, opts, keep_trajectories=False):
    """qtl_smesolve with host arrays (the system's last n_sc collapse operators
    are measured).  Returns dict(expect[n_e, nt], measurement[n_sc, nt], stats)
    and, with keep_trajectories, the per-trajectory values as ssesolve."""
    lib = load()
    p0 = np.ascontiguousarray(psi0, dtype=np.complex128)
    tl = np.ascontiguousarray(tlist, dtype=np.float64)
    ex = np.zeros((max(n_e, 1), len(tl)), dtype=np.complex128)
    ms = np.zeros((max(n_sc, 1), len(tl)), dtype=np.float64)
    te, tm = _traj_buffers(n_e, n_sc, len(tl), int(ntraj), keep_trajectories)
    st = Stats()
    _check(lib.qtl_smesolve(sys, int(n_sc), _ptr(p0), _ptr(tl), len(tl), int(ntraj),
                            C.c_uint64(int(seed) & (2**64 - 1)), C.byref(opts), _ptr(ex), _ptr(ms), C.byref(st),
                            _ptr(te), _ptr(tm)),
           "qtl_smesolve")
    return _with_traj(dict(expect=ex[:n_e], measurement=ms[:n_sc], stats=st.as_dict()), n_e, n_sc, te, tm)


def system_free(sys):
    load().qtl_system_free(sys)


def system_dim(sys):
    return int(load().qtl_system_dim(sys))


def system_liouvillian_nnz(sys):
    return int(load().qtl_system_liouvillian_nnz(sys))


def system_nnz(sys, which):
    """qtl_system_nnz: stored entries of H (0), A = -i H_eff (1), the
    Liouvillian (2); of A (3) and the Liouvillian (4) those with a zero real or
    imaginary part."""
    return int(load().qtl_system_nnz(sys, int(which)))


def mesolve(sys, n_e, state0, tlist, opts, save_states=False):
    """qtl_mesolve with host arrays.  Returns dict(expect[n_e, nt], states, stats)."""
    lib = load()
    s0 = np.ascontiguousarray(state0, dtype=np.complex128)
    is_ket = 1 if s0.ndim == 1 else 0
    if not is_ket:
        s0 = np.ascontiguousarray(s0.reshape(-1, order="F"))
    tl = np.ascontiguousarray(tlist, dtype=np.float64)
    nt = len(tl)
    n = system_dim(sys)
    ex = np.zeros((max(n_e, 1), nt), dtype=np.complex128)
    states = np.zeros((nt, n * n), dtype=np.complex128) if save_states else None
    st = Stats()
    status = lib.qtl_mesolve(sys, _ptr(s0), is_ket, _ptr(tl), nt, C.byref(opts), _ptr(ex),
                             _ptr(states), C.byref(st))
    _check(status, "qtl_mesolve")
    out = dict(expect=ex[:n_e], stats=st.as_dict(), states=None)
    if states is not None:
        out["states"] = states.reshape(nt, n, n).transpose(0, 2, 1).copy()
    return out


def mesolve_async(sys, state0_dev, is_ket, tlist_dev, opts, expect_dev, states_dev, info_dev):
    """qtl_mesolve_async with device tensors (torch) on opts.cuda_stream."""
    _check(load().qtl_mesolve_async(sys, _ptr(state0_dev), int(is_ket), _ptr(tlist_dev),
                                    int(tlist_dev.numel()), C.byref(opts), _ptr(expect_dev),
                                    _ptr(states_dev), _ptr(info_dev)), "qtl_mesolve_async")


def mcsolve(sys, n_e, psi0, tlist, ntraj, seed, opts, traj_offset=0, keep_trajectories=False):
    """qtl_mcsolve with host arrays.  Returns dict(expect, traj_expect?, stats)."""
    lib = load()
    p0 = np.ascontiguousarray(psi0, dtype=np.complex128)
    tl = np.ascontiguousarray(tlist, dtype=np.float64)
    nt = len(tl)
    ex = np.zeros((max(n_e, 1), nt), dtype=np.complex128)
    tex = np.zeros((max(n_e, 1), nt, ntraj), dtype=np.complex128) if keep_trajectories else None
    st = Stats()
    status = lib.qtl_mcsolve(sys, _ptr(p0), _ptr(tl), nt, int(ntraj), C.c_uint64(int(seed) & (2**64 - 1)),
                             int(traj_offset), C.byref(opts), _ptr(ex), _ptr(tex), C.byref(st))
    _check(status, "qtl_mcsolve")
    out = dict(expect=ex[:n_e], stats=st.as_dict())
    if tex is not None:
        out["traj_expect"] = np.moveaxis(tex[:n_e], 2, 0)   # [traj, e, t]
    return out


def mcsolve_async(sys, psi0_dev, tlist_dev, ntraj, seed, opts, expect_dev, traj_expect_dev,
                  info_dev, traj_offset=0):
    _check(load().qtl_mcsolve_async(sys, _ptr(psi0_dev), _ptr(tlist_dev), int(tlist_dev.numel()),
                                    int(ntraj), C.c_uint64(int(seed) & (2**64 - 1)),
                                    int(traj_offset), C.byref(opts), _ptr(expect_dev),
                                    _ptr(traj_expect_dev), _ptr(info_dev)), "qtl_mcsolve_async")


def batch_cluster_size(n):
    """Cluster size the batch entry points give a system of dimension n."""
    c = 1
    while c < 16 and c * 1024 < n * n:
        c *= 2
    return c


def mesolve_batch(handles, n_es, states0, tlist, opts):
    """qtl_mesolve_batch with host arrays: one expectation array [n_e, nt] and
    one stats dict per system."""
    lib = load()
    nb = len(handles)
    tl = np.ascontiguousarray(tlist, dtype=np.float64)
    nt = len(tl)
    st0 = [np.ascontiguousarray(x, dtype=np.complex128) for x in states0]
    st0 = [x if x.ndim == 1 else np.ascontiguousarray(x.reshape(-1, order="F")) for x in st0]
    is_ket = (C.c_int32 * nb)(*[1 if np.ndim(x) == 1 and len(x) == system_dim(h) else 0
                                 for x, h in zip(st0, handles)])
    outs = [np.zeros((max(ne, 1), nt), dtype=np.complex128) for ne in n_es]
    harr = (C.c_void_p * nb)(*[h.value if hasattr(h, "value") else h for h in handles])
    sarr = (C.c_void_p * nb)(*[x.ctypes.data for x in st0])
    earr = (C.c_void_p * nb)(*[o.ctypes.data for o in outs])
    stats = (Stats * nb)()
    _check(lib.qtl_mesolve_batch(harr, nb, sarr, is_ket, _ptr(tl), nt, C.byref(opts), earr, stats),
           "qtl_mesolve_batch")
    return [dict(expect=o[:ne], stats=stats[b].as_dict()) for b, (o, ne) in enumerate(zip(outs, n_es))]


def mesolve_batch_async(handles, states_dev, is_ket, tlist_dev, opts, expects_dev, info_dev):
    """qtl_mesolve_batch_async: device tensors, enqueued on opts.cuda_stream."""
    nb = len(handles)
    harr = (C.c_void_p * nb)(*[h.value if hasattr(h, "value") else h for h in handles])
    sarr = (C.c_void_p * nb)(*[x.data_ptr() for x in states_dev])
    karr = (C.c_int32 * nb)(*[int(k) for k in is_ket])
    earr = (C.c_void_p * nb)(*[x.data_ptr() for x in expects_dev])
    _check(load().qtl_mesolve_batch_async(harr, nb, sarr, karr, _ptr(tlist_dev), int(tlist_dev.numel()),
                                          C.byref(opts), earr, _ptr(info_dev)), "qtl_mesolve_batch_async")
    return (harr, sarr, karr, earr)


class Batch:
    """qtl_batch_*: a batch plan over device tensors (kept alive here),
    optionally autotuned, replayed from a captured CUDA graph by launch()."""

    def __init__(self, handles, states_dev, is_ket, tlist_dev, opts, expects_dev, info_dev, autotune=False):
        nb = len(handles)
        self._keep = (list(states_dev), tlist_dev, list(expects_dev), info_dev)
        harr = (C.c_void_p * nb)(*[h.value if hasattr(h, "value") else h for h in handles])
        sarr = (C.c_void_p * nb)(*[x.data_ptr() for x in states_dev])
        karr = (C.c_int32 * nb)(*[int(k) for k in is_ket])
        earr = (C.c_void_p * nb)(*[x.data_ptr() for x in expects_dev])
        self.handle = C.c_void_p()
        _check(load().qtl_batch_create(harr, nb, sarr, karr, _ptr(tlist_dev), int(tlist_dev.numel()),
                                       C.byref(opts), earr, _ptr(info_dev), 1 if autotune else 0,
                                       C.byref(self.handle)), "qtl_batch_create")

    def launch(self, stream):
        _check(load().qtl_batch_launch(self.handle, C.c_void_p(int(stream))), "qtl_batch_launch")

    def groups(self):
        """[(cluster_size, nsolves, [(candidate cluster size, probe ms), ...]), ...]"""
        lib = load()
        out = []
        for k in range(int(lib.qtl_batch_groups(self.handle))):
            cs, ns, nc = C.c_int32(), C.c_int32(), C.c_int32()
            cc = (C.c_int32 * 8)()
            cm = (C.c_double * 8)()
            _check(lib.qtl_batch_group_info(self.handle, k, C.byref(cs), C.byref(ns), C.byref(nc), cc, cm),
                   "qtl_batch_group_info")
            out.append((cs.value, ns.value, [(cc[i], cm[i]) for i in range(nc.value)]))
        return out

    def group_of(self, b):
        return int(load().qtl_batch_group_of(self.handle, int(b)))

    def free(self):
        if self.handle:
            load().qtl_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Server:
    """qtl_server_*: a request queue admitted by HBM budget, requests running
    concurrently on the server's streams.  submit() keeps the request's host
    buffers alive until its result has been taken."""

    def __init__(self, hbm_budget_bytes=0, max_inflight=8):
        self.handle = C.c_void_p()
        _check(load().qtl_server_create(int(hbm_budget_bytes), int(max_inflight), C.byref(self.handle)),
               "qtl_server_create")
        self._keep = {}

    def submit(self, kind, system, state0, tlist, opts, ntraj=0, seed=0):
        st = np.ascontiguousarray(state0, dtype=np.complex128)
        is_ket = 1 if st.ndim == 1 and len(st) == system.n else 0
        if st.ndim == 2:
            st = np.ascontiguousarray(st.reshape(-1, order="F"))
        tl = np.ascontiguousarray(tlist, dtype=np.float64)
        ex = np.zeros((max(system.n_e, 1), len(tl)), dtype=np.complex128)
        req = Request(0 if kind == "mesolve" else 1, system.handle, st.ctypes.data, is_ket, tl.ctypes.data,
                      len(tl), int(ntraj), C.c_uint64(int(seed) & (2**64 - 1)), opts)
        t = C.c_uint64()
        _check(load().qtl_server_submit(self.handle, C.byref(req), ex.ctypes.data, C.byref(t)),
               "qtl_server_submit")
        self._keep[t.value] = (st, tl, ex, system.n_e)
        return t.value

    def _take(self, ticket, res):
        st, tl, ex, ne = self._keep.pop(ticket)
        return dict(status=int(res.status), expect=ex[:ne], stats=res.stats.as_dict(),
                    t_submit=res.t_submit, t_start=res.t_start, t_end=res.t_end)

    def poll(self, ticket):
        res = Result()
        s = load().qtl_server_poll(self.handle, C.c_uint64(ticket), C.byref(res))
        if s == QTL_EBUSY:
            return None
        _check(s, "qtl_server_poll")
        return self._take(ticket, res)

    def wait(self, ticket):
        res = Result()
        _check(load().qtl_server_wait(self.handle, C.c_uint64(ticket), C.byref(res)), "qtl_server_wait")
        return self._take(ticket, res)

    def cancel(self, ticket):
        return load().qtl_server_cancel(self.handle, C.c_uint64(ticket))

    def usage(self):
        b, q, r = C.c_size_t(), C.c_int32(), C.c_int32()
        _check(load().qtl_server_usage(self.handle, C.byref(b), C.byref(q), C.byref(r)), "qtl_server_usage")
        return b.value, q.value, r.value

    def free(self):
        if self.handle:
            load().qtl_server_free(self.handle)
            self.handle = None


NOALLOC_SCRATCH_BYTES = 32 << 20


def mcsolve_noalloc(n, a_csr, c_csr, n_c, o_csr, n_e, psi0_dev, tlist_dev, ntraj, seed, opts,
                    expect_dev, info_dev, traj_offset=0):
    """qtl_mcsolve_noalloc: every operator is a tuple (row_ptr, col_idx, vals) of
    device tensors (int32, int32, complex128); A = -i H_eff is n x n, the
    collapse operators and observables are stacked row-wise.  Allocates
    nothing on the device; enqueued on opts.cuda_stream."""
    def parts(csr):
        return (None, None, None) if csr is None else tuple(_ptr(x) for x in csr)
    arp, aci, av = parts(a_csr)
    crp, cci, cv = parts(c_csr)
    orp, oci, ov = parts(o_csr)
    _check(load().qtl_mcsolve_noalloc(int(n), arp, aci, av, int(a_csr[2].numel()), int(n_c), crp,
                                      cci, cv, int(n_e), orp, oci, ov, _ptr(psi0_dev),
                                      _ptr(tlist_dev), int(tlist_dev.numel()), int(ntraj),
                                      C.c_uint64(int(seed) & (2**64 - 1)), int(traj_offset),
                                      C.byref(opts), _ptr(expect_dev), _ptr(info_dev)),
           "qtl_mcsolve_noalloc")


def ss_opts(tol=1e-12, restart=60, max_iter=20000, stream=None, precision="fp64"):
    o = SsOpts()
    load().qtl_ss_opts_default(C.byref(o))
    o.tol, o.restart, o.max_iter, o.cuda_stream = float(tol), int(restart), int(max_iter), stream
    o.precision = PRECISIONS[precision]
    return o


def steadystate(sys, opts):
    """qtl_steadystate: returns dict(rho (n x n), stats)."""
    n = system_dim(sys)
    out = np.zeros(n * n, dtype=np.complex128)
    st = SsStats()
    _check(load().qtl_steadystate(sys, C.byref(opts), _ptr(out), C.byref(st)), "qtl_steadystate")
    return dict(rho=out.reshape((n, n), order="F"), stats=st.as_dict())


def steadystate_fourier(sys, X, F, omega, nmax, opts):
    """qtl_steadystate_fourier: returns dict(rho = {k: rho_k}, stats)."""
    n = system_dim(sys)
    K = 2 * int(nmax) + 1
    out = np.zeros(K * n * n, dtype=np.complex128)
    st = SsStats()
    xo = _OpHolder(X)
    _check(load().qtl_steadystate_fourier(sys, C.byref(xo.op), float(F), float(omega), int(nmax),
                                          C.byref(opts), _ptr(out), C.byref(st)),
           "qtl_steadystate_fourier")
    rho = {a - int(nmax): out[a * n * n:(a + 1) * n * n].reshape((n, n), order="F") for a in range(K)}
    return dict(rho=rho, stats=st.as_dict())


def zgemm_async(A, B, C, op_a=0, op_b=0, precision="fp64", stream=None, err=None):
    """qtl_zgemm_async on torch complex128 device tensors (n x n; column-major
    storage, i.e. pass the transposes of row-major tensors): C = op(A) op(B).
    err: a device int32 tensor (precision "mixed")."""
    n = int(A.shape[0])
    _check(load().qtl_zgemm_async(n, _ptr(A), int(op_a), _ptr(B), int(op_b), _ptr(C), PRECISIONS[precision],
                                  stream, _ptr(err)), "qtl_zgemm_async")


def dsf_mesolve(H_fn, c_fn, e_fn, op_list, alpha0, state0, tlist, threshold, **kw):
    """qtl_dsf_mesolve.  H_fn(ops), c_fn(ops), e_fn(ops) build the Hamiltonian,
    collapse operators and observables from ops = [a_k + alpha_k I]; the
    library calls back whenever a coherence alpha_k changes.  op_list: the
    mode operators a_k on the full space.  Returns dict(expect[k, t],
    alpha[k, t], shifts, stats)."""
    import scipy.sparse as sp
    lib = load()
    mods = [sp.csr_matrix(a, dtype=np.complex128) for a in op_list]
    dim = mods[0].shape[0]
    eye = sp.identity(dim, dtype=np.complex128, format="csr")
    n_e = len(e_fn(mods))
    errors = []

    def build(alpha_p, n_modes, user, out):
        try:
            al = [complex(alpha_p[k].re, alpha_p[k].im) for k in range(n_modes)]
            ops = [a + x * eye for a, x in zip(mods, al)]
            out[0] = system_create(H_fn(ops), c_fn(ops), e_fn(ops)).value
            return QTL_OK
        except Exception as ex:   # reported after the call
            errors.append(ex)
            return QTL_EINVAL

    cb = DSF_BUILD(build)
    holders = [_OpHolder(a) for a in mods]
    ops_arr = (Op * len(mods))(*[h.op for h in holders])
    a0 = np.ascontiguousarray(np.asarray(alpha0, dtype=np.complex128))
    s0 = np.ascontiguousarray(state0, dtype=np.complex128)
    is_ket = 1 if s0.ndim == 1 else 0
    if not is_ket:
        s0 = np.ascontiguousarray(s0.reshape(-1, order="F"))
    tl = np.ascontiguousarray(tlist, dtype=np.float64)
    nt = len(tl)
    ex = np.zeros((max(n_e, 1), nt), dtype=np.complex128)
    al = np.zeros((len(mods), nt), dtype=np.complex128)
    shifts = C.c_int32(0)
    st = Stats()
    status = lib.qtl_dsf_mesolve(cb, None, len(mods), ops_arr, _ptr(a0), _ptr(s0), is_ket, _ptr(tl), nt,
                                 float(threshold), C.byref(make_opts(**kw)), n_e, _ptr(ex), _ptr(al),
                                 C.byref(shifts), C.byref(st))
    if errors:
        raise errors[0]
    _check(status, "qtl_dsf_mesolve")
    return dict(expect=ex[:n_e], alpha=al, shifts=int(shifts.value), stats=st.as_dict())


def dsf_mcsolve(H_fn, c_fn, e_fn, op_list, alpha0, psi0, tlist, threshold, ntraj, seed,
                keep_trajectories=False, **kw):
    """qtl_dsf_mcsolve: DSF on quantum trajectories, each in its own frame.
    H_fn, c_fn, e_fn and op_list as for dsf_mesolve (the library calls back
    for every trajectory whose coherence changes).  Returns dict(expect[k, t],
    traj_expect[j, k, t]?, shifts, stats)."""
    import scipy.sparse as sp
    lib = load()
    mods = [sp.csr_matrix(a, dtype=np.complex128) for a in op_list]
    dim = mods[0].shape[0]
    eye = sp.identity(dim, dtype=np.complex128, format="csr")
    n_e = len(e_fn(mods))
    errors = []

    def build(alpha_p, n_modes, user, out):
        try:
            al = [complex(alpha_p[k].re, alpha_p[k].im) for k in range(n_modes)]
            ops = [a + x * eye for a, x in zip(mods, al)]
            out[0] = system_create(H_fn(ops), c_fn(ops), e_fn(ops)).value
            return QTL_OK
        except Exception as ex:   # reported after the call
            errors.append(ex)
            return QTL_EINVAL

    cb = DSF_BUILD(build)
    holders = [_OpHolder(a) for a in mods]
    ops_arr = (Op * len(mods))(*[h.op for h in holders])
    a0 = np.ascontiguousarray(np.asarray(alpha0, dtype=np.complex128))
    p0 = np.ascontiguousarray(psi0, dtype=np.complex128)
    tl = np.ascontiguousarray(tlist, dtype=np.float64)
    nt = len(tl)
    ex = np.zeros((max(n_e, 1), nt), dtype=np.complex128)
    tex = np.zeros((int(ntraj), max(n_e, 1), nt), dtype=np.complex128) if keep_trajectories else None
    shifts = C.c_int64(0)
    st = Stats()
    status = lib.qtl_dsf_mcsolve(cb, None, len(mods), ops_arr, _ptr(a0), _ptr(p0), _ptr(tl), nt,
                                 float(threshold), int(ntraj), C.c_uint64(int(seed) & (2**64 - 1)),
                                 C.byref(make_opts(**kw)), n_e, _ptr(ex), _ptr(tex), C.byref(shifts),
                                 C.byref(st))
    if errors:
        raise errors[0]
    _check(status, "qtl_dsf_mcsolve")
    out = dict(expect=ex[:n_e], shifts=int(shifts.value), stats=st.as_dict())
    if keep_trajectories:
        out["traj_expect"] = tex[:, :n_e]
    return out


class System:
    """Owning wrapper: System(H, c_ops, e_ops) -> .mesolve(...) / .mcsolve(...)."""

    def __init__(self, H, c_ops=(), e_ops=(), td=()):
        self.handle = system_create(H, c_ops, e_ops)
        try:
            for Hk, f in td:
                system_add_td(self.handle, Hk, f)
        except Exception:
            system_free(self.handle)
            self.handle = None
            raise
        self.n = system_dim(self.handle)
        self.n_e = len(e_ops)
        self.n_c = len(c_ops)

    def mesolve(self, state0, tlist, save_states=False, **kw):
        return mesolve(self.handle, self.n_e, state0, tlist, make_opts(**kw), save_states)

    def ssesolve(self, psi0, tlist, ntraj, seed, keep_trajectories=False, **kw):
        """The collapse operators given at construction are the stochastic operators."""
        return ssesolve(self.handle, self.n_e, self.n_c, psi0, tlist, ntraj, seed, make_opts(**kw),
                        keep_trajectories)

    def smesolve(self, n_sc, psi0, tlist, ntraj, seed, keep_trajectories=False, **kw):
        """The last n_sc collapse operators given at construction are measured."""
        return smesolve(self.handle, self.n_e, n_sc, psi0, tlist, ntraj, seed, make_opts(**kw),
                        keep_trajectories)

    def sesolve(self, psi0, tlist, **kw):
        return sesolve(self.handle, self.n_e, psi0, tlist, make_opts(**kw))

    def steadystate(self, **kw):
        return steadystate(self.handle, ss_opts(**kw))

    def steadystate_fourier(self, X, F, omega, nmax, **kw):
        return steadystate_fourier(self.handle, X, F, omega, nmax, ss_opts(**kw))

    def mcsolve(self, psi0, tlist, ntraj, seed, traj_offset=0, keep_trajectories=False, **kw):
        return mcsolve(self.handle, self.n_e, psi0, tlist, ntraj, seed, make_opts(**kw),
                       traj_offset, keep_trajectories)

    def free(self):
        if self.handle:
            system_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
