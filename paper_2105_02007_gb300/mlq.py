"""Thin ctypes binding of libmlq (include/mlq.h): argument marshalling only.

Every step of the solve runs in the library's CUDA kernels; this module never
computes the method.  Arrays may be numpy arrays (host) or torch CUDA tensors
(device); outputs are returned as numpy arrays unless device tensors are
passed in.  If the compiled library is missing this module raises at import
time: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libmlq.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libmlq is not built ({LIB_PATH} missing); run paper_2105_02007_gb300.build.build()")

_lib = ctypes.CDLL(LIB_PATH)

MLQ_FP64, MLQ_MIXED = 0, 1
MLQ_EINVAL, MLQ_ENOMEM, MLQ_ETIMEOUT, MLQ_EUNSUPPORTED = -1, -2, -5, -6
S_CONVERGED, S_MAXITER, S_NONFINITE, S_CANCELLED = 0, 1, 2, 3


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("rtol", ctypes.c_double), ("rtol_inner", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("max_sweeps", ctypes.c_int), ("cluster", ctypes.c_int),
                ("threads", ctypes.c_int), ("storage", ctypes.c_int), ("graphs", ctypes.c_int),
                ("precond", ctypes.c_int)]


class Model(ctypes.Structure):
    _fields_ = [("s_l", ctypes.c_double), ("s_t", ctypes.c_double), ("a", ctypes.c_double),
                ("eps", ctypes.c_double), ("gamma", ctypes.c_double), ("T", ctypes.c_double)]


class Scheme(ctypes.Structure):
    _fields_ = [("ionic", ctypes.c_int), ("theta", ctypes.c_double), ("alpha", ctypes.c_double),
                ("u_rest", ctypes.c_double), ("u_th", ctypes.c_double), ("u_peak", ctypes.c_double),
                ("amp", ctypes.c_double), ("sigma", ctypes.c_double), ("t1", ctypes.c_double),
                ("x0", ctypes.c_double * 3)]


class Request(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int), ("samples", ctypes.c_int64), ("xi", ctypes.c_void_p),
                ("target_rmse", ctypes.c_double), ("chunk", ctypes.c_int32)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("worst", ctypes.c_int32), ("samples_used", ctypes.c_int64),
                ("mean", ctypes.c_double), ("rmse", ctypes.c_double), ("latency_ms", ctypes.c_double),
                ("batches", ctypes.c_int64), ("first_ms", ctypes.c_double), ("last_ms", ctypes.c_double)]


class MemberStats(ctypes.Structure):
    _fields_ = [("kernel_ms", ctypes.c_double), ("level", ctypes.c_int), ("coarse", ctypes.c_int),
                ("cluster", ctypes.c_int), ("resident", ctypes.c_int), ("threads", ctypes.c_int),
                ("npt", ctypes.c_int), ("samples", ctypes.c_int64),
                ("nodes", ctypes.c_int64), ("steps", ctypes.c_int64), ("cg_iterations", ctypes.c_int64),
                ("start_ms", ctypes.c_double), ("end_ms", ctypes.c_double)]


_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_lib.mlq_default_options.argtypes = [ctypes.POINTER(Options), ctypes.c_int]
_lib.mlq_default_model.argtypes = [ctypes.POINTER(Model)]
_lib.mlq_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, _vp, ctypes.POINTER(Options)]
_lib.mlq_destroy.argtypes = [_vp]
_lib.mlq_set_options.argtypes = [_vp, ctypes.POINTER(Options)]
_lib.mlq_set_model.argtypes = [_vp, ctypes.POINTER(Model)]
_lib.mlq_add_level.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp, ctypes.c_double, ctypes.c_int32]
_lib.mlq_add_level_mesh.argtypes = [_vp, ctypes.c_int, _i64, _vp, _i64, _vp, _vp, ctypes.c_double, ctypes.c_int32]
_lib.mlq_group_selftest.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _i64]
_lib.mlq_set_initial_state.argtypes = [_vp, ctypes.c_int, _vp, _vp]
_lib.mlq_set_initial_disk.argtypes = [_vp, ctypes.c_int, ctypes.c_double]
_lib.mlq_set_kl.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp]
_lib.mlq_build_kl.argtypes = [ctypes.c_int, _vp, _vp, ctypes.c_double, ctypes.c_double, ctypes.c_int, _vp, _vp]
_lib.mlq_centroid_table.argtypes = [ctypes.c_int, _vp, _vp, ctypes.c_int, _vp, _vp]
_lib.mlq_build_kl_mesh.argtypes = [ctypes.c_int, _i64, _vp, _i64, _vp, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                   _vp, _vp]
_lib.mlq_p1_at_points.argtypes = [ctypes.c_int, _i64, _vp, _i64, _vp, ctypes.c_int, _vp, _i64, _vp, _vp]
_lib.mlq_p1_at_points_gpu.argtypes = [ctypes.c_int, _i64, _vp, _i64, _vp, ctypes.c_int, _vp, _i64, _vp, _vp]
_lib.mlq_mlmc_allocation.argtypes = [ctypes.c_int, _vp, _vp, ctypes.c_double, _i64, _vp]
_lib.mlq_mesh_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, _i64, _vp, _i64, _vp, _vp]
_lib.mlq_mesh_destroy.argtypes = [_vp]
_lib.mlq_mesh_set_kl.argtypes = [_vp, ctypes.c_int, _vp, _vp]
_lib.mlq_mesh_solve_opts.argtypes = [_vp, _vp, _vp, ctypes.c_double, ctypes.c_int32, _vp, _vp, _i64, _vp, _vp,
                                     _vp, _vp]
_lib.mlq_mesh_solve.argtypes = [_vp, _vp, ctypes.c_double, ctypes.c_int32, ctypes.c_double, _vp, _vp, _i64, _vp, _vp,
                                _vp, _vp]
_lib.mlq_solve.argtypes = [_vp, ctypes.c_int, _i64, _vp, ctypes.c_int, _vp, _vp, _vp, _vp, _vp]
_lib.mlq_solve_state.argtypes = [_vp, ctypes.c_int, _i64, _vp, _vp, _vp, _vp, _vp]
_lib.mlq_set_points.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_double]
_lib.mlq_solve_points.argtypes = [_vp, ctypes.c_int, _i64, _vp, _vp, _vp, _vp, _vp]
_lib.mlq_trace_prolong.argtypes = [ctypes.c_int, _vp, _vp]
_lib.mlq_time_norms.argtypes = [ctypes.c_int, ctypes.c_double, _vp, _vp, _vp]
_lib.mlq_mlmc_combine.argtypes = [ctypes.c_int, _vp, _vp, _vp, _vp, _vp]
_lib.mlq_estimate_adaptive.argtypes = [_vp, ctypes.c_int, ctypes.c_double, _i64, _vp, _vp, _vp, _vp, _vp, _vp]
_lib.mlq_field_prolong.argtypes = [ctypes.c_int, _vp, _vp, _vp]
_lib.mlq_field_norms.argtypes = [ctypes.c_int, _vp, _vp, _vp, _vp, _vp]
_lib.mlq_pimped_ml_combine.argtypes = [ctypes.c_int, _vp, _vp, _vp]
_lib.mlq_default_scheme.argtypes = [_vp]
_lib.mlq_set_scheme.argtypes = [_vp, _vp]
_lib.mlq_estimate.argtypes = [_vp, ctypes.c_int, _vp, _vp, _vp, _vp, _vp, _vp]
_lib.mlq_submit.argtypes = [_vp, _vp, _vp]
_lib.mlq_poll.argtypes = [_vp, ctypes.c_uint64, _vp]
_lib.mlq_serve_limits.argtypes = [_vp, ctypes.c_int, ctypes.c_size_t]
_lib.mlq_workspace_bytes.argtypes = [_vp, ctypes.c_int, _i64, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]
_lib.mlq_launch_count.argtypes = [_vp, ctypes.POINTER(_i64)]
_lib.mlq_level_launch.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                  ctypes.POINTER(ctypes.c_int)]
_lib.mlq_autotune.argtypes = [_vp, ctypes.c_int, _i64, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                              ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
_lib.mlq_solve_noalloc.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int32, _vp, _vp, ctypes.c_int, _vp, _vp,
                                   _vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp]
_lib.mlq_synthesize.argtypes = [_vp, ctypes.c_int, _i64, _vp, _vp]
_lib.mlq_set_profiling.argtypes = [_vp, ctypes.c_int]
_lib.mlq_member_profile.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(MemberStats)]
_lib.mlq_strerror.restype = ctypes.c_char_p
_lib.mlq_strerror.argtypes = [ctypes.c_int]
_lib.mlq_last_cuda_error.restype = ctypes.c_char_p
_lib.mlq_last_cuda_error.argtypes = [_vp]

EXPORTED = ["mlq_default_options", "mlq_default_model", "mlq_default_scheme", "mlq_set_scheme", "mlq_create", "mlq_destroy", "mlq_set_options",
            "mlq_set_model", "mlq_add_level", "mlq_add_level_mesh", "mlq_group_selftest", "mlq_set_initial_state", "mlq_set_initial_disk", "mlq_set_kl",
            "mlq_build_kl", "mlq_centroid_table", "mlq_build_kl_mesh", "mlq_p1_at_points", "mlq_p1_at_points_gpu", "mlq_mesh_create",
            "mlq_mesh_destroy", "mlq_mesh_set_kl", "mlq_mesh_solve", "mlq_mesh_solve_opts", "mlq_mlmc_allocation", "mlq_mlmc_combine", "mlq_pimped_ml_combine", "mlq_estimate_adaptive", "mlq_field_prolong", "mlq_field_norms", "mlq_solve", "mlq_solve_state", "mlq_set_points", "mlq_solve_points", "mlq_trace_prolong",
            "mlq_time_norms", "mlq_estimate", "mlq_workspace_bytes",
            "mlq_launch_count", "mlq_level_launch", "mlq_strerror", "mlq_last_cuda_error", "mlq_set_profiling",
            "mlq_member_profile", "mlq_autotune", "mlq_solve_noalloc", "mlq_synthesize", "mlq_submit", "mlq_poll", "mlq_serve_limits"]


class MLQError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        msg = f"{where}: {_lib.mlq_strerror(code).decode()} ({code})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)
        self.code = code


def _check(code: int, where: str, ctx=None):
    if code != 0:
        detail = _lib.mlq_last_cuda_error(ctx).decode() if ctx else ""
        raise MLQError(code, where, detail)


def _host(a, dtype):
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr, arr.ctypes.data_as(_vp)


def _ptr(a, dtype):
    """Pointer to a numpy array (made contiguous) or a torch tensor (host or
    CUDA).  Returns (keepalive, pointer)."""
    if a is None:
        return None, None
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        assert a.is_contiguous()
        return a, _vp(a.data_ptr())
    return _host(a, dtype)


def default_options(precision: int = MLQ_FP64, **kw) -> Options:
    o = Options()
    _check(_lib.mlq_default_options(ctypes.byref(o), precision), "mlq_default_options")
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def default_model(**kw) -> Model:
    m = Model()
    _check(_lib.mlq_default_model(ctypes.byref(m)), "mlq_default_model")
    for k, v in kw.items():
        setattr(m, k, v)
    return m


def _dims(m):
    """(dim, int32[3]) from m (2D, m x m nodes) or (mx, my, mz) (3D)."""
    if np.ndim(m) == 0:
        return 2, np.array([int(m), 0, 0], dtype=np.int32)
    return 3, np.array([int(v) for v in m], dtype=np.int32)


def _counts(dim, d):
    """(nodes, elements) of a structured mesh."""
    if dim == 2:
        return int(d[0]) ** 2, 2 * (int(d[0]) - 1) ** 2
    return int(d[0] * d[1] * d[2]), 6 * int((d[0] - 1) * (d[1] - 1) * (d[2] - 1))


def build_kl(m, sigma2: float, ell: float, K: int, lengths=None):
    """KL modes (n x K) and eigenvalues (K) on the structured mesh: m x m
    nodes on the unit square, or m = (mx, my, mz) nodes on the box with the
    given lengths (default 1 x 1 x 0.25) in Kuhn tetrahedra."""
    dim, dims = _dims(m)
    n, _ = _counts(dim, dims)
    lg = None if lengths is None else np.ascontiguousarray(lengths, dtype=np.float64)
    modes = np.zeros((n, K))
    lam = np.zeros(K)
    _check(_lib.mlq_build_kl(dim, dims.ctypes.data_as(_vp), None if lg is None else lg.ctypes.data_as(_vp),
                             sigma2, ell, K, modes.ctypes.data_as(_vp), lam.ctypes.data_as(_vp)), "mlq_build_kl")
    return modes, lam


def centroid_table(m_fine, modes_f: np.ndarray, m_coarse) -> np.ndarray:
    """Midpoint-rule transfer of fine nodal modes to the coarse elements (2D:
    m x m meshes; 3D: (mx, my, mz) meshes of the same box)."""
    K = modes_f.shape[1]
    dim, fd = _dims(m_fine)
    _, cd = _dims(m_coarse)
    mf, pm = _host(modes_f, np.float64)
    phi = np.zeros((_counts(dim, cd)[1], K))
    _check(_lib.mlq_centroid_table(dim, fd.ctypes.data_as(_vp), pm, K, cd.ctypes.data_as(_vp),
                                   phi.ctypes.data_as(_vp)), "mlq_centroid_table")
    return phi


def group_selftest(ctas: int, rounds: int, missing: int = 0, max_polls: int = 1 << 16, device: int = 0) -> int:
    """mlq_group_selftest: the status code (MLQ_OK = 0, MLQ_ETIMEOUT when a
    barrier wait ran out)."""
    return int(_lib.mlq_group_selftest(device, ctas, rounds, missing, max_polls))


def _mesh_args(xyz, conn):
    xyz, px = _host(xyz, np.float64)
    conn, pc = _host(conn, np.int32)
    return xyz, px, conn, pc


def build_kl_mesh(xyz: np.ndarray, conn: np.ndarray, sigma2: float, ell: float, K: int):
    """KL modes (n x K) and eigenvalues (K) on a general simplicial mesh
    (nodes n x dim, simplices n_e x (dim + 1))."""
    xyz, px, conn, pc = _mesh_args(xyz, conn)
    n, dim = xyz.shape
    modes = np.zeros((n, K))
    lam = np.zeros(K)
    _check(_lib.mlq_build_kl_mesh(dim, n, px, conn.shape[0], pc, sigma2, ell, K, modes.ctypes.data_as(_vp),
                                  lam.ctypes.data_as(_vp)), "mlq_build_kl_mesh")
    return modes, lam


def p1_at_points(xyz: np.ndarray, conn: np.ndarray, f: np.ndarray, pts: np.ndarray, device: bool = False) -> np.ndarray:
    """Values at points (np x dim) of the P1 interpolants of nodal fields
    f (n x K) on a general simplicial mesh (the transfer between unrelated
    meshes); device=True locates the points on the current CUDA device
    (mlq_p1_at_points_gpu), else on the host cores."""
    xyz, px, conn, pc = _mesh_args(xyz, conn)
    n, dim = xyz.shape
    f2 = np.asarray(f, dtype=np.float64)
    f2 = f2[:, None] if f2.ndim == 1 else f2
    f2, pf = _host(f2, np.float64)
    pts, pp = _host(pts, np.float64)
    out = np.zeros((pts.shape[0], f2.shape[1]))
    fn = _lib.mlq_p1_at_points_gpu if device else _lib.mlq_p1_at_points
    _check(fn(dim, n, px, conn.shape[0], pc, f2.shape[1], pf, pts.shape[0], pp, out.ctypes.data_as(_vp)),
           "mlq_p1_at_points_gpu" if device else "mlq_p1_at_points")
    return out


def mlmc_allocation(var, cost, eps: float, nmin: int = 2) -> np.ndarray:
    """Samples per level minimising the cost for RMSE_stat <= eps
    (mlq_mlmc_allocation)."""
    var, pv = _host(var, np.float64)
    cost, pc = _host(cost, np.float64)
    N = np.zeros(var.size, dtype=np.int64)
    _check(_lib.mlq_mlmc_allocation(var.size - 1, pv, pc, eps, nmin, N.ctypes.data_as(_vp)), "mlq_mlmc_allocation")
    return N


class MeshLevel:
    """A level on a general tetrahedral mesh (mlq_mesh_*) for non-nested
    hierarchies: Jacobi-PCG in FP64, or FP32 inside FP64 refinement."""

    def __init__(self, xyz: np.ndarray, conn: np.ndarray, frames=None, device: int = 0):
        self._xyz, px, self._conn, pc = _mesh_args(xyz, conn)
        self.n, self.ne = self._xyz.shape[0], self._conn.shape[0]
        fr, pf = (None, None) if frames is None else _host(frames, np.float64)
        h = _vp()
        _check(_lib.mlq_mesh_create(ctypes.byref(h), device, self.n, px, self.ne, pc, pf), "mlq_mesh_create")
        self._h = h
        self.K = 0

    def close(self):
        if getattr(self, "_h", None):
            _lib.mlq_mesh_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        self.close()

    def set_kl(self, phi: np.ndarray, theta_mean=None):
        phi, pp = _host(phi, np.float64)
        tm, pt = (None, None) if theta_mean is None else _host(theta_mean, np.float64)
        _check(_lib.mlq_mesh_set_kl(self._h, phi.shape[1], pp, pt), "mlq_mesh_set_kl")
        self.K = phi.shape[1]

    def solve(self, xi: np.ndarray, dt: float, nsteps: int, v0: np.ndarray, w0=None, rtol: float = 1e-13,
              model=None, precision=None, **opts):
        """S samples xi (S x K) over nsteps blocks from v0, w0.  precision None:
        mlq_mesh_solve (FP64, rtol); MLQ_FP64 / MLQ_MIXED: mlq_mesh_solve_opts
        with the default options of that precision updated by opts (rtol,
        cluster, max_iter, ...).  Returns (Q, status, iters)."""
        if precision is not None:
            o = default_options(precision, **opts)
            return self._solve_opts(xi, dt, nsteps, v0, w0, model, o)
        xi, px = _host(xi, np.float64)
        S = xi.shape[0]
        v0, pv = _host(v0, np.float64)
        w0a, pw = (None, None) if w0 is None else _host(w0, np.float64)
        md = Model()
        _lib.mlq_default_model(ctypes.byref(md))
        for k, v in (model or {}).items():
            setattr(md, k, v)
        q = np.zeros(S)
        st = np.zeros(S, dtype=np.int32)
        it = np.zeros(S, dtype=np.int32)
        _check(_lib.mlq_mesh_solve(self._h, ctypes.byref(md), dt, nsteps, rtol, pv, pw, S, px,
                                   q.ctypes.data_as(_vp), st.ctypes.data_as(_vp), it.ctypes.data_as(_vp)),
               "mlq_mesh_solve")
        return q, st, it

    def _solve_opts(self, xi, dt, nsteps, v0, w0, model, o):
        xi, px = _host(xi, np.float64)
        S = xi.shape[0]
        v0, pv = _host(v0, np.float64)
        w0a, pw = (None, None) if w0 is None else _host(w0, np.float64)
        md = Model()
        _lib.mlq_default_model(ctypes.byref(md))
        for k, v in (model or {}).items():
            setattr(md, k, v)
        q = np.zeros(S)
        st = np.zeros(S, dtype=np.int32)
        it = np.zeros(S, dtype=np.int32)
        _check(_lib.mlq_mesh_solve_opts(self._h, ctypes.byref(md), ctypes.byref(o), dt, nsteps, pv, pw, S, px,
                                        q.ctypes.data_as(_vp), st.ctypes.data_as(_vp), it.ctypes.data_as(_vp)),
               "mlq_mesh_solve_opts")
        return q, st, it


MLQ_ETOOBIG = -7


def solve_noalloc(m: int, dt: float, nsteps: int, phi, xi, q, status=None, iters=None, theta_mean=None,
                  v0=None, w0=None, stream=None, model: Model | None = None, options: Options | None = None):
    """The library's allocation-free solve (mlq_solve_noalloc): every array
    argument is a CUDA tensor owned by the caller; the work is queued on
    `stream` (a cudaStream_t handle, None = legacy default stream) and the
    call returns without waiting."""
    def dp(t):
        return None if t is None else _vp(t.data_ptr())

    K = int(xi.shape[1])
    code = _lib.mlq_solve_noalloc(m, dt, nsteps, ctypes.byref(model) if model is not None else None,
                                  ctypes.byref(options) if options is not None else None, K, dp(phi),
                                  dp(theta_mean), dp(xi), int(xi.shape[0]), dp(v0), dp(w0), dp(q), dp(status),
                                  dp(iters), _vp(stream) if stream else None)
    _check(code, "mlq_solve_noalloc")


class Context:
    """One libmlq context on a CUDA device, issuing work on a CUDA stream."""

    def __init__(self, device: int = 0, precision: int = MLQ_FP64, stream=None, **opts):
        self._h = _vp()
        self.options = default_options(precision, **opts)
        sp = _vp(stream) if stream else None
        _check(_lib.mlq_create(ctypes.byref(self._h), device, sp, ctypes.byref(self.options)), "mlq_create")
        self.levels = {}

    def close(self):
        if self._h:
            _lib.mlq_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_options(self, **kw):
        for k, v in kw.items():
            setattr(self.options, k, v)
        _check(_lib.mlq_set_options(self._h, ctypes.byref(self.options)), "mlq_set_options", self._h)

    def set_model(self, **kw):
        _check(_lib.mlq_set_model(self._h, ctypes.byref(default_model(**kw))), "mlq_set_model", self._h)

    def set_scheme(self, **kw):
        """Time scheme and ionic model (mlq_set_scheme): ionic=1 selects the
        paper's scheme; other keys override mlq_default_scheme's values
        (x0 as a sequence)."""
        sc = Scheme()
        _lib.mlq_default_scheme(ctypes.byref(sc))
        for k, v in kw.items():
            if k == "x0":
                for i, c in enumerate(v):
                    sc.x0[i] = float(c)
            else:
                setattr(sc, k, v)
        _check(_lib.mlq_set_scheme(self._h, ctypes.byref(sc)), "mlq_set_scheme", self._h)

    def add_level(self, level: int, m, dt: float, nsteps: int, lengths=None):
        """Level on m x m nodes (2D) or m = (mx, my, mz) nodes of the box with
        `lengths` (3D, default 1 x 1 x 0.25)."""
        dim, dims = _dims(m)
        lg = None if lengths is None else np.ascontiguousarray(lengths, dtype=np.float64)
        _check(_lib.mlq_add_level(self._h, level, dim, dims.ctypes.data_as(_vp),
                                  None if lg is None else lg.ctypes.data_as(_vp), dt, nsteps),
               "mlq_add_level", self._h)
        n, ne = _counts(dim, dims)
        self.levels[level] = dict(m=m, dt=dt, nsteps=nsteps, n=n, ne=ne)

    def add_level_mesh(self, level: int, xyz: np.ndarray, conn: np.ndarray, dt: float, nsteps: int, frames=None):
        """Level on a general tetrahedral mesh (xyz n x 3, conn ne x 4, optional
        fibre frames ne x 6): a level of mlq_solve / mlq_estimate whose members
        run the general-mesh solver."""
        x, px, c, pc = _mesh_args(xyz, conn)
        fr, pf = (None, None) if frames is None else _host(frames, np.float64)
        _check(_lib.mlq_add_level_mesh(self._h, level, x.shape[0], px, c.shape[0], pc, pf, dt, nsteps),
               "mlq_add_level_mesh", self._h)
        self.levels[level] = dict(m=None, dt=dt, nsteps=nsteps, n=x.shape[0], ne=c.shape[0], mesh=True)

    def set_initial_state(self, level: int, v0, w0=None):
        v, pv = _host(v0, np.float64)
        w, pw = (None, None) if w0 is None else _host(w0, np.float64)
        _check(_lib.mlq_set_initial_state(self._h, level, pv, pw), "mlq_set_initial_state", self._h)

    def set_initial_disk(self, level: int, radius: float):
        _check(_lib.mlq_set_initial_disk(self._h, level, radius), "mlq_set_initial_disk", self._h)

    def set_kl(self, level: int, phi: np.ndarray, theta_mean=None):
        p, pp = _host(phi, np.float64)
        t, pt = (None, None) if theta_mean is None else _host(theta_mean, np.float64)
        _check(_lib.mlq_set_kl(self._h, level, p.shape[1], pp, pt), "mlq_set_kl", self._h)
        self.levels[level]["K"] = p.shape[1]

    def solve(self, level: int, xi, with_coarse: bool = False, out=None):
        """Solve the samples xi (S x K) on `level` (and level-1).  Returns a
        dict of numpy arrays q_fine, q_coarse, y, status, iters, or fills the
        given device tensors in `out`."""
        xk, px = _ptr(xi, np.float64)
        S = int(xi.shape[0])
        if out is None:
            res = dict(q_fine=np.zeros(S), q_coarse=np.zeros(S) if with_coarse else None,
                       y=np.zeros(S), status=np.zeros(S, dtype=np.int32), iters=np.zeros(S, dtype=np.int32))
        else:
            res = out
        ptrs = {k: (None if v is None else _ptr(v, np.float64 if k in ("q_fine", "q_coarse", "y") else np.int32)[1])
                for k, v in res.items()}
        _check(_lib.mlq_solve(self._h, level, S, px, int(bool(with_coarse)), ptrs.get("q_fine"),
                              ptrs.get("q_coarse"), ptrs.get("y"), ptrs.get("status"), ptrs.get("iters")),
               "mlq_solve", self._h)
        return res

    def solve_state(self, level: int, xi):
        """Final state of the samples xi (S x K) on `level` (mlq_solve_state):
        dict of numpy arrays v, w (S x n), q (S) and status (S)."""
        xk, px = _ptr(xi, np.float64)
        S = int(xi.shape[0])
        n = self.levels[level]["n"]
        res = dict(v=np.zeros((S, n)), w=np.zeros((S, n)), q=np.zeros(S), status=np.zeros(S, dtype=np.int32))
        _check(_lib.mlq_solve_state(self._h, level, S, px, res["v"].ctypes.data_as(_vp),
                                    res["w"].ctypes.data_as(_vp), res["q"].ctypes.data_as(_vp),
                                    res["status"].ctypes.data_as(_vp)), "mlq_solve_state", self._h)
        return res

    def set_points(self, level: int, pts, u_th: float):
        """Point QoIs of `level` at pts (np x dim) with threshold u_th (mlq_set_points)."""
        lv = self.levels[level]
        dim = 3 if lv.get("mesh") or isinstance(lv["m"], (tuple, list)) else 2
        p = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, dim)
        _check(_lib.mlq_set_points(self._h, level, p.shape[0], p.ctypes.data_as(_vp) if p.size else None,
                                   float(u_th)), "mlq_set_points", self._h)
        self.levels[level]["npts"] = p.shape[0]

    def solve_points(self, level: int, xi):
        """Traces and activation times of the samples xi (S x K) on `level`
        (mlq_solve_points): dict of numpy arrays trace (S, np, nsteps + 1),
        act (S, np), q (S), status (S)."""
        xk, px = _ptr(xi, np.float64)
        S = int(xi.shape[0])
        L = self.levels[level]
        npts, nt = L["npts"], L["nsteps"]
        res = dict(trace=np.zeros((S, npts, nt + 1)), act=np.zeros((S, npts)), q=np.zeros(S),
                   status=np.zeros(S, dtype=np.int32))
        _check(_lib.mlq_solve_points(self._h, level, S, px, res["trace"].ctypes.data_as(_vp),
                                     res["act"].ctypes.data_as(_vp), res["q"].ctypes.data_as(_vp),
                                     res["status"].ctypes.data_as(_vp)), "mlq_solve_points", self._h)
        return res

    def estimate_adaptive(self, xis, eps: float, n_pilot: int = 16):
        """Adaptive MLMC over the pools xis[l] (Nmax_l x K) for a target
        statistical error eps (mlq_estimate_adaptive).  Returns (N_l, mean,
        var_l, rmse)."""
        L = len(xis) - 1
        keep = [_ptr(x, np.float64) for x in xis]
        Nmax = np.array([int(x.shape[0]) for x in xis], dtype=np.int64)
        xp = (_vp * (L + 1))(*[k[1] for k in keep])
        N = np.zeros(L + 1, dtype=np.int64)
        mean = ctypes.c_double()
        var = np.zeros(L + 1)
        rmse = ctypes.c_double()
        _check(_lib.mlq_estimate_adaptive(self._h, L, float(eps), int(n_pilot), Nmax.ctypes.data_as(_vp), xp,
                                          N.ctypes.data_as(_vp), ctypes.byref(mean), var.ctypes.data_as(_vp),
                                          ctypes.byref(rmse)), "mlq_estimate_adaptive", self._h)
        return N, mean.value, var, rmse.value

    def estimate(self, xis, return_y: bool = False):
        """MLMC over levels 0..L with xis[l] (N_l x K).  Returns (mean,
        var_l, rmse[, y_l])."""
        L = len(xis) - 1
        keep = [_ptr(x, np.float64) for x in xis]
        N = np.array([int(x.shape[0]) for x in xis], dtype=np.int64)
        xp = (_vp * (L + 1))(*[k[1] for k in keep])
        mean = ctypes.c_double()
        var = np.zeros(L + 1)
        rmse = ctypes.c_double()
        ys = [np.zeros(int(n)) for n in N] if return_y else None
        yp = (_vp * (L + 1))(*[y.ctypes.data_as(_vp) for y in ys]) if return_y else None
        _check(_lib.mlq_estimate(self._h, L, N.ctypes.data_as(_vp), xp, ctypes.byref(mean),
                                 var.ctypes.data_as(_vp), ctypes.byref(rmse), yp), "mlq_estimate", self._h)
        if return_y:
            return mean.value, var, rmse.value, ys
        return mean.value, var, rmse.value

    def synthesize(self, level: int, xi):
        """KL synthesis alone: (cos 2 theta, sin 2 theta), shape (S, n_elem, 2)."""
        keep, px = _ptr(xi, np.float64)
        S = int(xi.shape[0])
        out = np.zeros((S, self.levels[level]["ne"], 2))
        _check(_lib.mlq_synthesize(self._h, level, S, px, out.ctypes.data_as(_vp)), "mlq_synthesize", self._h)
        return out

    def workspace_bytes(self, level: int, S: int, with_coarse: bool = False) -> int:
        b = ctypes.c_size_t()
        _check(_lib.mlq_workspace_bytes(self._h, level, S, int(with_coarse), ctypes.byref(b)),
               "mlq_workspace_bytes", self._h)
        return b.value

    def autotune(self, level: int, xi, probe_steps: int = 2):
        """Time the launch shapes of a level on a short probe run and keep
        the fastest.  Returns (cluster, threads, probe ms)."""
        keep, px = _ptr(xi, np.float64)
        c, t, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _check(_lib.mlq_autotune(self._h, level, int(xi.shape[0]), px, probe_steps, ctypes.byref(c),
                                 ctypes.byref(t), ctypes.byref(ms)), "mlq_autotune", self._h)
        return c.value, t.value, ms.value

    def set_profiling(self, enable: bool = True):
        _check(_lib.mlq_set_profiling(self._h, int(enable)), "mlq_set_profiling", self._h)

    def member_profile(self):
        """Per-member slab-kernel timings and CG iteration totals of the last
        solve / estimate (profiling must be on)."""
        buf = (MemberStats * 16)()
        cnt = ctypes.c_int()
        _check(_lib.mlq_member_profile(self._h, 16, ctypes.byref(cnt), buf), "mlq_member_profile", self._h)
        return [{f: getattr(buf[k], f) for f, _ in MemberStats._fields_} for k in range(min(cnt.value, 16))]

    def submit(self, level: int, xi, target_rmse: float = 0.0, chunk: int = 16) -> int:
        """Queue a request for the mean of Q_level over the rows of xi (host,
        samples x K), stopping at the first chunk boundary where the
        statistical error sqrt(V_n / n) <= target_rmse.  Returns a ticket."""
        x, px = _host(xi, np.float64)
        req = Request(level, int(x.shape[0]), px, float(target_rmse), int(chunk))
        t = ctypes.c_uint64()
        _check(_lib.mlq_submit(self._h, ctypes.byref(req), ctypes.byref(t)), "mlq_submit", self._h)
        return t.value

    def serve_limits(self, lanes: int = 4, max_bytes: int = 0):
        """Serving lanes and workspace budget (mlq_serve_limits)."""
        _check(_lib.mlq_serve_limits(self._h, int(lanes), int(max_bytes)), "mlq_serve_limits", self._h)

    def poll(self, ticket: int):
        """None while the request runs, else a dict of its result (the ticket
        is released)."""
        res = Result()
        code = _lib.mlq_poll(self._h, ctypes.c_uint64(ticket), ctypes.byref(res))
        if code == -4:
            return None
        _check(code, "mlq_poll", self._h)
        return {f: getattr(res, f) for f, _ in Result._fields_}

    def wait(self, ticket: int, timeout: float = 600.0, interval: float = 0.002):
        """Poll until the request is done (or raise TimeoutError)."""
        import time

        end = time.monotonic() + timeout
        while True:
            r = self.poll(ticket)
            if r is not None:
                return r
            if time.monotonic() > end:
                raise TimeoutError(f"request {ticket} not done after {timeout} s")
            time.sleep(interval)

    def launch_count(self) -> int:
        c = _i64()
        _check(_lib.mlq_launch_count(self._h, ctypes.byref(c)), "mlq_launch_count")
        return c.value

    def level_launch(self, level: int, with_resident: bool = False):
        """(cluster, threads[, resident]) chosen for a level; resident is 2 for
        the register-resident kernel, 1 for shared-memory vectors, 0 global."""
        c, t, r = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(_lib.mlq_level_launch(self._h, level, ctypes.byref(c), ctypes.byref(t), ctypes.byref(r)),
               "mlq_level_launch")
        return (c.value, t.value, r.value) if with_resident else (c.value, t.value)


def trace_prolong(u_c):
    """Coarse trace on the fine time grid (mlq_trace_prolong)."""
    u = np.ascontiguousarray(u_c, dtype=np.float64)
    out = np.zeros(2 * (u.size - 1) + 1)
    _check(_lib.mlq_trace_prolong(u.size - 1, u.ctypes.data_as(_vp), out.ctypes.data_as(_vp)), "mlq_trace_prolong")
    return out


def time_norms(e, T: float):
    """(L2(0,T), H1(0,T)) norms of the linear interpolant of e (mlq_time_norms)."""
    a = np.ascontiguousarray(e, dtype=np.float64)
    l2 = ctypes.c_double()
    h1 = ctypes.c_double()
    _check(_lib.mlq_time_norms(a.size - 1, float(T), a.ctypes.data_as(_vp), ctypes.byref(l2), ctypes.byref(h1)),
           "mlq_time_norms")
    return l2.value, h1.value


def mlmc_combine(ys):
    """eq. StandardML over per-sample level differences ys[l] (host arrays),
    sums in index order (mlq_mlmc_combine).  Returns (mean, var_l, rmse)."""
    arrs = [np.ascontiguousarray(y, dtype=np.float64) for y in ys]
    L = len(arrs) - 1
    N = np.array([a.size for a in arrs], dtype=np.int64)
    ptrs = (_vp * (L + 1))(*[a.ctypes.data_as(_vp) for a in arrs])
    mean = ctypes.c_double()
    var = np.zeros(L + 1)
    rmse = ctypes.c_double()
    _check(_lib.mlq_mlmc_combine(L, N.ctypes.data_as(_vp), ptrs, ctypes.byref(mean), var.ctypes.data_as(_vp),
                                 ctypes.byref(rmse)), "mlq_mlmc_combine")
    return mean.value, var, rmse.value


def field_prolong(m_coarse, vc):
    """The coarse field vc on the nested fine mesh (mlq_field_prolong);
    m_coarse: nodes per side (2D) or (mx, my, mz) (3D)."""
    dim, dims = _dims(m_coarse)
    v = np.ascontiguousarray(vc, dtype=np.float64)
    nf = int(np.prod([2 * int(d) - 1 for d in dims]) if dim == 3 else (2 * int(dims[0]) - 1) ** 2)
    out = np.zeros(nf)
    _check(_lib.mlq_field_prolong(dim, dims.ctypes.data_as(_vp), v.ctypes.data_as(_vp), out.ctypes.data_as(_vp)),
           "mlq_field_prolong")
    return out


def field_norms(m, e, lengths=None):
    """(L2(D), H1(D)) norms of the P1 field e on a structured level (mlq_field_norms)."""
    dim, dims = _dims(m)
    a = np.ascontiguousarray(e, dtype=np.float64)
    lg = None if lengths is None else np.ascontiguousarray(lengths, dtype=np.float64)
    l2 = ctypes.c_double()
    h1 = ctypes.c_double()
    _check(_lib.mlq_field_norms(dim, dims.ctypes.data_as(_vp), None if lg is None else lg.ctypes.data_as(_vp),
                                a.ctypes.data_as(_vp), ctypes.byref(l2), ctypes.byref(h1)), "mlq_field_norms")
    return l2.value, h1.value


def pimped_ml_combine(F_terms, N):
    """eq. PimpedML over F_terms[l] = F_{L-l} at the first N[l] points
    (mlq_pimped_ml_combine)."""
    arrs = [np.ascontiguousarray(f, dtype=np.float64) for f in F_terms]
    L = len(arrs) - 1
    n = np.ascontiguousarray(N, dtype=np.int64)
    ptrs = (_vp * (L + 1))(*[a.ctypes.data_as(_vp) for a in arrs])
    est = ctypes.c_double()
    _check(_lib.mlq_pimped_ml_combine(L, n.ctypes.data_as(_vp), ptrs, ctypes.byref(est)), "mlq_pimped_ml_combine")
    return est.value
