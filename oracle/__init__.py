"""Test infrastructure: the plain FP64 CPU oracle.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg and reference arm (``--impl reference``) may import this package.  It shares no code with the CUDA path; the only
thing both sides take from a common module are the seeded sample points
(``paper_2105_02007_gb300.inputs``), which hold none of the method's
arithmetic.

The compiled part (``mlq_oracle.c``) implements the per-sample forward solve
exactly as the paper defines it (see that file's header).  This module adds a
ctypes loader, numpy wrappers and the estimators of Sec. 4:

  single level  QoI^SL_L = Q_L(F_L)                                   (eq. SL)
  multilevel    QoI^ML_L = sum_l Q_{L-l}(F_l - F_{l-1}), F_{-1} = 0   (eq. StandardML)

  non-nested   QoI^ML_L = sum_l (Q_l - Q_{l-1})(F_{L-l}), Q_{-1} = 0     (eq. PimpedML)

Parity status per function (each is pinned by ``tests/test_oracle_pins.py``
or, for the fibre frames, point location and eq. PimpedML,
``tests/test_oracle_lv.py``):
  mesh2d, mesh3d, assemble, kl_build, centroid_table, solve, solve_batch, solve_states,
  solve_points, activation_time, time_norms, solve_paper, solve_paper_batch,
  p1_at_points, centroid_table_unrelated, mc_estimate, mlmc_estimate,
  qmc_estimate, pimped_ml_estimate: pinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mlq_oracle.c")
_LIB = os.path.join(_HERE, "libmlq_oracle.so")
_lib = None

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP if available).  Returns the path."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    c = ctypes
    lib.mlqo_mesh2d.argtypes = [c.c_int, _f64p, _i32p]
    lib.mlqo_mesh3d.argtypes = [c.c_int, c.c_int, c.c_int, c.c_double, c.c_double, c.c_double, _f64p, _i32p]
    lib.mlqo_pattern_nnz.argtypes = [c.c_int, c.c_int64, c.c_int64, _i32p]
    lib.mlqo_pattern_nnz.restype = c.c_int64
    lib.mlqo_assemble.argtypes = [c.c_int, c.c_int64, _f64p, c.c_int64, _i32p, c.c_void_p, c.c_double,
                                  c.c_double, _i64p, _i32p, _f64p, _f64p]
    lib.mlqo_kl_build.argtypes = [c.c_int, c.c_int64, _f64p, c.c_int64, _i32p, c.c_double, c.c_double,
                                  c.c_int, _f64p, _f64p, c.c_void_p, c.c_void_p]
    lib.mlqo_centroid_table.argtypes = [c.c_int, _i32p, _f64p, _f64p, c.c_int, _f64p, c.c_int64, _i32p,
                                        _f64p]
    lib.mlqo_solve.argtypes = [c.c_int, c.c_int64, _f64p, c.c_int64, _i32p, _f64p, _f64p, c.c_double,
                               c.c_int, c.c_double, c.c_int64, _f64p, _f64p, c.POINTER(c.c_double),
                               c.POINTER(c.c_int64), c.POINTER(c.c_int32)]
    lib.mlqo_solve_batch.argtypes = [c.c_int, c.c_int64, _f64p, c.c_int64, _i32p, c.c_int, _f64p, c.c_void_p,
                                     c.c_int64, _f64p, _f64p, c.c_double, c.c_int, c.c_double, c.c_int64,
                                     _f64p, c.c_void_p, c.c_int, _f64p, _i64p, _i32p]
    lib.mlqo_assemble_f.argtypes = [c.c_int, c.c_int64, _f64p, c.c_int64, _i32p, c.c_void_p, c.c_void_p,
                                    c.c_double, c.c_double, _i64p, _i32p, _f64p, _f64p]
    lib.mlqo_solve_batch_f.argtypes = [c.c_int, c.c_int64, _f64p, c.c_int64, _i32p, c.c_void_p, c.c_int, _f64p,
                                       c.c_void_p, c.c_int64, _f64p, _f64p, c.c_double, c.c_int, c.c_double,
                                       c.c_int64, _f64p, c.c_void_p, c.c_int, _f64p, _i64p, _i32p]
    lib.mlqo_p1_at_points.argtypes = [c.c_int, c.c_int64, _f64p, c.c_int64, _i32p, c.c_int, _f64p, c.c_int64,
                                      _f64p, _f64p, c.c_void_p, c.c_void_p]
    lib.mlqo_solve_paper.argtypes = [c.c_int, c.c_int64, _f64p, c.c_int64, _i32p, _f64p, _f64p, c.c_double, c.c_int,
                                     c.c_double, c.c_int64, _f64p, c.POINTER(c.c_double), c.POINTER(c.c_int64),
                                     c.POINTER(c.c_int32)]
    lib.mlqo_max_threads.restype = c.c_int
    _lib = lib
    return lib


def max_threads() -> int:
    return int(_load().mlqo_max_threads())


# --------------------------------------------------------------------------
# meshes (Sec. 3.1)
# --------------------------------------------------------------------------
class Mesh:
    """A simplicial mesh: nodes and elements (dims and box lengths for the
    structured meshes, zeros for an unstructured one)."""

    def __init__(self, dim, dims, lengths, xyz, conn):
        self.dim = dim
        self.dims = tuple(int(v) for v in dims)
        self.lengths = tuple(float(v) for v in lengths)
        self.xyz = xyz
        self.conn = conn

    @property
    def n(self) -> int:
        return self.xyz.shape[0]

    @property
    def ne(self) -> int:
        return self.conn.shape[0]


def mesh2d(m: int) -> Mesh:
    """Unit square, m x m nodes, two triangles per square (see mlq_oracle.c)."""
    xy = np.zeros((m * m, 2))
    conn = np.zeros((2 * (m - 1) ** 2, 3), dtype=np.int32)
    assert _load().mlqo_mesh2d(m, xy, conn) == 0
    return Mesh(2, (m,), (1.0, 1.0), xy, conn)


def unstructured_mesh(xyz: np.ndarray, conn: np.ndarray) -> Mesh:
    """A mesh given by its nodes (n x dim) and simplices (n_e x (dim + 1))."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    d = xyz.shape[1]
    assert conn.shape[1] == d + 1
    return Mesh(d, (0,) * d, (0.0,) * d, xyz, conn)


def mesh3d(mx: int, my: int, mz: int, lx: float = 1.0, ly: float = 1.0, lz: float = 0.25) -> Mesh:
    """Box [0,lx]x[0,ly]x[0,lz], mx*my*mz nodes, six Kuhn tetrahedra per cube."""
    xyz = np.zeros((mx * my * mz, 3))
    conn = np.zeros((6 * (mx - 1) * (my - 1) * (mz - 1), 4), dtype=np.int32)
    assert _load().mlqo_mesh3d(mx, my, mz, lx, ly, lz, xyz, conn) == 0
    return Mesh(3, (mx, my, mz), (lx, ly, lz), xyz, conn)


# --------------------------------------------------------------------------
# matrices (Sec. 3.1, eq. AdmV)
# --------------------------------------------------------------------------
def _opt(a, shape=None):
    if a is None:
        return None, None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        assert a.shape == shape, (a.shape, shape)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def assemble(mesh: Mesh, theta=None, s_l: float = 1.0, s_t: float = 0.2, frames=None):
    """CSR (rp, ci, M values, K values) of the consistent mass matrix and the
    stiffness matrix of D = s_t I + (s_l - s_t) f f^T, f = cos t e1 + sin t e2
    with (e1, e2) the element's frame (frames: n_e x 6) or the x-y axes."""
    lib = _load()
    nnz = lib.mlqo_pattern_nnz(mesh.dim, mesh.n, mesh.ne, mesh.conn)
    rp = np.zeros(mesh.n + 1, dtype=np.int64)
    ci = np.zeros(nnz, dtype=np.int32)
    mv = np.zeros(nnz)
    kv = np.zeros(nnz)
    th = None
    if theta is not None:
        th = np.ascontiguousarray(theta, dtype=np.float64)
        assert th.shape == (mesh.ne,)
    ptr = th.ctypes.data_as(ctypes.c_void_p) if th is not None else None
    fr, fptr = _opt(frames, (mesh.ne, 6))
    assert lib.mlqo_assemble_f(mesh.dim, mesh.n, mesh.xyz, mesh.ne, mesh.conn, ptr, fptr, s_l, s_t, rp, ci, mv,
                               kv) == 0
    return rp, ci, mv, kv


def csr_to_dense(rp, ci, val, n):
    A = np.zeros((n, n))
    for i in range(n):
        A[i, ci[rp[i]:rp[i + 1]]] = val[rp[i]:rp[i + 1]]
    return A


# --------------------------------------------------------------------------
# KL expansion (Sec. 2.3)
# --------------------------------------------------------------------------
def kl_build(mesh: Mesh, sigma2: float, ell: float, K: int, return_factor: bool = False):
    """Modes v_k (n x K, v_i^T M v_j = lambda_i delta_ij) and eigenvalues
    lambda (K) of the rank-K pivoted-Cholesky KL expansion of the covariance
    sigma2 exp(-|x-y|^2/ell) (eqs. approxEig, redEig)."""
    lib = _load()
    modes = np.zeros((mesh.n, K))
    lam = np.zeros(K)
    L = np.zeros((mesh.n, K)) if return_factor else None
    piv = np.zeros(K, dtype=np.int64) if return_factor else None
    st = lib.mlqo_kl_build(mesh.dim, mesh.n, mesh.xyz, mesh.ne, mesh.conn, sigma2, ell, K, modes, lam,
                           L.ctypes.data_as(ctypes.c_void_p) if L is not None else None,
                           piv.ctypes.data_as(ctypes.c_void_p) if piv is not None else None)
    assert st == 0, st
    if return_factor:
        return modes, lam, L, piv
    return modes, lam


def kl_synthesis(phi: np.ndarray, xi: np.ndarray, theta_mean=None) -> np.ndarray:
    """eq. KLlowrank per element: theta[s, e] = theta_mean[e] + sum_k phi[e, k]
    xi[s, k], returned as (cos 2 theta, sin 2 theta) with shape (S, n_elem, 2),
    the form the fibre tensor D = s_t I + (s_l - s_t) f f^T depends on."""
    theta = np.asarray(xi, dtype=np.float64) @ np.asarray(phi, dtype=np.float64).T
    if theta_mean is not None:
        theta = theta + np.asarray(theta_mean)[None, :]
    return np.stack([np.cos(2.0 * theta), np.sin(2.0 * theta)], axis=-1)


def centroid_table(fine: Mesh, modes_f: np.ndarray, coarse: Mesh) -> np.ndarray:
    """Phi[e, k] = fine P1 interpolant of mode k at the centroid of coarse
    element e: the midpoint-rule transfer of Sec. 4."""
    K = modes_f.shape[1]
    phi = np.zeros((coarse.ne, K))
    fd = np.array(fine.dims, dtype=np.int32)
    fl = np.array(fine.lengths, dtype=np.float64)
    assert _load().mlqo_centroid_table(fine.dim, fd, fl, np.ascontiguousarray(modes_f), K, coarse.xyz,
                                       coarse.ne, coarse.conn, phi) == 0
    return phi


# --------------------------------------------------------------------------
# forward solve
# --------------------------------------------------------------------------
DEFAULT_MODEL = dict(s_l=1.0, s_t=0.2, a=0.1, eps=0.01, gamma=0.5)


def _model_vec(model):
    m = dict(DEFAULT_MODEL)
    if model:
        m.update(model)
    return np.array([m["s_l"], m["s_t"], m["a"], m["eps"], m["gamma"]], dtype=np.float64)


def initial_state(mesh: Mesh, radius: float = 0.1):
    """v = 1 inside the ball of the given radius around the origin, else 0;
    w = 0."""
    r2 = np.sum(mesh.xyz ** 2, axis=1)
    v = np.where(r2 <= radius * radius, 1.0, 0.0)
    return v, np.zeros(mesh.n)


def solve(mesh: Mesh, theta, dt: float, nsteps: int, v0=None, w0=None, model=None, rtol: float = 1e-13,
          maxit: int | None = None):
    """One sample with angle field theta (per element).  Returns
    (Q, v_final, w_final, total CG iterations, status)."""
    lib = _load()
    if v0 is None:
        v0, w0 = initial_state(mesh)
    v = np.array(v0, dtype=np.float64)
    w = np.zeros(mesh.n) if w0 is None else np.array(w0, dtype=np.float64)
    q = ctypes.c_double()
    it = ctypes.c_int64()
    st = ctypes.c_int32()
    maxit = 10 * mesh.n if maxit is None else maxit
    th = np.ascontiguousarray(theta, dtype=np.float64)
    assert lib.mlqo_solve(mesh.dim, mesh.n, mesh.xyz, mesh.ne, mesh.conn, th, _model_vec(model), dt, nsteps,
                          rtol, maxit, v, w, ctypes.byref(q), ctypes.byref(it), ctypes.byref(st)) == 0
    return q.value, v, w, it.value, st.value


def solve_batch(mesh: Mesh, phi: np.ndarray, xi: np.ndarray, dt: float, nsteps: int, v0=None, w0=None,
                theta_mean=None, model=None, rtol: float = 1e-13, maxit: int | None = None,
                nthreads: int = 0, frames=None):
    """S samples: theta_e = theta_mean_e + sum_k phi[e,k] xi[s,k] (eq. KLlowrank),
    the fibre turned by theta_e in the plane of the element's frame (frames:
    n_e x 6) or of the x-y axes.  Returns (Q[S], iters[S], status[S])."""
    lib = _load()
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    S, K = xi.shape
    assert phi.shape == (mesh.ne, K)
    if v0 is None:
        v0, w0 = initial_state(mesh)
    v0 = np.ascontiguousarray(v0, dtype=np.float64)
    w0a = None if w0 is None else np.ascontiguousarray(w0, dtype=np.float64)
    tm = None if theta_mean is None else np.ascontiguousarray(theta_mean, dtype=np.float64)
    q = np.zeros(S)
    it = np.zeros(S, dtype=np.int64)
    st = np.zeros(S, dtype=np.int32)
    maxit = 10 * mesh.n if maxit is None else maxit
    fr, fptr = _opt(frames, (mesh.ne, 6))
    assert lib.mlqo_solve_batch_f(mesh.dim, mesh.n, mesh.xyz, mesh.ne, mesh.conn, fptr, K,
                                  np.ascontiguousarray(phi, dtype=np.float64),
                                  tm.ctypes.data_as(ctypes.c_void_p) if tm is not None else None, S, xi,
                                  _model_vec(model), dt, nsteps, rtol, maxit, v0,
                                  w0a.ctypes.data_as(ctypes.c_void_p) if w0a is not None else None, nthreads,
                                  q, it, st) == 0
    return q, it, st


def solve_states(mesh: Mesh, phi: np.ndarray, xi: np.ndarray, dt: float, nsteps: int, v0=None, w0=None,
                 theta_mean=None, model=None, rtol: float = 1e-13):
    """Final states of S samples, one at a time: theta_e = theta_mean_e +
    sum_k phi[e, k] xi[s, k] (eq. KLlowrank) and the same block loop as
    solve().  Returns (Q[S], v[S, n], w[S, n], status[S])."""
    xi = np.atleast_2d(np.asarray(xi, dtype=np.float64))
    S = xi.shape[0]
    q = np.zeros(S)
    V = np.zeros((S, mesh.n))
    W = np.zeros((S, mesh.n))
    st = np.zeros(S, dtype=np.int32)
    for s in range(S):
        theta = np.asarray(phi, dtype=np.float64) @ xi[s]
        if theta_mean is not None:
            theta = theta + np.asarray(theta_mean, dtype=np.float64)
        q[s], V[s], W[s], _, st[s] = solve(mesh, theta, dt, nsteps, v0=v0, w0=w0, model=model, rtol=rtol)
    return q, V, W, st


def activation_time(trace: np.ndarray, dt: float, u_th: float) -> float:
    """a(x0) = min{t in [0, T] : u(x0, t) >= u_th} (Sec. 2.4, activation
    map) for the trace u(x0, t_n), t_n = n dt, read as linear in time between
    the block ends; -1 if the threshold is never reached."""
    for n, u in enumerate(trace):
        if u >= u_th:
            if n == 0:
                return 0.0
            up = trace[n - 1]
            return dt * ((n - 1) + (u_th - up) / (u - up))
    return -1.0


def solve_points(mesh: Mesh, phi: np.ndarray, xi: np.ndarray, dt: float, nsteps: int, pts: np.ndarray,
                 u_th: float, v0=None, w0=None, theta_mean=None, model=None, rtol: float = 1e-13):
    """Point QoIs of Sec. 2.4 for S samples: the action potential u(x_p, t_n)
    (the P1 interpolant of v_h(t_n) at x_p) after every time block, n = 0..nsteps,
    and the activation time of each trace.  The blocks run one solve() call
    each from the state the last one left, so the arithmetic is that of
    solve().  Returns (trace[S, np, nsteps+1], act[S, np], Q[S], status[S])."""
    xi = np.atleast_2d(np.asarray(xi, dtype=np.float64))
    pts = np.atleast_2d(np.asarray(pts, dtype=np.float64))
    S, npts = xi.shape[0], pts.shape[0]
    trace = np.zeros((S, npts, nsteps + 1))
    act = np.zeros((S, npts))
    q = np.zeros(S)
    st = np.zeros(S, dtype=np.int32)
    if v0 is None:
        v0, w0 = initial_state(mesh)
    for s in range(S):
        theta = np.asarray(phi, dtype=np.float64) @ xi[s]
        if theta_mean is not None:
            theta = theta + np.asarray(theta_mean, dtype=np.float64)
        v = np.array(v0, dtype=np.float64)
        w = np.zeros(mesh.n) if w0 is None else np.array(w0, dtype=np.float64)
        trace[s, :, 0] = p1_at_points(mesh, v[:, None], pts)[:, 0]
        for n in range(1, nsteps + 1):
            q[s], v, w, _, sst = solve(mesh, theta, dt, 1, v0=v, w0=w, model=model, rtol=rtol)
            st[s] = max(st[s], sst)
            trace[s, :, n] = p1_at_points(mesh, v[:, None], pts)[:, 0]
        if nsteps == 0:
            q[s] = solve(mesh, theta, dt, 0, v0=v, w0=w, model=model, rtol=rtol)[0]
        for p in range(npts):
            act[s, p] = activation_time(trace[s, p], dt, u_th)
    return trace, act, q, st


def time_norms(e: np.ndarray, T: float):
    """L2(0, T) and H1(0, T) norms (eq. point-error, q = 0 and 1) of the
    function linear between the values e_n at t_n = n T / nt.  Each step's
    integral of e^2 by Simpson's rule (exact for the quadratic e^2 there), of
    e'^2 as the constant slope squared times the step."""
    e = np.asarray(e, dtype=np.float64)
    nt = e.size - 1
    dt = T / nt
    mid = 0.5 * (e[:-1] + e[1:])
    l2sq = float(np.sum(dt / 6.0 * (e[:-1] ** 2 + 4.0 * mid ** 2 + e[1:] ** 2)))
    h1sq = float(np.sum(((e[1:] - e[:-1]) / dt) ** 2 * dt))
    return np.sqrt(l2sq), np.sqrt(l2sq + h1sq)


# The paper's scheme: Crank-Nicolson (theta = 1/2) or backward Euler
# (theta = 1) slabs, the one-variable ionic current of eq. ionic_term on the
# new time level, the stimulus I_app of Sec. 5.1, Newton's method.
PAPER_MODEL = dict(s_l=1.0, s_t=0.2, alpha=1.4e-3, u_rest=0.0, u_th=28.0, u_peak=115.0, theta=0.5,
                   amp=115.0, sigma=0.1, t1=0.005, x0=(0.0, 0.0, 0.0))


def _paper_vec(pm):
    p = dict(PAPER_MODEL)
    p.update(pm or {})
    x0 = list(p["x0"]) + [0.0] * (3 - len(p["x0"]))
    return np.array([p["s_l"], p["s_t"], p["alpha"], p["u_rest"], p["u_th"], p["u_peak"], p["theta"], p["amp"],
                     p["sigma"], p["t1"], x0[0], x0[1], x0[2]], dtype=np.float64)


def solve_paper(mesh: Mesh, theta, dt: float, nsteps: int, u0=None, pm=None, rtol: float = 1e-13,
                maxit: int | None = None):
    """One sample of the paper's scheme (see mlq_oracle.c).  Returns (Q,
    u_final, Newton steps, status).  u0 defaults to u_rest everywhere."""
    lib = _load()
    p = _paper_vec(pm)
    u = np.full(mesh.n, p[3]) if u0 is None else np.array(u0, dtype=np.float64)
    q = ctypes.c_double()
    nw = ctypes.c_int64()
    st = ctypes.c_int32()
    maxit = 10 * mesh.n if maxit is None else maxit
    th = np.ascontiguousarray(theta, dtype=np.float64)
    assert lib.mlqo_solve_paper(mesh.dim, mesh.n, mesh.xyz, mesh.ne, mesh.conn, th, p, dt, nsteps, rtol, maxit, u,
                                ctypes.byref(q), ctypes.byref(nw), ctypes.byref(st)) == 0
    return q.value, u, nw.value, st.value


def solve_paper_batch(mesh: Mesh, phi: np.ndarray, xi: np.ndarray, dt: float, nsteps: int, u0=None, pm=None,
                      theta_mean=None, rtol: float = 1e-13):
    """S samples of the paper's scheme, theta_e = theta_mean_e + sum_k
    phi[e, k] xi[s, k] (eq. KLlowrank).  Returns (Q[S], u[S, n], status[S])."""
    xi = np.atleast_2d(np.asarray(xi, dtype=np.float64))
    S = xi.shape[0]
    q = np.zeros(S)
    U = np.zeros((S, mesh.n))
    st = np.zeros(S, dtype=np.int32)
    for s in range(S):
        th = np.asarray(phi, dtype=np.float64) @ xi[s]
        if theta_mean is not None:
            th = th + np.asarray(theta_mean, dtype=np.float64)
        q[s], U[s], _, st[s] = solve_paper(mesh, th, dt, nsteps, u0=u0, pm=pm, rtol=rtol)
    return q, U, st


def p1_at_points(mesh: Mesh, f: np.ndarray, pts: np.ndarray, return_location: bool = False):
    """Values at points (np x dim) of the P1 interpolants on `mesh` of the
    nodal fields f (n x K): the first simplex containing a point, else (a
    point outside the discretised domain) the first simplex whose smallest
    barycentric coordinate is within 1e-12 of the largest, extended
    linearly."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    if f.ndim == 1:
        f = f[:, None]
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    K = f.shape[1]
    out = np.zeros((pts.shape[0], K))
    el = np.zeros(pts.shape[0], dtype=np.int32)
    lm = np.zeros(pts.shape[0])
    assert _load().mlqo_p1_at_points(mesh.dim, mesh.n, mesh.xyz, mesh.ne, mesh.conn, K, f, pts.shape[0], pts, out,
                                     el.ctypes.data_as(ctypes.c_void_p), lm.ctypes.data_as(ctypes.c_void_p)) == 0
    return (out, el, lm) if return_location else out


def centroid_table_unrelated(fine: Mesh, modes_f: np.ndarray, coarse: Mesh) -> np.ndarray:
    """Phi[e, k] = fine P1 interpolant of mode k at the centroid of element e
    of an unrelated (non-nested) mesh: the intergrid transfer of Sec. 4 by
    point location."""
    cen = coarse.xyz[coarse.conn].mean(axis=1)
    return p1_at_points(fine, modes_f, cen)


# --------------------------------------------------------------------------
# estimators (Sec. 4)
# --------------------------------------------------------------------------
def mc_estimate(q: np.ndarray):
    """Plain Monte Carlo mean and its statistical RMSE sqrt(var/N)."""
    q = np.asarray(q, dtype=np.float64)
    n = q.size
    mean = float(np.sum(q) / n)
    var = float(np.sum((q - mean) ** 2) / (n - 1)) if n > 1 else 0.0
    return mean, var, (var / n) ** 0.5


def mlmc_estimate(y_levels):
    """eq. StandardML with MC rules: sum over levels of the sample mean of
    Y_l = F_l - F_{l-1} (F_{-1} = 0).  Returns (estimate, V_l list, RMSE_stat)
    with RMSE_stat = sqrt(sum_l V_l / N_l)."""
    est = 0.0
    var = []
    mse = 0.0
    for y in y_levels:
        m, v, _ = mc_estimate(y)
        est += m
        var.append(v)
        mse += v / np.asarray(y).size
    return est, var, mse ** 0.5


def pimped_ml_estimate(F_terms, N):
    """eq. PimpedML with nested sample rules: sum_{l=0}^L (Q_l - Q_{l-1})(F_{L-l}),
    Q_l the mean over the first N_l points (N_0 <= ... <= N_L), Q_{-1} = 0.
    F_terms[l] holds F_{L-l} (the QoI on mesh L-l) at the first N_l points.
    Each term needs one mesh only, so the meshes need not be nested."""
    est = 0.0
    for l, f in enumerate(F_terms):
        f = np.asarray(f, dtype=np.float64)
        assert f.size >= N[l]
        est += float(np.sum(f[:N[l]]) / N[l])
        if l > 0:
            est -= float(np.sum(f[:N[l - 1]]) / N[l - 1])
    return est


def qmc_estimate(q_by_shift: np.ndarray):
    """Randomly shifted lattice rule: rows = shifts, columns = points.  The
    estimate is the mean of the per-shift means; its RMSE the standard
    deviation of those means over sqrt(R)."""
    q = np.asarray(q_by_shift, dtype=np.float64)
    R = q.shape[0]
    means = q.mean(axis=1)
    est = float(means.mean())
    rmse = float(np.std(means, ddof=1) / np.sqrt(R)) if R > 1 else 0.0
    return est, rmse
