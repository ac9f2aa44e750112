"""Synthetic left-ventricle shell: meshes and rule-based fibres.

Input data of the non-nested multilevel configuration (a truncated prolate
ellipsoid shell, four unrelated tetrahedral meshes, helix fibres plus a KL
perturbation of the fibre angle; the paper's Sec. 5.4 runs the method on a
patient geometry with non-nested meshes and reconstructed fibres, which are
not available).  Like ``inputs``, this module holds none of the method's
arithmetic: it only produces node coordinates, tetrahedra and, per
tetrahedron, the orthonormal pair of wall-tangent directions and the mean
fibre angle that the fibre field is built from.

Geometry: prolate spheroidal coordinates with focal length d,
    x = d sinh(mu) sin(nu) cos(phi), y = d sinh(mu) sin(nu) sin(phi),
    z = d cosh(mu) cos(nu),
wall mu_endo <= mu <= mu_epi, truncated at the base plane z = 0 (nu = pi/2)
and closed at the apex (nu = pi, the axis).  The parameter box is cut into
n_mu x n_nu x n_phi cells (periodic in phi); cells between ring nu_j and ring
nu_{j+1} are split into six tetrahedra along the axis permutations (Kuhn
splitting; every face diagonal joins the cell corner of lowest to the corner
of highest index pair, so neighbouring cells agree on shared faces, also
across the seam phi = 0), and the cells of the last ring close on one axis
node per mu layer as wedges of three tetrahedra whose quadrilateral faces
take the same diagonals.

Fibres: per tetrahedron the circumferential unit vector e_c = d x / d phi and
the longitudinal unit vector e_l = d x / d nu (both tangent to the wall,
orthogonal) at the centroid, and the helix angle alpha(t) = 60 deg - 120 deg
t with t the transmural coordinate (0 endocardium, 1 epicardium); the fibre
of a sample is f = cos(alpha + theta) e_c + sin(alpha + theta) e_l with theta
the KL field.
"""
from __future__ import annotations

import math

import numpy as np

# unit-free proportions of a left ventricle: cavity height / base radius ~ 1.7,
# wall thickness ~ 0.4 of the base radius at the equator
FOCAL = 1.0
MU_ENDO = 0.55
MU_EPI = 0.85
NU_BASE = 0.5 * math.pi

# four unrelated resolutions (n_mu, n_nu, n_phi): ~20k, 80k, 320k, 1.3M nodes
LEVELS = [(4, 40, 100), (7, 62, 160), (12, 100, 250), (19, 160, 400)]

_KUHN = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))


def _point(mu, nu, phi, d):
    s = d * np.sinh(mu) * np.sin(nu)
    return np.stack([s * np.cos(phi), s * np.sin(phi), d * np.cosh(mu) * np.cos(nu)], axis=-1)


def shell_volume(mu0: float = MU_ENDO, mu1: float = MU_EPI, d: float = FOCAL) -> float:
    """Exact volume of the truncated shell: the half spheroid below z = 0 has
    volume (2/3) pi d^3 sinh(mu)^2 cosh(mu)."""
    half = lambda mu: 2.0 / 3.0 * math.pi * d ** 3 * math.sinh(mu) ** 2 * math.cosh(mu)
    return half(mu1) - half(mu0)


def lv_mesh(n_mu: int, n_nu: int, n_phi: int, d: float = FOCAL, mu_endo: float = MU_ENDO, mu_epi: float = MU_EPI):
    """Nodes (n x 3) and positively oriented tetrahedra (n_e x 4, int32).
    Ring node (i, j, k) (mu_i, nu_j, phi_k; j < n_nu) has index
    k + n_phi (j + n_nu i); the axis node of layer i has index
    (n_mu + 1) n_nu n_phi + i."""
    if n_mu < 1 or n_nu < 2 or n_phi < 3:
        raise ValueError("lv_mesh needs n_mu >= 1, n_nu >= 2, n_phi >= 3")
    mu = mu_endo + (mu_epi - mu_endo) * np.arange(n_mu + 1) / n_mu
    nu = NU_BASE + (math.pi - NU_BASE) * np.arange(n_nu) / n_nu   # ring n_nu would be the axis
    phi = 2.0 * math.pi * np.arange(n_phi) / n_phi
    M, N, P = np.meshgrid(mu, nu, phi, indexing="ij")
    ring = _point(M, N, P, d).reshape(-1, 3)
    axis = np.stack([np.zeros(n_mu + 1), np.zeros(n_mu + 1), d * np.cosh(mu) * math.cos(math.pi)], axis=-1)
    xyz = np.ascontiguousarray(np.concatenate([ring, axis]), dtype=np.float64)

    def rid(i, j, k):
        return (k % n_phi) + n_phi * (j + n_nu * i)

    aid = lambda i: (n_mu + 1) * n_nu * n_phi + i
    # Kuhn tetrahedra of the cells between rings j and j + 1
    i, j, k = np.meshgrid(np.arange(n_mu), np.arange(n_nu - 1), np.arange(n_phi), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    tets = []
    for perm in _KUHN:
        c = [np.zeros_like(i), np.zeros_like(i), np.zeros_like(i)]
        verts = [rid(i, j, k)]
        for ax in perm:
            c[ax] = c[ax] + 1
            verts.append(rid(i + c[0], j + c[1], k + c[2]))
        tets.append(np.stack(verts, axis=-1))
    # wedges between the last ring and the axis: a, b on layer i, a', b' on
    # layer i + 1 (phi_k, phi_k+1), c, c' the axis nodes; the quadrilateral
    # faces take the diagonals a-b', a-c', b-c'
    i, k = np.meshgrid(np.arange(n_mu), np.arange(n_phi), indexing="ij")
    i, k = i.ravel(), k.ravel()
    jl = n_nu - 1
    a, b = rid(i, jl, k), rid(i, jl, k + 1)
    a1, b1 = rid(i + 1, jl, k), rid(i + 1, jl, k + 1)
    c, c1 = aid(i), aid(i + 1)
    tets += [np.stack([a, b, c, c1], axis=-1), np.stack([a, b, b1, c1], axis=-1),
             np.stack([a, a1, b1, c1], axis=-1)]
    conn = np.concatenate([t.reshape(-1, 4) for t in tets]).astype(np.int32)
    # orientation: swap two vertices where the signed volume is negative
    X = xyz[conn]
    vol = np.einsum("ij,ij->i", np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]), X[:, 3] - X[:, 0])
    neg = vol < 0
    conn[neg, 2], conn[neg, 3] = conn[neg, 3].copy(), conn[neg, 2].copy()
    return xyz, np.ascontiguousarray(conn)


def prolate_coordinates(p: np.ndarray, d: float = FOCAL):
    """(mu, nu, phi) of Cartesian points p (n x 3): cosh mu = (r1 + r2) / 2d,
    cos nu = (r2 - r1) / 2d with r1, r2 the distances to the foci (0, 0, +-d)."""
    r1 = np.linalg.norm(p - np.array([0.0, 0.0, d]), axis=1)
    r2 = np.linalg.norm(p + np.array([0.0, 0.0, d]), axis=1)
    mu = np.arccosh(np.maximum((r1 + r2) / (2.0 * d), 1.0))
    nu = np.arccos(np.clip((r2 - r1) / (2.0 * d), -1.0, 1.0))
    phi = np.arctan2(p[:, 1], p[:, 0])
    return mu, nu, phi


def lv_fibres(xyz: np.ndarray, conn: np.ndarray, d: float = FOCAL, mu_endo: float = MU_ENDO,
              mu_epi: float = MU_EPI):
    """Per tetrahedron: frames (n_e x 6: e_c then e_l) and the helix angle
    alpha (n_e), evaluated at the centroid."""
    cen = xyz[conn].mean(axis=1)
    mu, nu, phi = prolate_coordinates(cen, d)
    e_c = np.stack([-np.sin(phi), np.cos(phi), np.zeros_like(phi)], axis=-1)
    e_l = np.stack([np.sinh(mu) * np.cos(nu) * np.cos(phi), np.sinh(mu) * np.cos(nu) * np.sin(phi),
                    -np.cosh(mu) * np.sin(nu)], axis=-1)
    e_l /= np.linalg.norm(e_l, axis=1, keepdims=True)
    t = np.clip((mu - mu_endo) / (mu_epi - mu_endo), 0.0, 1.0)
    alpha = np.deg2rad(60.0 - 120.0 * t)
    return np.ascontiguousarray(np.concatenate([e_c, e_l], axis=1)), np.ascontiguousarray(alpha)


def lv_level(level: int):
    """(xyz, conn, frames, alpha) of one of the four preset resolutions."""
    xyz, conn = lv_mesh(*LEVELS[level])
    frames, alpha = lv_fibres(xyz, conn)
    return xyz, conn, frames, alpha


def stimulus(xyz: np.ndarray, radius: float = 0.25, d: float = FOCAL, mu_endo: float = MU_ENDO):
    """Initial state: v = 1 within `radius` of the endocardial apex
    (0, 0, -d cosh mu_endo), else 0; w = 0."""
    apex = np.array([0.0, 0.0, -d * math.cosh(mu_endo)])
    v = np.where(np.linalg.norm(xyz - apex, axis=1) <= radius, 1.0, 0.0)
    return v, np.zeros(xyz.shape[0])
