/*
 * mlq_oracle.c -- TEST INFRASTRUCTURE, not product code.
 *
 * A plain, slow, FP64 CPU implementation of the per-sample forward solve of
 * the stochastic monodomain equation (Ben Bader, Harbrecht, Krause, Multerer,
 * Quaglino, Schmidlin, "Space-time multilevel quadrature methods and their
 * application for cardiac electrophysiology", arXiv 2105.02007).  Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg and
 * reference arm may load this library.  It shares no code, header or table with the CUDA path.
 *
 * Every step follows the paper's definitions directly:
 *   - P1 Lagrange spaces on nested simplicial meshes            (Sec. 3.1)
 *   - mass / stiffness matrices M_l, K_l                        (Sec. 3.1, eq. semi-disc)
 *   - conductivity G = g I + (|V| - g) V V^T / V^T V,           (Sec. 2.1, eq. AdmV)
 *     here written D = s_t I + (s_l - s_t) f f^T, f = unit fiber
 *   - reaction r(u) = dt M I_ion(u)  (nodal current times      (Sec. 3.2, eq. mono_disc)
 *     consistent mass)
 *   - time blocks solved one after another, each block's        (Sec. 3.3, multiple time blocks)
 *     initial value being the previous block's end state; here
 *     one backward-Euler step per block with the reaction taken
 *     explicitly, so each block is an SPD solve
 *   - KL expansion by pivoted Cholesky + reduced eigenproblem   (Sec. 2.3, eqs. approxEig, redEig)
 *   - fine-to-coarse transfer of the field by the midpoint rule (Sec. 4, intergrid transfer)
 *   - the same transfer between unrelated meshes: P1 values   (Sec. 4; non-nested meshes,
 *     at the other mesh's centroids by point location           Sec. 5.4)
 *   - fibres turning in the plane of a per-element frame       (eq. AdmV with a general
 *     (e.g. the wall-tangent pair of a ventricle shell)          fibre direction)
 *
 * Storage is CSR with an explicit pattern; the linear solver is textbook
 * Jacobi-preconditioned CG.  Nothing is blocked, fused or reordered.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MLQO_OK 0
#define MLQO_EINVAL -1
#define MLQO_ENOMEM -2

/* per-sample solver status codes */
#define MLQO_S_CONVERGED 0
#define MLQO_S_MAXITER 1
#define MLQO_S_NONFINITE 2

/* ------------------------------------------------------------------------ */
/* Meshes (Sec. 3.1: nested shape-regular simplicial meshes, h_l ~ 2^-l).    */
/* ------------------------------------------------------------------------ */

/* Structured triangulation of the unit square on m x m nodes.
 * Node (i,j) has index i + m*j and sits at (i/(m-1), j/(m-1)).
 * Square (i,j) is split along its (1,1) diagonal into
 *   element 2*(i+(m-1)*j)+0 : (i,j) (i+1,j) (i+1,j+1)
 *   element 2*(i+(m-1)*j)+1 : (i,j) (i+1,j+1) (i,j+1)
 * Red refinement of this mesh gives the mesh on 2m-1 nodes, so the levels
 * are nested. */
int mlqo_mesh2d(int m, double *xy, int32_t *conn)
{
    if (m < 2) return MLQO_EINVAL;
    for (int j = 0; j < m; ++j)
        for (int i = 0; i < m; ++i) {
            int64_t v = i + (int64_t)m * j;
            xy[2 * v + 0] = (double)i / (double)(m - 1);
            xy[2 * v + 1] = (double)j / (double)(m - 1);
        }
    for (int j = 0; j + 1 < m; ++j)
        for (int i = 0; i + 1 < m; ++i) {
            int64_t c = i + (int64_t)(m - 1) * j;
            int32_t n00 = i + m * j, n10 = n00 + 1, n01 = n00 + m, n11 = n00 + m + 1;
            int32_t *t0 = conn + 6 * c, *t1 = t0 + 3;
            t0[0] = n00; t0[1] = n10; t0[2] = n11;
            t1[0] = n00; t1[1] = n11; t1[2] = n01;
        }
    return MLQO_OK;
}

/* Structured Kuhn (Freudenthal) tetrahedralisation of the box
 * [0,Lx]x[0,Ly]x[0,Lz] on mx*my*mz nodes.  Node (i,j,k) has index
 * i + mx*(j + my*k).  Cube c = i + (mx-1)*(j + (my-1)*k) is split into the six
 * tetrahedra 6c+s, s = 0..5, whose vertices walk from the cube's lowest corner
 * to its highest one along the unit steps e_{a}, e_{b}, e_{c} taken in the
 * axis order of permutation s of the list
 *   (0,1,2) (0,2,1) (1,0,2) (1,2,0) (2,0,1) (2,1,0).
 * Regular refinement of this mesh gives the mesh with halved spacing. */
static const int kuhn_perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

int mlqo_mesh3d(int mx, int my, int mz, double Lx, double Ly, double Lz, double *xyz, int32_t *conn)
{
    if (mx < 2 || my < 2 || mz < 2) return MLQO_EINVAL;
    for (int k = 0; k < mz; ++k)
        for (int j = 0; j < my; ++j)
            for (int i = 0; i < mx; ++i) {
                int64_t v = i + (int64_t)mx * (j + (int64_t)my * k);
                xyz[3 * v + 0] = Lx * (double)i / (double)(mx - 1);
                xyz[3 * v + 1] = Ly * (double)j / (double)(my - 1);
                xyz[3 * v + 2] = Lz * (double)k / (double)(mz - 1);
            }
    for (int k = 0; k + 1 < mz; ++k)
        for (int j = 0; j + 1 < my; ++j)
            for (int i = 0; i + 1 < mx; ++i) {
                int64_t c = i + (int64_t)(mx - 1) * (j + (int64_t)(my - 1) * k);
                for (int s = 0; s < 6; ++s) {
                    int idx[3] = {i, j, k};
                    int32_t *t = conn + 4 * (6 * c + s);
                    t[0] = (int32_t)(idx[0] + mx * (idx[1] + my * idx[2]));
                    for (int q = 0; q < 3; ++q) {
                        idx[kuhn_perm[s][q]] += 1;
                        t[q + 1] = (int32_t)(idx[0] + mx * (idx[1] + my * idx[2]));
                    }
                }
            }
    return MLQO_OK;
}

/* ------------------------------------------------------------------------ */
/* Element matrices (Sec. 3.1: M = [int phi_j phi_i], K = [int G grad phi_j . */
/* grad phi_i]) for P1 on a simplex, and the conductivity of eq. AdmV.       */
/* ------------------------------------------------------------------------ */

/* Barycentric-coordinate gradients of a simplex with vertices X[0..d]
 * (row-major, d coordinates each).  g[a*d + c] = d lambda_a / d x_c.
 * Returns the simplex volume |e|. */
static double simplex_gradients(int d, const double *X, double *g)
{
    double J[9], Ji[9];
    for (int r = 0; r < d; ++r)       /* J[r][c] = X[c+1][r] - X[0][r] */
        for (int c = 0; c < d; ++c) J[r * d + c] = X[(c + 1) * d + r] - X[r];
    double det;
    if (d == 2) {
        det = J[0] * J[3] - J[1] * J[2];
        Ji[0] = J[3] / det; Ji[1] = -J[1] / det;
        Ji[2] = -J[2] / det; Ji[3] = J[0] / det;
    } else {
        det = J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
              J[2] * (J[3] * J[7] - J[4] * J[6]);
        Ji[0] = (J[4] * J[8] - J[5] * J[7]) / det;
        Ji[1] = (J[2] * J[7] - J[1] * J[8]) / det;
        Ji[2] = (J[1] * J[5] - J[2] * J[4]) / det;
        Ji[3] = (J[5] * J[6] - J[3] * J[8]) / det;
        Ji[4] = (J[0] * J[8] - J[2] * J[6]) / det;
        Ji[5] = (J[2] * J[3] - J[0] * J[5]) / det;
        Ji[6] = (J[3] * J[7] - J[4] * J[6]) / det;
        Ji[7] = (J[1] * J[6] - J[0] * J[7]) / det;
        Ji[8] = (J[0] * J[4] - J[1] * J[3]) / det;
    }
    /* lambda_a for a >= 1 is row (a-1) of J^{-1} applied to (x - X0):
     * grad lambda_a = row (a-1) of J^{-1}.  lambda_0 = 1 - sum. */
    for (int c = 0; c < d; ++c) {
        double s = 0.0;
        for (int a = 1; a <= d; ++a) {
            g[a * d + c] = Ji[(a - 1) * d + c];
            s += Ji[(a - 1) * d + c];
        }
        g[c] = -s;
    }
    double vol = fabs(det);
    return d == 2 ? vol / 2.0 : vol / 6.0;
}

/* D = s_t I + (s_l - s_t) f f^T: eq. AdmV with g = s_t and |V| = s_l.  The
 * unit fibre f = cos(th) e1 + sin(th) e2 turns by th in the plane of an
 * orthonormal pair (e1, e2) given per element (frame = e1 then e2, 6 values;
 * NULL: the x-y plane, f = (cos th, sin th[, 0])). */
static void conductivity(int d, double th, const double *frame, double s_l, double s_t, double *D)
{
    double f[3] = {cos(th), sin(th), 0.0};
    if (frame) {
        const double c = cos(th), s = sin(th);
        for (int r = 0; r < 3; ++r) f[r] = c * frame[r] + s * frame[3 + r];
    }
    for (int r = 0; r < d; ++r)
        for (int c = 0; c < d; ++c) D[r * d + c] = (r == c ? s_t : 0.0) + (s_l - s_t) * f[r] * f[c];
}

/* P1 element stiffness K_e[a][b] = |e| grad lambda_a^T D grad lambda_b and
 * consistent mass M_e[a][b] = |e| (1 + delta_ab) / ((d+1)(d+2)). */
static void element_matrices(int d, const double *X, const double *D, double *Ke, double *Me)
{
    double g[12];
    double vol = simplex_gradients(d, X, g);
    int nv = d + 1;
    double mscale = vol / (double)((d + 1) * (d + 2));
    for (int a = 0; a < nv; ++a)
        for (int b = 0; b < nv; ++b) {
            double s = 0.0;
            for (int r = 0; r < d; ++r)
                for (int c = 0; c < d; ++c) s += g[a * d + r] * D[r * d + c] * g[b * d + c];
            Ke[a * nv + b] = vol * s;
            Me[a * nv + b] = mscale * (a == b ? 2.0 : 1.0);
        }
}

/* ------------------------------------------------------------------------ */
/* CSR pattern and assembly.                                                 */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t n, nnz;
    int64_t *rp;
    int32_t *ci;
} pattern_t;

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Sparsity of the P1 matrices: (i,j) is present iff i and j share an element. */
static int build_pattern(int d, int64_t n, int64_t ne, const int32_t *conn, pattern_t *P)
{
    int nv = d + 1;
    int64_t *cnt = calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt) return MLQO_ENOMEM;
    for (int64_t e = 0; e < ne; ++e)
        for (int a = 0; a < nv; ++a) cnt[conn[e * nv + a] + 1] += nv;
    for (int64_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
    int32_t *raw = malloc(sizeof(int32_t) * (size_t)cnt[n]);
    int64_t *fill = malloc(sizeof(int64_t) * (size_t)n);
    if (!raw || !fill) { free(cnt); free(raw); free(fill); return MLQO_ENOMEM; }
    for (int64_t i = 0; i < n; ++i) fill[i] = cnt[i];
    for (int64_t e = 0; e < ne; ++e)
        for (int a = 0; a < nv; ++a) {
            int32_t i = conn[e * nv + a];
            for (int b = 0; b < nv; ++b) raw[fill[i]++] = conn[e * nv + b];
        }
    P->n = n;
    P->rp = malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!P->rp) { free(cnt); free(raw); free(fill); return MLQO_ENOMEM; }
    int64_t nnz = 0;
    P->rp[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int32_t *row = raw + cnt[i];
        int64_t len = cnt[i + 1] - cnt[i];
        qsort(row, (size_t)len, sizeof(int32_t), cmp_i32);
        int64_t u = 0;
        for (int64_t t = 0; t < len; ++t)
            if (t == 0 || row[t] != row[t - 1]) row[u++] = row[t];
        nnz += u;
        fill[i] = u;
    }
    P->ci = malloc(sizeof(int32_t) * (size_t)nnz);
    if (!P->ci) { free(cnt); free(raw); free(fill); free(P->rp); return MLQO_ENOMEM; }
    int64_t pos = 0;
    for (int64_t i = 0; i < n; ++i) {
        memcpy(P->ci + pos, raw + cnt[i], sizeof(int32_t) * (size_t)fill[i]);
        pos += fill[i];
        P->rp[i + 1] = pos;
    }
    P->nnz = nnz;
    free(cnt); free(raw); free(fill);
    return MLQO_OK;
}

static void free_pattern(pattern_t *P)
{
    free(P->rp); free(P->ci);
    P->rp = NULL; P->ci = NULL;
}

static int64_t find_col(const pattern_t *P, int64_t i, int32_t j)
{
    int64_t lo = P->rp[i], hi = P->rp[i + 1] - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (P->ci[mid] == j) return mid;
        if (P->ci[mid] < j) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* Assemble M and K(theta) (theta per element; NULL means theta = 0) into the
 * pattern's value arrays. */
static void assemble(int d, const double *xyz, int64_t ne, const int32_t *conn, const double *theta,
                     const double *frames, double s_l, double s_t, const pattern_t *P, double *mval, double *kval)
{
    int nv = d + 1;
    if (mval) memset(mval, 0, sizeof(double) * (size_t)P->nnz);
    if (kval) memset(kval, 0, sizeof(double) * (size_t)P->nnz);
    for (int64_t e = 0; e < ne; ++e) {
        double X[12], D[9], Ke[16], Me[16];
        for (int a = 0; a < nv; ++a)
            for (int c = 0; c < d; ++c) X[a * d + c] = xyz[(int64_t)conn[e * nv + a] * d + c];
        conductivity(d, theta ? theta[e] : 0.0, frames ? frames + e * 6 : NULL, s_l, s_t, D);
        element_matrices(d, X, D, Ke, Me);
        for (int a = 0; a < nv; ++a)
            for (int b = 0; b < nv; ++b) {
                int64_t k = find_col(P, conn[e * nv + a], conn[e * nv + b]);
                if (mval) mval[k] += Me[a * nv + b];
                if (kval) kval[k] += Ke[a * nv + b];
            }
    }
}

/* Public: number of nonzeros of the P1 pattern. */
int64_t mlqo_pattern_nnz(int d, int64_t n, int64_t ne, const int32_t *conn)
{
    pattern_t P;
    if (build_pattern(d, n, ne, conn, &P) != MLQO_OK) return -1;
    int64_t nnz = P.nnz;
    free_pattern(&P);
    return nnz;
}

/* Public: CSR of M and K(theta) with fibre frames (NULL: the x-y plane).
 * rp has n+1 entries, ci/mval/kval nnz. */
int mlqo_assemble_f(int d, int64_t n, const double *xyz, int64_t ne, const int32_t *conn, const double *theta,
                    const double *frames, double s_l, double s_t, int64_t *rp, int32_t *ci, double *mval,
                    double *kval)
{
    pattern_t P;
    int st = build_pattern(d, n, ne, conn, &P);
    if (st != MLQO_OK) return st;
    assemble(d, xyz, ne, conn, theta, frames, s_l, s_t, &P, mval, kval);
    memcpy(rp, P.rp, sizeof(int64_t) * (size_t)(n + 1));
    memcpy(ci, P.ci, sizeof(int32_t) * (size_t)P.nnz);
    free_pattern(&P);
    return MLQO_OK;
}

/* Public: CSR of M and K(theta), fibres in the x-y plane. */
int mlqo_assemble(int d, int64_t n, const double *xyz, int64_t ne, const int32_t *conn, const double *theta,
                  double s_l, double s_t, int64_t *rp, int32_t *ci, double *mval, double *kval)
{
    return mlqo_assemble_f(d, n, xyz, ne, conn, theta, NULL, s_l, s_t, rp, ci, mval, kval);
}

/* ------------------------------------------------------------------------ */
/* Transfer between unrelated meshes (Sec. 4, intergrid transfer; non-nested */
/* levels of Sec. 5.4): the P1 interpolant of nodal fields at points.        */
/* ------------------------------------------------------------------------ */

/* Barycentric coordinates of point x in simplex e (d+1 values). */
static void barycentric(int d, const double *xyz, const int32_t *conn, int64_t e, const double *x, double *lam)
{
    int nv = d + 1;
    double X0[3], A[9];
    for (int c = 0; c < d; ++c) X0[c] = xyz[(int64_t)conn[e * nv] * d + c];
    /* columns of A: X_a - X_0, a = 1..d */
    for (int a = 1; a <= d; ++a)
        for (int c = 0; c < d; ++c) A[c * d + (a - 1)] = xyz[(int64_t)conn[e * nv + a] * d + c] - X0[c];
    double r[3];
    for (int c = 0; c < d; ++c) r[c] = x[c] - X0[c];
    /* solve A l = r by Cramer's rule */
    double det, l[3];
    if (d == 2) {
        det = A[0] * A[3] - A[1] * A[2];
        l[0] = (r[0] * A[3] - A[1] * r[1]) / det;
        l[1] = (A[0] * r[1] - r[0] * A[2]) / det;
    } else {
        det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) + A[2] * (A[3] * A[7] - A[4] * A[6]);
        for (int col = 0; col < 3; ++col) {
            double B[9];
            memcpy(B, A, sizeof(B));
            for (int c = 0; c < 3; ++c) B[c * 3 + col] = r[c];
            l[col] = (B[0] * (B[4] * B[8] - B[5] * B[7]) - B[1] * (B[3] * B[8] - B[5] * B[6]) +
                      B[2] * (B[3] * B[7] - B[4] * B[6])) / det;
        }
    }
    double s = 0.0;
    for (int a = 0; a < d; ++a) { lam[a + 1] = l[a]; s += l[a]; }
    lam[0] = 1.0 - s;
}

/* Public: out[p, k] = sum_a lambda_a f[node_a, k] for the simplex that
 * contains point p (the first in element order when p lies on a shared
 * face).  A point in no simplex (a centroid of another mesh of a curved
 * domain that falls outside this discretisation) takes, over all simplices,
 * the first (in element order) whose smallest barycentric coordinate is
 * within 1e-12 of the largest, and the linear extension of its P1 function.
 * Containing simplices are found through a uniform grid of buckets over the
 * node bounding box, each bucket listing (in element order) the simplices
 * whose bounding box meets it: a simplex that contains p is listed in p's
 * bucket.  elem_out / lam_min_out (may be NULL): the simplex used and its
 * smallest barycentric coordinate. */
int mlqo_p1_at_points(int d, int64_t n, const double *xyz, int64_t ne, const int32_t *conn, int K, const double *f,
                      int64_t np, const double *pts, double *out, int32_t *elem_out, double *lam_min_out)
{
    if ((d != 2 && d != 3) || n < 1 || ne < 1 || K < 0) return MLQO_EINVAL;
    int nv = d + 1;
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int c = 0; c < d; ++c) lo[c] = hi[c] = xyz[c];
    for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c < d; ++c) {
            double v = xyz[i * d + c];
            if (v < lo[c]) lo[c] = v;
            if (v > hi[c]) hi[c] = v;
        }
    int nb = (int)ceil(pow((double)ne / 4.0, 1.0 / d));
    if (nb < 1) nb = 1;
    if (nb > 1024) nb = 1024;
    double w[3] = {1.0, 1.0, 1.0};
    for (int c = 0; c < d; ++c) w[c] = (hi[c] - lo[c]) / nb > 0 ? (hi[c] - lo[c]) / nb : 1.0;
    int64_t nbuck = 1;
    for (int c = 0; c < d; ++c) nbuck *= nb;
    int64_t *cnt = calloc((size_t)nbuck + 1, sizeof(int64_t));
    if (!cnt) return MLQO_ENOMEM;
    int32_t *list = NULL;
    int64_t *fillp = NULL;
    /* two passes: count, then fill (element order within each bucket) */
    for (int pass = 0; pass < 2; ++pass) {
        for (int64_t e = 0; e < ne; ++e) {
            int ib[3][2] = {{0, 0}, {0, 0}, {0, 0}};
            for (int c = 0; c < d; ++c) {
                double a = xyz[(int64_t)conn[e * nv] * d + c], b = a;
                for (int q = 1; q < nv; ++q) {
                    double v = xyz[(int64_t)conn[e * nv + q] * d + c];
                    if (v < a) a = v;
                    if (v > b) b = v;
                }
                int i0 = (int)floor((a - lo[c]) / w[c]), i1 = (int)floor((b - lo[c]) / w[c]);
                ib[c][0] = i0 < 0 ? 0 : (i0 >= nb ? nb - 1 : i0);
                ib[c][1] = i1 < 0 ? 0 : (i1 >= nb ? nb - 1 : i1);
            }
            for (int kz = ib[2][0]; kz <= ib[2][1]; ++kz)
                for (int ky = ib[1][0]; ky <= ib[1][1]; ++ky)
                    for (int kx = ib[0][0]; kx <= ib[0][1]; ++kx) {
                        int64_t bkt = kx + (int64_t)nb * (ky + (int64_t)nb * kz);
                        if (pass == 0) cnt[bkt + 1]++;
                        else list[fillp[bkt]++] = (int32_t)e;
                    }
        }
        if (pass == 0) {
            for (int64_t b = 0; b < nbuck; ++b) cnt[b + 1] += cnt[b];
            list = malloc(sizeof(int32_t) * (size_t)(cnt[nbuck] > 0 ? cnt[nbuck] : 1));
            fillp = malloc(sizeof(int64_t) * (size_t)nbuck);
            if (!list || !fillp) { free(cnt); free(list); free(fillp); return MLQO_ENOMEM; }
            for (int64_t b = 0; b < nbuck; ++b) fillp[b] = cnt[b];
        }
    }
    free(fillp);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 256)
#endif
    for (int64_t p = 0; p < np; ++p) {
        const double *x = pts + p * d;
        int64_t home = 0, stride = 1;
        for (int c = 0; c < d; ++c) {
            int i = (int)floor((x[c] - lo[c]) / w[c]);
            i = i < 0 ? 0 : (i >= nb ? nb - 1 : i);
            home += i * stride;
            stride *= nb;
        }
        int64_t best = -1;
        double best_min = -INFINITY, best_lam[4] = {0, 0, 0, 0}, lam[4];
        for (int64_t t = cnt[home]; t < cnt[home + 1]; ++t) {
            int64_t e = list[t];
            barycentric(d, xyz, conn, e, x, lam);
            double mn = lam[0];
            for (int a = 1; a < nv; ++a) if (lam[a] < mn) mn = lam[a];
            if (mn >= -1e-12) {
                best = e;
                best_min = mn;
                memcpy(best_lam, lam, sizeof(lam));
                break;
            }
        }
        if (best < 0) {
            /* in no simplex: over all of them the largest smallest coordinate,
             * then the first simplex within 1e-12 of it (near-ties, e.g. beyond
             * a boundary vertex shared by several simplices, go to the lowest
             * index whatever the rounding) */
            for (int64_t e = 0; e < ne; ++e) {
                barycentric(d, xyz, conn, e, x, lam);
                double mn = lam[0];
                for (int a = 1; a < nv; ++a) if (lam[a] < mn) mn = lam[a];
                if (mn > best_min) best_min = mn;
            }
            for (int64_t e = 0; e < ne; ++e) {
                barycentric(d, xyz, conn, e, x, lam);
                double mn = lam[0];
                for (int a = 1; a < nv; ++a) if (lam[a] < mn) mn = lam[a];
                if (mn >= best_min - 1e-12) {
                    best = e;
                    best_min = mn;
                    memcpy(best_lam, lam, sizeof(lam));
                    break;
                }
            }
        }
        if (elem_out) elem_out[p] = (int32_t)best;
        if (lam_min_out) lam_min_out[p] = best_min;
        for (int k = 0; k < K; ++k) {
            double v = 0.0;
            for (int a = 0; a < nv; ++a) v += best_lam[a] * f[(int64_t)conn[best * nv + a] * K + k];
            out[p * K + k] = v;
        }
    }
    free(cnt);
    free(list);
    return MLQO_OK;
}

/* ------------------------------------------------------------------------ */
/* Karhunen-Loeve expansion (Sec. 2.2-2.3).                                  */
/* ------------------------------------------------------------------------ */

/* Scalar covariance c(x,y) = sigma2 * exp(-|x-y|^2 / ell), the paper's
 * kernel theta^2 exp(-|x-x'|^2 / sigma_KL) (Sec. 5.1). */
static double cov(int d, const double *x, const double *y, double sigma2, double ell)
{
    double r2 = 0.0;
    for (int c = 0; c < d; ++c) r2 += (x[c] - y[c]) * (x[c] - y[c]);
    return sigma2 * exp(-r2 / ell);
}

/* Cyclic Jacobi eigenvalue iteration for a symmetric K x K matrix A
 * (row-major, destroyed).  On return lam[k] are the eigenvalues and column k
 * of V (row-major V[r*K+k]) the matching orthonormal eigenvector.
 * Golub & Van Loan, Matrix Computations, Sec. 8.5 (cyclic Jacobi). */
static void jacobi_eigen(int K, double *A, double *lam, double *V)
{
    for (int r = 0; r < K; ++r)
        for (int c = 0; c < K; ++c) V[r * K + c] = (r == c) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int r = 0; r < K; ++r)
            for (int c = 0; c < K; ++c) {
                tot += A[r * K + c] * A[r * K + c];
                if (r != c) off += A[r * K + c] * A[r * K + c];
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < K - 1; ++p)
            for (int q = p + 1; q < K; ++q) {
                double apq = A[p * K + q];
                if (apq == 0.0) continue;
                double app = A[p * K + p], aqq = A[q * K + q];
                /* symmetric Schur 2x2: choose (c,s) zeroing A[p][q] */
                double tau = (aqq - app) / (2.0 * apq);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                /* A <- J^T A J with J the rotation in the (p,q) plane */
                for (int k = 0; k < K; ++k) {
                    double akp = A[k * K + p], akq = A[k * K + q];
                    A[k * K + p] = c * akp - s * akq;
                    A[k * K + q] = s * akp + c * akq;
                }
                for (int k = 0; k < K; ++k) {
                    double apk = A[p * K + k], aqk = A[q * K + k];
                    A[p * K + k] = c * apk - s * aqk;
                    A[q * K + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < K; ++k) {
                    double vkp = V[k * K + p], vkq = V[k * K + q];
                    V[k * K + p] = c * vkp - s * vkq;
                    V[k * K + q] = s * vkp + c * vkq;
                }
            }
    }
    for (int k = 0; k < K; ++k) lam[k] = A[k * K + k];
}

/* KL modes of the scalar field with covariance c = sigma2 exp(-|x-y|^2/ell)
 * on a P1 mesh (eq. algEig with d = 1 block):
 *   1. C ~ L L^T by K steps of pivoted Cholesky, entries of C computed on the
 *      fly; pivot = largest remaining diagonal, ties -> lowest node index
 *      (eq. approxEig and the Remark after it);
 *   2. reduced problem L^T M L vt = lambda vt, M the consistent mass matrix
 *      (eq. redEig), solved by cyclic Jacobi, eigenvalues sorted descending;
 *   3. v_k = L vt_k, so that v_i^T M v_j = lambda_i delta_ij;
 *   4. sign: the entry of largest magnitude of v_k is positive (ties ->
 *      lowest index).
 * modes[i*K+k] = v_k(x_i); lambda[k]; Lout (optional) = the factor L, n x K.
 * pivots (optional) = the K pivot nodes. */
int mlqo_kl_build(int d, int64_t n, const double *xyz, int64_t ne, const int32_t *conn, double sigma2,
                  double ell, int K, double *modes, double *lambda, double *Lout, int64_t *pivots)
{
    if (K < 1 || K > n) return MLQO_EINVAL;
    double *L = calloc((size_t)n * K, sizeof(double));
    double *diag = malloc(sizeof(double) * (size_t)n);
    if (!L || !diag) { free(L); free(diag); return MLQO_ENOMEM; }
    for (int64_t i = 0; i < n; ++i) diag[i] = cov(d, xyz + i * d, xyz + i * d, sigma2, ell);
    for (int k = 0; k < K; ++k) {
        int64_t p = 0;
        for (int64_t i = 1; i < n; ++i)
            if (diag[i] > diag[p]) p = i;
        if (pivots) pivots[k] = p;
        double piv = sqrt(diag[p]);
        for (int64_t i = 0; i < n; ++i) {
            double s = cov(d, xyz + i * d, xyz + p * d, sigma2, ell);
            for (int j = 0; j < k; ++j) s -= L[i * K + j] * L[p * K + j];
            L[i * K + k] = s / piv;
        }
        for (int64_t i = 0; i < n; ++i) diag[i] -= L[i * K + k] * L[i * K + k];
    }
    free(diag);

    /* B = L^T M L */
    pattern_t P;
    int st = build_pattern(d, n, ne, conn, &P);
    if (st != MLQO_OK) { free(L); return st; }
    double *mval = malloc(sizeof(double) * (size_t)P.nnz);
    double *ML = calloc((size_t)n * K, sizeof(double));
    double *B = calloc((size_t)K * K, sizeof(double));
    double *lam = malloc(sizeof(double) * K), *V = malloc(sizeof(double) * K * K);
    if (!mval || !ML || !B || !lam || !V) {
        free(L); free(mval); free(ML); free(B); free(lam); free(V); free_pattern(&P);
        return MLQO_ENOMEM;
    }
    assemble(d, xyz, ne, conn, NULL, NULL, 1.0, 1.0, &P, mval, NULL);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t t = P.rp[i]; t < P.rp[i + 1]; ++t)
            for (int k = 0; k < K; ++k) ML[i * K + k] += mval[t] * L[(int64_t)P.ci[t] * K + k];
    for (int a = 0; a < K; ++a)
        for (int b = 0; b < K; ++b) {
            double s = 0.0;
            for (int64_t i = 0; i < n; ++i) s += L[i * K + a] * ML[i * K + b];
            B[a * K + b] = s;
        }
    /* symmetrise against round-off before the eigen-solve */
    for (int a = 0; a < K; ++a)
        for (int b = a + 1; b < K; ++b) {
            double s = 0.5 * (B[a * K + b] + B[b * K + a]);
            B[a * K + b] = s; B[b * K + a] = s;
        }
    jacobi_eigen(K, B, lam, V);

    /* sort descending (selection sort keeps the oracle obvious) */
    int *ord = malloc(sizeof(int) * K);
    for (int k = 0; k < K; ++k) ord[k] = k;
    for (int a = 0; a < K; ++a) {
        int best = a;
        for (int b = a + 1; b < K; ++b)
            if (lam[ord[b]] > lam[ord[best]]) best = b;
        int t = ord[a]; ord[a] = ord[best]; ord[best] = t;
    }
    for (int k = 0; k < K; ++k) {
        int src = ord[k];
        lambda[k] = lam[src];
        for (int64_t i = 0; i < n; ++i) {
            double s = 0.0;
            for (int j = 0; j < K; ++j) s += L[i * K + j] * V[j * K + src];
            modes[i * K + k] = s;
        }
        int64_t imax = 0;
        for (int64_t i = 1; i < n; ++i)
            if (fabs(modes[i * K + k]) > fabs(modes[imax * K + k])) imax = i;
        if (modes[imax * K + k] < 0.0)
            for (int64_t i = 0; i < n; ++i) modes[i * K + k] = -modes[i * K + k];
    }
    if (Lout) memcpy(Lout, L, sizeof(double) * (size_t)n * K);
    free(ord); free(L); free(mval); free(ML); free(B); free(lam); free(V); free_pattern(&P);
    return MLQO_OK;
}

/* ------------------------------------------------------------------------ */
/* Fine-to-coarse transfer of the field by the midpoint rule (Sec. 4):       */
/* every coarse element takes the value of the fine-level field at its       */
/* centroid.  The fine field is the P1 interpolant of nodal values on a      */
/* structured fine mesh (mesh2d / mesh3d layout).                            */
/* ------------------------------------------------------------------------ */

/* Evaluate the P1 interpolant of K nodal fields f (n_f x K, row-major) on the
 * structured 2D fine mesh with mf x mf nodes at the point p; out[K]. */
static void p1_eval_2d(int mf, const double *f, int K, const double *p, double *out)
{
    double h = 1.0 / (double)(mf - 1);
    double sx = p[0] / h, sy = p[1] / h;
    int i = (int)floor(sx), j = (int)floor(sy);
    if (i > mf - 2) i = mf - 2;
    if (j > mf - 2) j = mf - 2;
    if (i < 0) i = 0;
    if (j < 0) j = 0;
    double u = sx - i, w = sy - j; /* local coordinates in [0,1]^2 */
    int64_t n00 = i + (int64_t)mf * j, n10 = n00 + 1, n01 = n00 + mf, n11 = n00 + mf + 1;
    /* lower triangle (u >= w): (0,0),(1,0),(1,1) with weights 1-u, u-w, w
     * upper triangle (u <  w): (0,0),(1,1),(0,1) with weights 1-w, u, w-u */
    for (int k = 0; k < K; ++k) {
        double val;
        if (u >= w) val = (1.0 - u) * f[n00 * K + k] + (u - w) * f[n10 * K + k] + w * f[n11 * K + k];
        else val = (1.0 - w) * f[n00 * K + k] + u * f[n11 * K + k] + (w - u) * f[n01 * K + k];
        out[k] = val;
    }
}

/* Same in 3D on the Kuhn mesh: the tetrahedron containing a point of the unit
 * cube is the one whose step order sorts the local coordinates descending;
 * its barycentric weights are the successive differences of the sorted
 * coordinates. */
static void p1_eval_3d(int mx, int my, int mz, double Lx, double Ly, double Lz, const double *f, int K,
                       const double *p, double *out)
{
    double s[3] = {p[0] / (Lx / (mx - 1)), p[1] / (Ly / (my - 1)), p[2] / (Lz / (mz - 1))};
    int m[3] = {mx, my, mz};
    int c[3];
    double u[3];
    for (int a = 0; a < 3; ++a) {
        c[a] = (int)floor(s[a]);
        if (c[a] > m[a] - 2) c[a] = m[a] - 2;
        if (c[a] < 0) c[a] = 0;
        u[a] = s[a] - c[a];
    }
    /* order axes by local coordinate, descending; stable on ties */
    int ax[3] = {0, 1, 2};
    for (int a = 0; a < 3; ++a)
        for (int b = a + 1; b < 3; ++b)
            if (u[ax[b]] > u[ax[a]]) { int t = ax[a]; ax[a] = ax[b]; ax[b] = t; }
    double wts[4] = {1.0 - u[ax[0]], u[ax[0]] - u[ax[1]], u[ax[1]] - u[ax[2]], u[ax[2]]};
    int idx[3] = {c[0], c[1], c[2]};
    int64_t vert[4];
    vert[0] = idx[0] + (int64_t)mx * (idx[1] + (int64_t)my * idx[2]);
    for (int q = 0; q < 3; ++q) {
        idx[ax[q]] += 1;
        vert[q + 1] = idx[0] + (int64_t)mx * (idx[1] + (int64_t)my * idx[2]);
    }
    for (int k = 0; k < K; ++k) {
        double v = 0.0;
        for (int q = 0; q < 4; ++q) v += wts[q] * f[vert[q] * K + k];
        out[k] = v;
    }
}

/* Phi[e*K+k] = fine P1 interpolant of mode k at the centroid of coarse
 * element e.  dim = 2: fine dims (mf), coarse mesh given explicitly.
 * dim = 3: fine dims (mx,my,mz) and box lengths in fdims[0..2], flen[0..2]. */
int mlqo_centroid_table(int d, const int *fdims, const double *flen, const double *modes_f, int K,
                        const double *xyz_c, int64_t ne_c, const int32_t *conn_c, double *phi)
{
    int nv = d + 1;
    for (int64_t e = 0; e < ne_c; ++e) {
        double cen[3] = {0, 0, 0};
        for (int a = 0; a < nv; ++a)
            for (int c = 0; c < d; ++c) cen[c] += xyz_c[(int64_t)conn_c[e * nv + a] * d + c];
        for (int c = 0; c < d; ++c) cen[c] /= (double)nv;
        if (d == 2) p1_eval_2d(fdims[0], modes_f, K, cen, phi + e * K);
        else p1_eval_3d(fdims[0], fdims[1], fdims[2], flen[0], flen[1], flen[2], modes_f, K, cen, phi + e * K);
    }
    return MLQO_OK;
}

/* ------------------------------------------------------------------------ */
/* Forward solve of one sample: IMEX backward-Euler time blocks.             */
/* ------------------------------------------------------------------------ */

static void csr_apply(const pattern_t *P, const double *val, const double *x, double *y)
{
    for (int64_t i = 0; i < P->n; ++i) {
        double s = 0.0;
        for (int64_t t = P->rp[i]; t < P->rp[i + 1]; ++t) s += val[t] * x[P->ci[t]];
        y[i] = s;
    }
}

static double dot(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Jacobi-preconditioned CG for A x = b from the given x, stopping when the
 * recursively updated residual satisfies ||r||_2 <= rtol ||b||_2 or after
 * maxit iterations.  Returns the iteration count; *status gets the outcome. */
static int64_t pcg(const pattern_t *P, const double *aval, const double *dinv, const double *b, double *x,
                   double rtol, int64_t maxit, double *r, double *z, double *p, double *q, int *status)
{
    int64_t n = P->n;
    csr_apply(P, aval, x, q);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
    for (int64_t i = 0; i < n; ++i) z[i] = dinv[i] * r[i];
    for (int64_t i = 0; i < n; ++i) p[i] = z[i];
    double rz = dot(n, r, z);
    double bnorm = sqrt(dot(n, b, b));
    double rnorm = sqrt(dot(n, r, r));
    int64_t it = 0;
    *status = MLQO_S_CONVERGED;
    while (rnorm > rtol * bnorm) {
        if (!isfinite(rnorm)) { *status = MLQO_S_NONFINITE; return it; }
        if (it >= maxit) { *status = MLQO_S_MAXITER; return it; }
        csr_apply(P, aval, p, q);
        double alpha = rz / dot(n, p, q);
        for (int64_t i = 0; i < n; ++i) x[i] += alpha * p[i];
        for (int64_t i = 0; i < n; ++i) r[i] -= alpha * q[i];
        for (int64_t i = 0; i < n; ++i) z[i] = dinv[i] * r[i];
        double rz_new = dot(n, r, z);
        double beta = rz_new / rz;
        rz = rz_new;
        for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        rnorm = sqrt(dot(n, r, r));
        ++it;
    }
    return it;
}

/* Model parameters, in this order: s_l, s_t, a, eps, gamma.
 *   reaction  R(v,w) = v (v - a)(1 - v) - w         (FitzHugh-Nagumo, cubic
 *   recovery  dw/dt  = eps (v - gamma w)              current of eq. ionic_term)
 *
 * One time block n -> n+1 (backward Euler for diffusion, reaction explicit):
 *   R   = R(v^n, w^n)                     nodal
 *   b   = M (v^n + dt R)                  reaction as consistent-mass load (eq. mono_disc)
 *   (M + dt K) v^{n+1} = b                solved by Jacobi-PCG from x0 = v^n
 *   w^{n+1} = w^n + dt eps (v^n - gamma w^n)
 * After nsteps blocks: Q = sum_i m_i v_i with m = M 1, i.e. the integral of
 * the P1 field v_h(T) over the domain.
 *
 * Returns Q; v, w are updated in place; iters/status report the solver. */
typedef struct {
    pattern_t P;
    double *mval, *kval, *aval, *dinv, *mlump;
    int64_t ne;
} problem_t;

static int problem_setup(int d, int64_t n, const double *xyz, int64_t ne, const int32_t *conn, problem_t *pr)
{
    memset(pr, 0, sizeof(*pr));
    int st = build_pattern(d, n, ne, conn, &pr->P);
    if (st != MLQO_OK) return st;
    size_t nnz = (size_t)pr->P.nnz;
    pr->mval = malloc(sizeof(double) * nnz);
    pr->mlump = malloc(sizeof(double) * (size_t)n);
    if (!pr->mval || !pr->mlump) return MLQO_ENOMEM;
    assemble(d, xyz, ne, conn, NULL, NULL, 1.0, 1.0, &pr->P, pr->mval, NULL);
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t t = pr->P.rp[i]; t < pr->P.rp[i + 1]; ++t) s += pr->mval[t];
        pr->mlump[i] = s;
    }
    pr->ne = ne;
    return MLQO_OK;
}

static void problem_free(problem_t *pr)
{
    free_pattern(&pr->P);
    free(pr->mval); free(pr->mlump);
    pr->mval = NULL; pr->mlump = NULL;
}

static double solve_one(int d, const double *xyz, const int32_t *conn, const problem_t *pr,
                        const double *theta, const double *frames, const double *model, double dt, int nsteps,
                        double rtol,
                        int64_t maxit, double *v, double *w, int64_t *iters_out, int *status_out)
{
    const pattern_t *P = &pr->P;
    int64_t n = P->n, nnz = P->nnz;
    double s_l = model[0], s_t = model[1], a = model[2], eps = model[3], gam = model[4];
    double *kval = malloc(sizeof(double) * (size_t)nnz);
    double *aval = malloc(sizeof(double) * (size_t)nnz);
    double *dinv = malloc(sizeof(double) * (size_t)n);
    double *y = malloc(sizeof(double) * (size_t)n), *b = malloc(sizeof(double) * (size_t)n);
    double *x = malloc(sizeof(double) * (size_t)n), *r = malloc(sizeof(double) * (size_t)n);
    double *z = malloc(sizeof(double) * (size_t)n), *p = malloc(sizeof(double) * (size_t)n);
    double *q = malloc(sizeof(double) * (size_t)n);
    assemble(d, xyz, pr->ne, conn, theta, frames, s_l, s_t, P, NULL, kval);
    for (int64_t t = 0; t < nnz; ++t) aval[t] = pr->mval[t] + dt * kval[t];
    for (int64_t i = 0; i < n; ++i) dinv[i] = 1.0 / aval[find_col(P, i, (int32_t)i)];
    int64_t iters = 0;
    int status = MLQO_S_CONVERGED;
    for (int step = 0; step < nsteps; ++step) {
        for (int64_t i = 0; i < n; ++i) {
            double R = v[i] * (v[i] - a) * (1.0 - v[i]) - w[i];
            y[i] = v[i] + dt * R;
        }
        csr_apply(P, pr->mval, y, b);
        for (int64_t i = 0; i < n; ++i) x[i] = v[i];
        int st;
        iters += pcg(P, aval, dinv, b, x, rtol, maxit, r, z, p, q, &st);
        if (st != MLQO_S_CONVERGED && status == MLQO_S_CONVERGED) status = st;
        for (int64_t i = 0; i < n; ++i) {
            w[i] = w[i] + dt * eps * (v[i] - gam * w[i]);
            v[i] = x[i];
        }
    }
    double Q = dot(n, pr->mlump, v);
    if (!isfinite(Q) && status == MLQO_S_CONVERGED) status = MLQO_S_NONFINITE;
    if (iters_out) *iters_out = iters;
    if (status_out) *status_out = status;
    free(kval); free(aval); free(dinv); free(y); free(b); free(x); free(r); free(z); free(p); free(q);
    return Q;
}

/* Public: one sample with an explicit per-element angle field theta.
 * v, w (length n) hold the initial state on entry and the final state on
 * exit.  q_out gets the QoI. */
int mlqo_solve(int d, int64_t n, const double *xyz, int64_t ne, const int32_t *conn, const double *theta,
               const double *model, double dt, int nsteps, double rtol, int64_t maxit, double *v, double *w,
               double *q_out, int64_t *iters_out, int32_t *status_out)
{
    problem_t pr;
    int st = problem_setup(d, n, xyz, ne, conn, &pr);
    if (st != MLQO_OK) { problem_free(&pr); return st; }
    int s;
    *q_out = solve_one(d, xyz, conn, &pr, theta, NULL, model, dt, nsteps, rtol, maxit, v, w, iters_out, &s);
    if (status_out) *status_out = s;
    problem_free(&pr);
    return MLQO_OK;
}

/* Public: a batch of S samples.  Sample s uses the angle field
 *   theta_e = theta_mean_e + sum_k phi[e*K+k] * xi[s*K+k]     (eq. KLlowrank)
 * turning the fibre in the plane of the element's frame (frames: n_e x 6, or
 * NULL for the x-y plane), and the initial state v0, w0 (w0 may be NULL = 0).
 * Samples run in parallel over nthreads OpenMP threads (<= 0: the runtime
 * default).  q_out[s], iters[s] (may be NULL), status[s] (may be NULL). */
int mlqo_solve_batch_f(int d, int64_t n, const double *xyz, int64_t ne, const int32_t *conn, const double *frames,
                       int K, const double *phi, const double *theta_mean, int64_t S, const double *xi,
                       const double *model, double dt, int nsteps, double rtol, int64_t maxit, const double *v0,
                       const double *w0, int nthreads, double *q_out, int64_t *iters, int32_t *status)
{
    problem_t pr;
    int st = problem_setup(d, n, xyz, ne, conn, &pr);
    if (st != MLQO_OK) { problem_free(&pr); return st; }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t s = 0; s < S; ++s) {
        double *theta = malloc(sizeof(double) * (size_t)ne);
        double *v = malloc(sizeof(double) * (size_t)n), *w = malloc(sizeof(double) * (size_t)n);
        for (int64_t e = 0; e < ne; ++e) {
            double t = theta_mean ? theta_mean[e] : 0.0;
            for (int k = 0; k < K; ++k) t += phi[e * K + k] * xi[s * K + k];
            theta[e] = t;
        }
        for (int64_t i = 0; i < n; ++i) { v[i] = v0[i]; w[i] = w0 ? w0[i] : 0.0; }
        int64_t it = 0;
        int sst = 0;
        q_out[s] = solve_one(d, xyz, conn, &pr, theta, frames, model, dt, nsteps, rtol, maxit, v, w, &it, &sst);
        if (iters) iters[s] = it;
        if (status) status[s] = sst;
        free(theta); free(v); free(w);
    }
    problem_free(&pr);
    return MLQO_OK;
}

/* Public: the batch with fibres in the x-y plane. */
int mlqo_solve_batch(int d, int64_t n, const double *xyz, int64_t ne, const int32_t *conn, int K,
                     const double *phi, const double *theta_mean, int64_t S, const double *xi,
                     const double *model, double dt, int nsteps, double rtol, int64_t maxit, const double *v0,
                     const double *w0, int nthreads, double *q_out, int64_t *iters, int32_t *status)
{
    return mlqo_solve_batch_f(d, n, xyz, ne, conn, NULL, K, phi, theta_mean, S, xi, model, dt, nsteps, rtol, maxit,
                              v0, w0, nthreads, q_out, iters, status);
}

/* ------------------------------------------------------------------------ */
/* The paper's time discretization (Sec. 3.1 eq. st-system with the reaction  */
/* of eq. mono_disc; the model of eq. ionic_term, the stimulus of Sec. 5.1). */
/* ------------------------------------------------------------------------ */

/* Parameters pm, in this order: s_l, s_t, alpha, u_rest, u_th, u_peak,
 * theta, amp, sigma, t1, x0, y0, z0.
 *   I_ion(u)   = alpha (u - u_rest)(u - u_th)(u - u_peak)           (eq. ionic_term)
 *   I_app(x,t) = (u_rest + amp exp(-|x - x0|^2 / sigma^2)) for 0 <= t < t1, else 0
 * One time block k -> k+1 (theta = 1/2: Crank-Nicolson, eq. st-system; 1:
 * backward Euler), the reaction on the new time level (eq. mono_disc):
 *   F(u) = (M + theta dt K) u + dt M I_ion(u)
 *          - (M - (1 - theta) dt K) u_k - dt M (theta g(t_{k+1}) + (1 - theta) g(t_k)) = 0
 * with g(t) the nodal values of I_app(., t), t_k = k dt.  Newton's method
 * from u_k: J(u) = M + theta dt K + dt M diag(I_ion'(u)) (not symmetric),
 * J d = -F(u) by BiCGSTAB with a Jacobi preconditioner, until ||F|| <=
 * rtol ||c||, c the u-independent part. */
static double ionic(const double *pm, double u) { return pm[2] * (u - pm[3]) * (u - pm[4]) * (u - pm[5]); }

static double ionic_deriv(const double *pm, double u)
{
    const double a = pm[3], b = pm[4], c = pm[5];
    return pm[2] * ((u - b) * (u - c) + (u - a) * (u - c) + (u - a) * (u - b));
}

static double iapp(int d, const double *x, const double *pm, double t)
{
    if (!(t >= 0.0 && t < pm[9])) return 0.0;
    double r2 = 0.0;
    for (int c = 0; c < d; ++c) r2 += (x[c] - pm[10 + c]) * (x[c] - pm[10 + c]);
    return pm[3] + pm[7] * exp(-r2 / (pm[8] * pm[8]));
}

/* BiCGSTAB (van der Vorst) with right Jacobi preconditioning for the CSR
 * values jval (pattern P): solve J x = b from x = 0 to ||b - J x|| <=
 * rtol ||b||.  Work vectors of length n: r rh p v s t y z.  Returns the
 * iterations (or -1 on breakdown / non-finite values). */
static int64_t bicgstab(const pattern_t *P, const double *jval, const double *dinv, const double *b, double *x,
                        double rtol, int64_t maxit, double *r, double *rh, double *p, double *v, double *s, double *t,
                        double *y, double *z)
{
    const int64_t n = P->n;
    for (int64_t i = 0; i < n; ++i) { x[i] = 0.0; r[i] = b[i]; rh[i] = b[i]; p[i] = 0.0; v[i] = 0.0; }
    const double bnorm = sqrt(dot(n, b, b));
    if (bnorm == 0.0) return 0;
    double rho = 1.0, alpha = 1.0, omega = 1.0;
    for (int64_t it = 0; it < maxit; ++it) {
        const double rho_new = dot(n, rh, r);
        if (rho_new == 0.0 || !isfinite(rho_new)) return -1;
        const double beta = (rho_new / rho) * (alpha / omega);
        for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
        for (int64_t i = 0; i < n; ++i) y[i] = dinv[i] * p[i];
        csr_apply(P, jval, y, v);
        alpha = rho_new / dot(n, rh, v);
        for (int64_t i = 0; i < n; ++i) s[i] = r[i] - alpha * v[i];
        if (sqrt(dot(n, s, s)) <= rtol * bnorm) {
            for (int64_t i = 0; i < n; ++i) x[i] += alpha * y[i];
            return it + 1;
        }
        for (int64_t i = 0; i < n; ++i) z[i] = dinv[i] * s[i];
        csr_apply(P, jval, z, t);
        omega = dot(n, t, s) / dot(n, t, t);
        for (int64_t i = 0; i < n; ++i) x[i] += alpha * y[i] + omega * z[i];
        for (int64_t i = 0; i < n; ++i) r[i] = s[i] - omega * t[i];
        rho = rho_new;
        const double rn = sqrt(dot(n, r, r));
        if (!isfinite(rn)) return -1;
        if (rn <= rtol * bnorm) return it + 1;
    }
    return maxit;
}

/* Public: one sample of the paper's scheme with angle field theta (per
 * element).  u (length n) holds the initial potential on entry and the
 * final one on exit; q_out = m^T u(T); newton_out = Newton steps summed over
 * the blocks (may be NULL); status (may be NULL). */
int mlqo_solve_paper(int d, int64_t n, const double *xyz, int64_t ne, const int32_t *conn, const double *theta,
                     const double *pm, double dt, int nsteps, double rtol, int64_t maxit, double *u, double *q_out,
                     int64_t *newton_out, int32_t *status)
{
    problem_t pr;
    int st = problem_setup(d, n, xyz, ne, conn, &pr);
    if (st != MLQO_OK) { problem_free(&pr); return st; }
    const pattern_t *P = &pr.P;
    const int64_t nnz = P->nnz;
    const double th = pm[6];
    double *kval = malloc(sizeof(double) * (size_t)nnz), *aval = malloc(sizeof(double) * (size_t)nnz);
    double *jval = malloc(sizeof(double) * (size_t)nnz), *dinv = malloc(sizeof(double) * (size_t)n);
    double *w[14];
    for (int k = 0; k < 14; ++k) w[k] = malloc(sizeof(double) * (size_t)n);
    double *c = w[0], *F = w[1], *du = w[2], *gk = w[3], *gk1 = w[4], *tmp = w[5];
    assemble(d, xyz, ne, conn, theta, NULL, pm[0], pm[1], P, NULL, kval);
    for (int64_t t = 0; t < nnz; ++t) aval[t] = pr.mval[t] + th * dt * kval[t];
    int64_t newton = 0;
    int sst = MLQO_S_CONVERGED;
    for (int k = 0; k < nsteps && sst != MLQO_S_NONFINITE; ++k) {
        for (int64_t i = 0; i < n; ++i) {
            gk[i] = iapp(d, xyz + i * d, pm, k * dt);
            gk1[i] = iapp(d, xyz + i * d, pm, (k + 1) * dt);
        }
        /* c = M u_k - (1 - theta) dt K u_k + dt M (theta g_{k+1} + (1 - theta) g_k) */
        for (int64_t i = 0; i < n; ++i) tmp[i] = u[i] + dt * (th * gk1[i] + (1.0 - th) * gk[i]);
        csr_apply(P, pr.mval, tmp, c);
        csr_apply(P, kval, u, tmp);
        for (int64_t i = 0; i < n; ++i) c[i] -= (1.0 - th) * dt * tmp[i];
        const double cnorm = sqrt(dot(n, c, c));
        int conv = 0;
        for (int it = 0; it < 100; ++it) {
            /* F = A u + dt M I(u) - c */
            csr_apply(P, aval, u, F);
            for (int64_t i = 0; i < n; ++i) tmp[i] = ionic(pm, u[i]);
            csr_apply(P, pr.mval, tmp, du);
            for (int64_t i = 0; i < n; ++i) F[i] += dt * du[i] - c[i];
            const double fn = sqrt(dot(n, F, F));
            if (!isfinite(fn)) { sst = MLQO_S_NONFINITE; break; }
            if (fn <= rtol * cnorm) { conv = 1; break; }
            /* J = A + dt M diag(I'(u)): column j of M scaled by I'(u_j) */
            for (int64_t i = 0; i < n; ++i)
                for (int64_t t = P->rp[i]; t < P->rp[i + 1]; ++t)
                    jval[t] = aval[t] + dt * pr.mval[t] * ionic_deriv(pm, u[P->ci[t]]);
            for (int64_t i = 0; i < n; ++i) dinv[i] = 1.0 / jval[find_col(P, i, (int32_t)i)];
            for (int64_t i = 0; i < n; ++i) F[i] = -F[i];
            if (bicgstab(P, jval, dinv, F, du, 1e-3 * rtol, maxit, w[6], w[7], w[8], w[9], w[10], w[11], w[12],
                         w[13]) < 0) { sst = MLQO_S_NONFINITE; break; }
            for (int64_t i = 0; i < n; ++i) u[i] += du[i];
            ++newton;
        }
        if (!conv && sst == MLQO_S_CONVERGED) sst = MLQO_S_MAXITER;
    }
    double Q = dot(n, pr.mlump, u);
    if (!isfinite(Q)) sst = MLQO_S_NONFINITE;
    *q_out = Q;
    if (newton_out) *newton_out = newton;
    if (status) *status = sst;
    free(kval); free(aval); free(jval); free(dinv);
    for (int k = 0; k < 14; ++k) free(w[k]);
    problem_free(&pr);
    return MLQO_OK;
}

/* Public: number of OpenMP threads a parallel region would use. */
int mlqo_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
