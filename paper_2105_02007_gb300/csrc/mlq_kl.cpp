// mlq_kl.cpp -- host-side setup of libmlq: KL modes (Sec. 2.3) and the
// midpoint-rule transfer of the fibre field to coarser levels (Sec. 4).
//
// Runs once per configuration, before any sample is solved, so it is plain
// C++ on the host.  The per-sample synthesis from these modes (eq. KLlowrank)
// is kernel K1.
#include "mlq.h"
#include "mlq_host.h"

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <cstdint>
#include <new>
#include <thread>
#include <vector>

namespace {

// Nodes per chunk of the host loops below.  Every reduction is formed per
// chunk and the chunk results are combined in chunk order, so the results
// depend on this constant but not on the number of threads.
constexpr int64_t kChunk = 8192;

// f(c) for c = 0 .. nchunks-1, spread over the host's cores
template <typename F>
void parallel_chunks(int64_t nchunks, F &&f)
{
    const int64_t hw = std::max(1u, std::thread::hardware_concurrency());
    const int64_t nt = std::min<int64_t>(hw, nchunks);
    if (nt <= 1) {
        for (int64_t c = 0; c < nchunks; ++c) f(c);
        return;
    }
    std::atomic<int64_t> next{0};
    auto work = [&]() {
        for (int64_t c; (c = next.fetch_add(1)) < nchunks;) f(c);
    };
    std::vector<std::thread> pool;
    pool.reserve(nt - 1);
    for (int64_t t = 1; t < nt; ++t) pool.emplace_back(work);
    work();
    for (auto &th : pool) th.join();
}

int64_t nchunks_of(int64_t n) { return (n + kChunk - 1) / kChunk; }

struct Grid2 {
    int m;
    double h;
    double x(int64_t node) const { return (double)(node % m) / (double)(m - 1); }
    double y(int64_t node) const { return (double)(node / m) / (double)(m - 1); }
};

// y = M x for the P1 mass matrix of the structured triangulation, using the
// closed-form entries: every triangle adds h^2/12 to the diagonal of each of
// its vertices and h^2/24 to each of its edges.
void mass_apply(const Grid2 &g, const double *x, double *y, int ncol)
{
    const int m = g.m, mc = m - 1;
    const double d = g.h * g.h / 12.0, e = g.h * g.h / 24.0;
    parallel_chunks(m, [&](int64_t jc) {
        const int j = (int)jc;
        for (int i = 0; i < m; ++i) {
            const int64_t P = i + (int64_t)m * j;
            const int cij = (i < mc && j < mc), cim = (i >= 1 && j < mc), cmm = (i >= 1 && j >= 1),
                      cjm = (i < mc && j >= 1);
            const int ninc = 2 * cij + cim + 2 * cmm + cjm;
            for (int c = 0; c < ncol; ++c) {
                double acc = ninc * d * x[P * ncol + c];
                if (i + 1 < m) acc += e * (cij + cjm) * x[(P + 1) * ncol + c];
                if (i > 0) acc += e * (cim + cmm) * x[(P - 1) * ncol + c];
                if (j + 1 < m) acc += e * (cij + cim) * x[(P + m) * ncol + c];
                if (j > 0) acc += e * (cjm + cmm) * x[(P - m) * ncol + c];
                if (i + 1 < m && j + 1 < m) acc += e * 2 * cij * x[(P + m + 1) * ncol + c];
                if (i > 0 && j > 0) acc += e * 2 * cmm * x[(P - m - 1) * ncol + c];
                y[P * ncol + c] = acc;
            }
        }
    });
}

// Symmetric eigen-decomposition by cyclic Jacobi rotations; the eigenvectors
// are the columns of Q (row-major).
void sym_eigen(int K, std::vector<double> A, std::vector<double> &lam, std::vector<double> &Q)
{
    Q.assign((size_t)K * K, 0.0);
    for (int k = 0; k < K; ++k) Q[(size_t)k * K + k] = 1.0;
    auto at = [&](int r, int c) -> double & { return A[(size_t)r * K + c]; };
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int r = 0; r < K; ++r)
            for (int c = 0; c < K; ++c) (r == c ? diag : off) += at(r, c) * at(r, c);
        if (off <= 1e-32 * diag) break;
        for (int p = 0; p + 1 < K; ++p)
            for (int q = p + 1; q < K; ++q) {
                const double apq = at(p, q);
                if (apq == 0.0) continue;
                const double theta = (at(q, q) - at(p, p)) / (2.0 * apq);
                const double t = std::copysign(1.0, theta) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < K; ++k) {  // columns p, q
                    const double x = at(k, p), y = at(k, q);
                    at(k, p) = c * x - s * y;
                    at(k, q) = s * x + c * y;
                }
                for (int k = 0; k < K; ++k) {  // rows p, q
                    const double x = at(p, k), y = at(q, k);
                    at(p, k) = c * x - s * y;
                    at(q, k) = s * x + c * y;
                }
                for (int k = 0; k < K; ++k) {
                    const double x = Q[(size_t)k * K + p], y = Q[(size_t)k * K + q];
                    Q[(size_t)k * K + p] = c * x - s * y;
                    Q[(size_t)k * K + q] = s * x + c * y;
                }
            }
    }
    lam.resize(K);
    for (int k = 0; k < K; ++k) lam[k] = at(k, k);
}

// Value at point (px, py) of the P1 interpolant of K nodal fields on the
// m x m structured triangulation.
void p1_at(const Grid2 &g, const double *f, int K, double px, double py, double *out)
{
    const int m = g.m;
    const double sx = px * (m - 1), sy = py * (m - 1);
    int i = std::min(std::max((int)std::floor(sx), 0), m - 2);
    int j = std::min(std::max((int)std::floor(sy), 0), m - 2);
    const double u = sx - i, w = sy - j;
    const int64_t a = i + (int64_t)m * j;
    // lower triangle (u >= w): (i,j) (i+1,j) (i+1,j+1); upper: (i,j) (i+1,j+1) (i,j+1)
    double wa, wb, wc;
    int64_t nb, nc;
    if (u >= w) {
        wa = 1.0 - u; wb = u - w; wc = w;
        nb = a + 1; nc = a + m + 1;
    } else {
        wa = 1.0 - w; wb = u; wc = w - u;
        nb = a + m + 1; nc = a + m;
    }
    for (int k = 0; k < K; ++k) out[k] = wa * f[a * K + k] + wb * f[nb * K + k] + wc * f[nc * K + k];
}

// 3D structured box of Kuhn tetrahedra (see the mesh convention in mlq.h):
// nodes i + mx (j + my k), six tetrahedra per cube stepping along the axes
// of one permutation.
struct Grid3h {
    int mx, my, mz;
    double hx, hy, hz;
    int64_t n() const { return (int64_t)mx * my * mz; }
};

const int kPerm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

// y = M x for the P1 mass matrix (|e|/20 (1 + delta_ab) per tetrahedron)
void mass_apply3(const Grid3h &g, const double *x, double *y, int ncol)
{
    const int64_t n = g.n();
    std::fill(y, y + n * ncol, 0.0);
    const double c = g.hx * g.hy * g.hz / 6.0 / 20.0;
    // a cell plane k adds into the node planes k and k + 1: the even cell
    // planes first, then the odd ones, each set in parallel
    for (int parity = 0; parity < 2; ++parity)
        parallel_chunks((g.mz - 1 - parity + 1) / 2, [&](int64_t kc) {
            const int k = 2 * (int)kc + parity;
            for (int j = 0; j + 1 < g.my; ++j)
                for (int i = 0; i + 1 < g.mx; ++i)
                    for (int s = 0; s < 6; ++s) {
                    int64_t v[4];
                    int idx[3] = {i, j, k};
                    v[0] = idx[0] + (int64_t)g.mx * (idx[1] + (int64_t)g.my * idx[2]);
                    for (int q = 0; q < 3; ++q) {
                        idx[kPerm[s][q]] += 1;
                        v[q + 1] = idx[0] + (int64_t)g.mx * (idx[1] + (int64_t)g.my * idx[2]);
                    }
                    for (int col = 0; col < ncol; ++col) {
                        double sum = 0.0;
                        for (int a = 0; a < 4; ++a) sum += x[v[a] * ncol + col];
                        for (int a = 0; a < 4; ++a) y[v[a] * ncol + col] += c * (sum + x[v[a] * ncol + col]);
                    }
                }
        });
}

// Value at (px, py, pz) of the P1 interpolant of K nodal fields on the Kuhn
// mesh: the tetrahedron of the cube is the one whose steps follow the local
// coordinates in decreasing order; the weights are the differences of the
// sorted coordinates (continuous across faces, so ties do not matter).
void p1_at3(const Grid3h &g, const double *f, int K, double px, double py, double pz, double *out)
{
    const double s[3] = {px / g.hx, py / g.hy, pz / g.hz};
    const int mm[3] = {g.mx, g.my, g.mz};
    int c[3];
    double u[3];
    for (int a = 0; a < 3; ++a) {
        c[a] = std::min(std::max((int)std::floor(s[a]), 0), mm[a] - 2);
        u[a] = s[a] - c[a];
    }
    int ord[3] = {0, 1, 2};
    std::stable_sort(ord, ord + 3, [&](int a, int b) { return u[a] > u[b]; });
    int idx[3] = {c[0], c[1], c[2]};
    const double wts[4] = {1.0 - u[ord[0]], u[ord[0]] - u[ord[1]], u[ord[1]] - u[ord[2]], u[ord[2]]};
    for (int k = 0; k < K; ++k) out[k] = 0.0;
    for (int q = 0; q < 4; ++q) {
        if (q > 0) idx[ord[q - 1]] += 1;
        const int64_t v = idx[0] + (int64_t)g.mx * (idx[1] + (int64_t)g.my * idx[2]);
        for (int k = 0; k < K; ++k) out[k] += wts[q] * f[v * K + k];
    }
}

// K steps of pivoted Cholesky of the covariance over the node coordinates
// (first maximum of the residual diagonal as pivot), B = L^T M L, its
// eigenpairs by cyclic Jacobi, modes v_k = L q_k sorted by decreasing
// eigenvalue, largest-magnitude entry positive (eqs. approxEig, redEig).
template <typename Coord, typename Mass>
int build_kl_nodes(int64_t n, Coord coord, Mass mass, double sigma2, double ell, int K, double *modes_out,
                   double *lambda_out)
{
    const int64_t nc = nchunks_of(n);
    auto chunk = [&](int64_t c, int64_t &t0, int64_t &t1) {
        t0 = c * kChunk;
        t1 = std::min(n, t0 + kChunk);
    };
    std::vector<double> X(n * 3);
    for (int64_t t = 0; t < n; ++t) coord(t, &X[t * 3]);
    auto cov = [&](int64_t a, int64_t b) {
        const double dx = X[a * 3] - X[b * 3], dy = X[a * 3 + 1] - X[b * 3 + 1], dz = X[a * 3 + 2] - X[b * 3 + 2];
        return sigma2 * std::exp(-(dx * dx + dy * dy + dz * dz) / ell);
    };
    // pivoted Cholesky: L (n x K, row-major), residual diagonal r; the pivot
    // is the first maximum of r (per-chunk first maxima, combined in order)
    std::vector<double> L((size_t)n * K, 0.0), r(n, sigma2);
    std::vector<double> cmax(nc);
    std::vector<int64_t> carg(nc);
    for (int k = 0; k < K; ++k) {
        parallel_chunks(nc, [&](int64_t c) {
            int64_t t0, t1;
            chunk(c, t0, t1);
            const int64_t a = std::max_element(r.begin() + t0, r.begin() + t1) - r.begin();
            cmax[c] = r[a];
            carg[c] = a;
        });
        int64_t piv = carg[0];
        for (int64_t c = 1; c < nc; ++c)
            if (cmax[c] > r[piv]) piv = carg[c];
        const double lp = std::sqrt(r[piv]);
        if (!(lp > 0.0)) return MLQ_EINVAL;
        parallel_chunks(nc, [&](int64_t c) {
            int64_t t0, t1;
            chunk(c, t0, t1);
            for (int64_t t = t0; t < t1; ++t) {
                double v = cov(t, piv);
                for (int q = 0; q < k; ++q) v -= L[(size_t)t * K + q] * L[(size_t)piv * K + q];
                v /= lp;
                L[(size_t)t * K + k] = v;
                r[t] -= v * v;
            }
        });
    }
    // B = L^T (M L): upper triangle summed per node range, the ranges added
    // in order (as many ranges as chunks while their K x K partial sums stay
    // within 2^24 values)
    std::vector<double> ML((size_t)n * K);
    mass(L.data(), ML.data(), K);
    const int64_t nb = std::min<int64_t>(nc, std::max<int64_t>(1, ((int64_t)1 << 24) / ((int64_t)K * K)));
    std::vector<double> Bc((size_t)nb * K * K, 0.0);
    parallel_chunks(nb, [&](int64_t c) {
        const int64_t t0 = n * c / nb, t1 = n * (c + 1) / nb;
        double *b = &Bc[(size_t)c * K * K];
        for (int64_t t = t0; t < t1; ++t) {
            const double *lt = &L[(size_t)t * K], *mt = &ML[(size_t)t * K];
            for (int a = 0; a < K; ++a) {
                const double la = lt[a];
                for (int q = a; q < K; ++q) b[(size_t)a * K + q] += la * mt[q];
            }
        }
    });
    std::vector<double> B((size_t)K * K, 0.0);
    for (int64_t c = 0; c < nb; ++c)
        for (int a = 0; a < K; ++a)
            for (int q = a; q < K; ++q) B[(size_t)a * K + q] += Bc[((size_t)c * K + a) * K + q];
    for (int a = 0; a < K; ++a)
        for (int q = 0; q < a; ++q) B[(size_t)a * K + q] = B[(size_t)q * K + a];
    std::vector<double> lam, Q;
    sym_eigen(K, B, lam, Q);
    std::vector<int> ord(K);
    for (int k = 0; k < K; ++k) ord[k] = k;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int c) { return lam[a] > lam[c]; });
    for (int k = 0; k < K; ++k) lambda_out[k] = lam[ord[k]];
    // modes v_k = L q_k; per mode the first entry of largest magnitude
    std::vector<double> big((size_t)nc * K, 0.0);
    std::vector<int64_t> arg((size_t)nc * K, 0);
    parallel_chunks(nc, [&](int64_t c) {
        int64_t t0, t1;
        chunk(c, t0, t1);
        for (int k = 0; k < K; ++k) arg[(size_t)c * K + k] = t0;
        for (int64_t t = t0; t < t1; ++t)
            for (int k = 0; k < K; ++k) {
                const int src = ord[k];
                double sum = 0.0;
                for (int q = 0; q < K; ++q) sum += L[(size_t)t * K + q] * Q[(size_t)q * K + src];
                modes_out[(size_t)t * K + k] = sum;
                if (std::fabs(sum) > big[(size_t)c * K + k]) {
                    big[(size_t)c * K + k] = std::fabs(sum);
                    arg[(size_t)c * K + k] = t;
                }
            }
    });
    std::vector<char> flip(K, 0);
    for (int k = 0; k < K; ++k) {
        double b = big[k];
        int64_t a = arg[k];
        for (int64_t c = 1; c < nc; ++c)
            if (big[(size_t)c * K + k] > b) {
                b = big[(size_t)c * K + k];
                a = arg[(size_t)c * K + k];
            }
        flip[k] = modes_out[(size_t)a * K + k] < 0.0;
    }
    parallel_chunks(nc, [&](int64_t c) {
        int64_t t0, t1;
        chunk(c, t0, t1);
        for (int64_t t = t0; t < t1; ++t)
            for (int k = 0; k < K; ++k)
                if (flip[k]) modes_out[(size_t)t * K + k] = -modes_out[(size_t)t * K + k];
    });
    return MLQ_OK;
}

// General simplicial mesh (triangles or tetrahedra given by node lists).
struct SimplexMesh {
    int d;
    int64_t n, ne;
    const double *xyz;     // n x d
    const int32_t *conn;   // ne x (d + 1)
};

// |e|: the simplex measure (area or volume) from the edge vectors
double simplex_measure(const SimplexMesh &m, int64_t e)
{
    const int nv = m.d + 1;
    const double *p0 = m.xyz + (int64_t)m.conn[e * nv] * m.d;
    double E[3][3] = {};
    for (int a = 1; a < nv; ++a)
        for (int c = 0; c < m.d; ++c) E[a - 1][c] = m.xyz[(int64_t)m.conn[e * nv + a] * m.d + c] - p0[c];
    if (m.d == 2) return 0.5 * std::fabs(E[0][0] * E[1][1] - E[0][1] * E[1][0]);
    const double cx = E[1][1] * E[2][2] - E[1][2] * E[2][1], cy = E[1][2] * E[2][0] - E[1][0] * E[2][2],
                 cz = E[1][0] * E[2][1] - E[1][1] * E[2][0];
    return std::fabs(E[0][0] * cx + E[0][1] * cy + E[0][2] * cz) / 6.0;
}

// Simplices at each node, in element order (CSR: start[n + 1], list)
void node_incidence(const SimplexMesh &m, std::vector<int64_t> &start, std::vector<int32_t> &list)
{
    const int nv = m.d + 1;
    start.assign((size_t)m.n + 1, 0);
    for (int64_t e = 0; e < m.ne; ++e)
        for (int a = 0; a < nv; ++a) ++start[(size_t)m.conn[e * nv + a] + 1];
    for (int64_t i = 0; i < m.n; ++i) start[(size_t)i + 1] += start[(size_t)i];
    list.resize((size_t)start[(size_t)m.n]);
    std::vector<int64_t> fill(start.begin(), start.end() - 1);
    for (int64_t e = 0; e < m.ne; ++e)
        for (int a = 0; a < nv; ++a) list[(size_t)fill[(size_t)m.conn[e * nv + a]]++] = (int32_t)e;
}

// y = M x for the P1 mass matrix, M_e = |e| (1 + delta_ab) / ((d + 1)(d + 2)),
// gathered per node: (M x)_i = sum over e at i of |e| / ((d+1)(d+2)) (x_i +
// sum_{a in e} x_a)
void mass_apply_mesh(const SimplexMesh &m, const std::vector<double> &meas, const std::vector<int64_t> &start,
                     const std::vector<int32_t> &list, const double *x, double *y, int ncol)
{
    const int nv = m.d + 1;
    const double w = 1.0 / (double)((m.d + 1) * (m.d + 2));
    parallel_chunks(nchunks_of(m.n), [&](int64_t c) {
        const int64_t i0 = c * kChunk, i1 = std::min(m.n, i0 + kChunk);
        std::vector<double> acc((size_t)ncol);
        for (int64_t i = i0; i < i1; ++i) {
            std::fill(acc.begin(), acc.end(), 0.0);
            for (int64_t t = start[(size_t)i]; t < start[(size_t)i + 1]; ++t) {
                const int64_t e = list[(size_t)t];
                const double c_e = meas[(size_t)e] * w;
                for (int col = 0; col < ncol; ++col) {
                    double sum = x[i * ncol + col];
                    for (int a = 0; a < nv; ++a) sum += x[(int64_t)m.conn[e * nv + a] * ncol + col];
                    acc[(size_t)col] += c_e * sum;
                }
            }
            for (int col = 0; col < ncol; ++col) y[i * ncol + col] = acc[(size_t)col];
        }
    });
}

bool mesh_ok(int dim, int64_t n, const double *xyz, int64_t ne, const int32_t *conn)
{
    if ((dim != 2 && dim != 3) || n < 1 || ne < 1 || !xyz || !conn) return false;
    for (int64_t t = 0; t < ne * (dim + 1); ++t)
        if (conn[t] < 0 || conn[t] >= n) return false;
    return true;
}

int build_kl_mesh(int dim, int64_t n, const double *xyz, int64_t ne, const int32_t *conn, double sigma2, double ell,
                  int K, double *modes_out, double *lambda_out)
{
    if (!mesh_ok(dim, n, xyz, ne, conn) || !modes_out || !lambda_out || !(sigma2 > 0.0) || !(ell > 0.0))
        return MLQ_EINVAL;
    if (K < 1 || K > n || K > 4096) return MLQ_EINVAL;
    const SimplexMesh m{dim, n, ne, xyz, conn};
    std::vector<double> meas((size_t)ne);
    for (int64_t e = 0; e < ne; ++e) meas[(size_t)e] = simplex_measure(m, e);
    std::vector<int64_t> start;
    std::vector<int32_t> list;
    node_incidence(m, start, list);
    auto coord = [&](int64_t t, double *x) {
        for (int c = 0; c < 3; ++c) x[c] = c < dim ? xyz[t * dim + c] : 0.0;
    };
    auto mass = [&](const double *x, double *y, int ncol) { mass_apply_mesh(m, meas, start, list, x, y, ncol); };
    return build_kl_nodes(n, coord, mass, sigma2, ell, K, modes_out, lambda_out);
}

// Barycentric coordinates of x in simplex e as ratios of signed measures
// (x replacing one vertex at a time); returns the smallest
double barycentric_of(const SimplexMesh &m, int64_t e, const double *x, double *lam)
{
    const int nv = m.d + 1;
    double P[4][3] = {};
    for (int a = 0; a < nv; ++a)
        for (int c = 0; c < m.d; ++c) P[a][c] = m.xyz[(int64_t)m.conn[e * nv + a] * m.d + c];
    auto signed_measure = [&](const double (*Q)[3]) {
        if (m.d == 2) return (Q[1][0] - Q[0][0]) * (Q[2][1] - Q[0][1]) - (Q[1][1] - Q[0][1]) * (Q[2][0] - Q[0][0]);
        const double a[3] = {Q[1][0] - Q[0][0], Q[1][1] - Q[0][1], Q[1][2] - Q[0][2]};
        const double b[3] = {Q[2][0] - Q[0][0], Q[2][1] - Q[0][1], Q[2][2] - Q[0][2]};
        const double c[3] = {Q[3][0] - Q[0][0], Q[3][1] - Q[0][1], Q[3][2] - Q[0][2]};
        return a[0] * (b[1] * c[2] - b[2] * c[1]) + a[1] * (b[2] * c[0] - b[0] * c[2]) + a[2] * (b[0] * c[1] - b[1] * c[0]);
    };
    const double whole = signed_measure(P);
    double mn = 1e300;
    for (int a = 0; a < nv; ++a) {
        double Q[4][3];
        std::memcpy(Q, P, sizeof(Q));
        for (int c = 0; c < m.d; ++c) Q[a][c] = x[c];
        lam[a] = signed_measure(Q) / whole;
        mn = std::min(mn, lam[a]);
    }
    return mn;
}

}  // namespace

namespace mlq {

// The simplex of a general mesh holding each point and the point's
// barycentric coordinates there: the first simplex, in element order, that
// contains the point (bucket grid over the node bounding box); a point in
// no simplex takes the first simplex whose smallest coordinate is within
// 1e-12 of the largest over all simplices.  elem: np, lam: np x (dim + 1).
int locate_points(int dim, int64_t n, const double *xyz, int64_t ne, const int32_t *conn, int64_t np,
                  const double *pts, int64_t *elem, double *lam_out)
{
    if (!mesh_ok(dim, n, xyz, ne, conn) || np < 0 || (np > 0 && (!pts || !elem || !lam_out))) return MLQ_EINVAL;
    const SimplexMesh m{dim, n, ne, xyz, conn};
    const int nv = dim + 1;
    // buckets: a uniform grid over the node bounding box; each lists, in
    // element order, the simplices whose bounding box meets it
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int c = 0; c < dim; ++c) lo[c] = hi[c] = xyz[c];
    for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c < dim; ++c) {
            lo[c] = std::min(lo[c], xyz[i * dim + c]);
            hi[c] = std::max(hi[c], xyz[i * dim + c]);
        }
    const int g = std::max(1, std::min(512, (int)std::lround(std::pow((double)ne / 6.0, 1.0 / dim))));
    double inv[3] = {1, 1, 1};
    for (int c = 0; c < dim; ++c) inv[c] = hi[c] > lo[c] ? g / (hi[c] - lo[c]) : 1.0;
    auto cell = [&](int c, double v) { return std::max(0, std::min(g - 1, (int)std::floor((v - lo[c]) * inv[c]))); };
    int64_t nb = 1;
    for (int c = 0; c < dim; ++c) nb *= g;
    std::vector<std::array<int, 6>> box((size_t)ne);
    std::vector<int64_t> bstart((size_t)nb + 1, 0);
    for (int64_t e = 0; e < ne; ++e) {
        std::array<int, 6> r{0, 0, 0, 0, 0, 0};
        for (int c = 0; c < dim; ++c) {
            double a = 1e300, b = -1e300;
            for (int q = 0; q < nv; ++q) {
                const double v = xyz[(int64_t)conn[e * nv + q] * dim + c];
                a = std::min(a, v);
                b = std::max(b, v);
            }
            r[2 * c] = cell(c, a);
            r[2 * c + 1] = cell(c, b);
        }
        box[(size_t)e] = r;
        for (int z = r[4]; z <= r[5]; ++z)
            for (int y = r[2]; y <= r[3]; ++y)
                for (int x = r[0]; x <= r[1]; ++x) ++bstart[(size_t)(x + (int64_t)g * (y + (int64_t)g * z)) + 1];
    }
    for (int64_t b = 0; b < nb; ++b) bstart[(size_t)b + 1] += bstart[(size_t)b];
    std::vector<int32_t> blist((size_t)bstart[(size_t)nb]);
    {
        std::vector<int64_t> fill(bstart.begin(), bstart.end() - 1);
        for (int64_t e = 0; e < ne; ++e) {
            const std::array<int, 6> &r = box[(size_t)e];
            for (int z = r[4]; z <= r[5]; ++z)
                for (int y = r[2]; y <= r[3]; ++y)
                    for (int x = r[0]; x <= r[1]; ++x)
                        blist[(size_t)fill[(size_t)(x + (int64_t)g * (y + (int64_t)g * z))]++] = (int32_t)e;
        }
    }
    parallel_chunks((np + 1023) / 1024, [&](int64_t c) {
        const int64_t p0 = c * 1024, p1 = std::min(np, p0 + 1024);
        for (int64_t p = p0; p < p1; ++p) {
            const double *x = pts + p * dim;
            int64_t b = 0, stride = 1;
            for (int cc = 0; cc < dim; ++cc) {
                b += cell(cc, x[cc]) * stride;
                stride *= g;
            }
            double lam[4], best_lam[4] = {0, 0, 0, 0};
            int64_t best = -1;
            // a simplex containing x meets x's bucket: the first of them
            for (int64_t t = bstart[(size_t)b]; t < bstart[(size_t)b + 1] && best < 0; ++t) {
                const int64_t e = blist[(size_t)t];
                if (barycentric_of(m, e, x, lam) >= -1e-12) {
                    best = e;
                    std::memcpy(best_lam, lam, sizeof(lam));
                }
            }
            if (best < 0) {
                // in no simplex: the first simplex whose smallest coordinate is
                // within 1e-12 of the largest over all simplices
                double best_min = -1e300;
                for (int64_t e = 0; e < ne; ++e) best_min = std::max(best_min, barycentric_of(m, e, x, lam));
                for (int64_t e = 0; e < ne && best < 0; ++e)
                    if (barycentric_of(m, e, x, lam) >= best_min - 1e-12) {
                        best = e;
                        std::memcpy(best_lam, lam, sizeof(lam));
                    }
            }
            elem[p] = best;
            for (int a = 0; a < nv; ++a) lam_out[p * nv + a] = best_lam[a];
        }
    });
    return MLQ_OK;
}

}  // namespace mlq

namespace {

int p1_at_points(int dim, int64_t n, const double *xyz, int64_t ne, const int32_t *conn, int K, const double *f,
                 int64_t np, const double *pts, double *out)
{
    if (!mesh_ok(dim, n, xyz, ne, conn) || K < 1 || np < 0 || (np > 0 && (!f || !pts || !out))) return MLQ_EINVAL;
    const int nv = dim + 1;
    std::vector<int64_t> elem((size_t)std::max<int64_t>(np, 1));
    std::vector<double> lam((size_t)std::max<int64_t>(np, 1) * nv);
    const int st = mlq::locate_points(dim, n, xyz, ne, conn, np, pts, elem.data(), lam.data());
    if (st != MLQ_OK) return st;
    parallel_chunks((np + 1023) / 1024, [&](int64_t c) {
        const int64_t p0 = c * 1024, p1 = std::min(np, p0 + 1024);
        for (int64_t p = p0; p < p1; ++p)
            for (int k = 0; k < K; ++k) {
                double v = 0.0;
                for (int a = 0; a < nv; ++a)
                    v += lam[(size_t)p * nv + a] * f[(int64_t)conn[elem[(size_t)p] * nv + a] * K + k];
                out[p * K + k] = v;
            }
    });
    return MLQ_OK;
}

int build_kl(int dim, const int32_t *dims, const double *lengths, double sigma2, double ell, int K,
             double *modes_out, double *lambda_out)
{
    if ((dim != 2 && dim != 3) || !dims || !modes_out || !lambda_out || !(sigma2 > 0.0) || !(ell > 0.0))
        return MLQ_EINVAL;
    if (dim == 3) {
        const double Lx = lengths ? lengths[0] : 1.0, Ly = lengths ? lengths[1] : 1.0,
                     Lz = lengths ? lengths[2] : 0.25;
        if (dims[0] < 2 || dims[1] < 2 || dims[2] < 2 || !(Lx > 0.0 && Ly > 0.0 && Lz > 0.0)) return MLQ_EINVAL;
        Grid3h g{dims[0], dims[1], dims[2], Lx / (dims[0] - 1), Ly / (dims[1] - 1), Lz / (dims[2] - 1)};
        const int64_t n = g.n();
        if (K < 1 || K > n || K > 4096) return MLQ_EINVAL;
        auto coord = [&](int64_t t, double *x) {
            x[0] = g.hx * (double)(t % g.mx);
            x[1] = g.hy * (double)((t / g.mx) % g.my);
            x[2] = g.hz * (double)(t / ((int64_t)g.mx * g.my));
        };
        auto mass = [&](const double *x, double *y, int ncol) { mass_apply3(g, x, y, ncol); };
        return build_kl_nodes(n, coord, mass, sigma2, ell, K, modes_out, lambda_out);
    }
    const int m = dims[0];
    if (m < 2) return MLQ_EINVAL;
    const int64_t n = (int64_t)m * m;
    if (K < 1 || K > n || K > 4096) return MLQ_EINVAL;
    Grid2 g{m, 1.0 / (m - 1)};
    auto coord = [&](int64_t t, double *x) {
        x[0] = g.x(t);
        x[1] = g.y(t);
        x[2] = 0.0;
    };
    auto mass = [&](const double *x, double *y, int ncol) { mass_apply(g, x, y, ncol); };
    return build_kl_nodes(n, coord, mass, sigma2, ell, K, modes_out, lambda_out);
}

int centroid_table(int dim, const int32_t *fine_dims, const double *modes_f, int K, const int32_t *coarse_dims,
                   double *phi_out)
{
    if ((dim != 2 && dim != 3) || !fine_dims || !coarse_dims || !modes_f || !phi_out || K < 1) return MLQ_EINVAL;
    if (dim == 3) {
        // the box is the same on both meshes; lengths drop out of the
        // node-index arithmetic, so unit spacing per axis is used
        for (int a = 0; a < 3; ++a)
            if (fine_dims[a] < 2 || coarse_dims[a] < 2) return MLQ_EINVAL;
        Grid3h gf{fine_dims[0], fine_dims[1], fine_dims[2], 1.0 / (fine_dims[0] - 1), 1.0 / (fine_dims[1] - 1),
                  1.0 / (fine_dims[2] - 1)};
        const double H[3] = {1.0 / (coarse_dims[0] - 1), 1.0 / (coarse_dims[1] - 1), 1.0 / (coarse_dims[2] - 1)};
        const int64_t cells_per_plane = (int64_t)(coarse_dims[0] - 1) * (coarse_dims[1] - 1);
        parallel_chunks(coarse_dims[2] - 1, [&](int64_t kc) {
            const int k = (int)kc;
            int64_t e = 6 * cells_per_plane * k;
            for (int j = 0; j + 1 < coarse_dims[1]; ++j)
                for (int i = 0; i + 1 < coarse_dims[0]; ++i)
                    for (int s = 0; s < 6; ++s, ++e) {
                        // centroid: 3/4, 2/4, 1/4 of a cell along the first, second, third step
                        double p[3] = {(double)i, (double)j, (double)k};
                        for (int q = 0; q < 3; ++q) p[kPerm[s][q]] += (3.0 - q) / 4.0;
                        p1_at3(gf, modes_f, K, p[0] * H[0], p[1] * H[1], p[2] * H[2], phi_out + e * K);
                    }
        });
        return MLQ_OK;
    }
    const int mf = fine_dims[0], mc = coarse_dims[0];
    if (mf < 2 || mc < 2) return MLQ_EINVAL;
    Grid2 gf{mf, 1.0 / (mf - 1)};
    const double H = 1.0 / (mc - 1);
    parallel_chunks(mc - 1, [&](int64_t jc) {
        const int j = (int)jc;
        for (int i = 0; i + 1 < mc; ++i) {
            const int64_t c = i + (int64_t)(mc - 1) * j;
            // centroids of the lower and upper triangle of square (i, j)
            const double xl = (i + 2.0 / 3.0) * H, yl = (j + 1.0 / 3.0) * H;
            const double xu = (i + 1.0 / 3.0) * H, yu = (j + 2.0 / 3.0) * H;
            p1_at(gf, modes_f, K, xl, yl, phi_out + (2 * c) * K);
            p1_at(gf, modes_f, K, xu, yu, phi_out + (2 * c + 1) * K);
        }
    });
    return MLQ_OK;
}

// host allocation or thread creation failures become status codes
template <typename F>
int guarded(F &&f)
{
    try {
        return f();
    } catch (const std::bad_alloc &) {
        return MLQ_ENOMEM;
    } catch (...) {
        return MLQ_ENOMEM;
    }
}

}  // namespace

extern "C" {

int mlq_build_kl(int dim, const int32_t *dims, const double *lengths, double sigma2, double ell, int K,
                 double *modes_out, double *lambda_out)
{
    return guarded([&] { return build_kl(dim, dims, lengths, sigma2, ell, K, modes_out, lambda_out); });
}

int mlq_centroid_table(int dim, const int32_t *fine_dims, const double *modes_f, int K, const int32_t *coarse_dims,
                       double *phi_out)
{
    return guarded([&] { return centroid_table(dim, fine_dims, modes_f, K, coarse_dims, phi_out); });
}

int mlq_build_kl_mesh(int dim, int64_t n, const double *xyz, int64_t ne, const int32_t *conn, double sigma2,
                      double ell, int K, double *modes_out, double *lambda_out)
{
    return guarded([&] { return build_kl_mesh(dim, n, xyz, ne, conn, sigma2, ell, K, modes_out, lambda_out); });
}

int mlq_p1_at_points(int dim, int64_t n, const double *xyz, int64_t ne, const int32_t *conn, int K, const double *f,
                     int64_t np, const double *pts, double *out)
{
    return guarded([&] { return p1_at_points(dim, n, xyz, ne, conn, K, f, np, pts, out); });
}

}  // extern "C"
