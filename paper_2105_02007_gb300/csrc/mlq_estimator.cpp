// mlq_estimator.cpp -- host helpers for the multilevel estimators.
//
// Sample allocation for eq. StandardML with Monte Carlo rules: the estimator's
// statistical error is RMSE_stat^2 = sum_l V_l / N_l (V_l the variance of the
// level difference Y_l, N_l its samples) and its cost sum_l N_l C_l.  The
// numbers of samples that minimise the cost subject to RMSE_stat <= eps are,
// by a Lagrange multiplier, N_l = eps^-2 sqrt(V_l / C_l) sum_k sqrt(V_k C_k),
// then rounded up.
#include "mlq.h"

#include <cmath>
#include <cstdint>

extern "C" int mlq_mlmc_allocation(int L, const double *var, const double *cost, double eps, int64_t nmin,
                                   int64_t *N_out)
{
    if (L < 0 || !var || !cost || !N_out || !(eps > 0.0) || nmin < 1) return MLQ_EINVAL;
    double sum = 0.0;
    for (int l = 0; l <= L; ++l) {
        if (!(var[l] >= 0.0) || !(cost[l] > 0.0) || !std::isfinite(var[l]) || !std::isfinite(cost[l]))
            return MLQ_EINVAL;
        sum += std::sqrt(var[l] * cost[l]);
    }
    for (int l = 0; l <= L; ++l) {
        const double n = std::ceil(std::sqrt(var[l] / cost[l]) * sum / (eps * eps));
        if (!(n < 4.0e18)) return MLQ_EINVAL;
        N_out[l] = n > (double)nmin ? (int64_t)n : nmin;
    }
    return MLQ_OK;
}

// Time quantities of interest (the action potential u(x_0, t) of Sec. 2.4):
// a trace on level l holds u at the block ends t_n = n dt_l, n = 0..nt, and
// is read as the function linear in time between them.  The level difference
// of eq. StandardML for such a QoI needs the coarse trace on the fine time
// grid (dt_l = dt_{l-1} / 2): the tensor-product intergrid transfer of
// Sec. 5, here in time alone, is linear interpolation, which keeps the coarse
// values at the even fine times and puts the mean of the two neighbours at
// the odd ones.
extern "C" int mlq_trace_prolong(int nt_coarse, const double *u_c, double *u_f)
{
    if (nt_coarse < 0 || !u_c || !u_f) return MLQ_EINVAL;
    for (int n = 0; n <= nt_coarse; ++n) {
        u_f[2 * n] = u_c[n];
        if (n < nt_coarse) u_f[2 * n + 1] = 0.5 * (u_c[n] + u_c[n + 1]);
    }
    return MLQ_OK;
}

// Norms on (0, T) of the function e linear between e_n at t_n = n T / nt
// (eq. point-error with q = 0 and q = 1): ||e||_{L2}^2 = sum over the steps
// of dt (e_n^2 + e_n e_{n+1} + e_{n+1}^2) / 3, the H1 seminorm squared
// sum (e_{n+1} - e_n)^2 / dt, and ||e||_{H1}^2 their sum.
extern "C" int mlq_time_norms(int nt, double T, const double *e, double *l2, double *h1)
{
    if (nt < 1 || !(T > 0.0) || !e) return MLQ_EINVAL;
    const double dt = T / nt;
    double a = 0.0, b = 0.0;
    for (int n = 0; n < nt; ++n) {
        a += dt * (e[n] * e[n] + e[n] * e[n + 1] + e[n + 1] * e[n + 1]) / 3.0;
        const double d = e[n + 1] - e[n];
        b += d * d / dt;
    }
    if (l2) *l2 = std::sqrt(a);
    if (h1) *h1 = std::sqrt(a + b);
    return MLQ_OK;
}

// eq. StandardML with Monte Carlo rules from per-sample level differences:
// level l contributes the sample mean of Y_l (N[l] values y[l][0..N[l]-1],
// summed in index order), its unbiased sample variance (two passes), and
// RMSE_stat = sqrt(sum_l V_l / N_l).  Summing in index order makes the
// result independent of how the samples were split over processes, as long
// as they are gathered back in index order.
extern "C" int mlq_mlmc_combine(int L, const int64_t *N, const double *const *y, double *mean_out, double *var_out,
                                double *rmse_out)
{
    if (L < 0 || !N || !y || !mean_out) return MLQ_EINVAL;
    for (int l = 0; l <= L; ++l)
        if (N[l] < 1 || !y[l]) return MLQ_EINVAL;
    double est = 0.0, mse = 0.0;
    for (int l = 0; l <= L; ++l) {
        const int64_t n = N[l];
        double m = 0.0;
        for (int64_t i = 0; i < n; ++i) m += y[l][i];
        m /= (double)n;
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) s += (y[l][i] - m) * (y[l][i] - m);
        const double v = n > 1 ? s / (double)(n - 1) : 0.0;
        est += m;
        mse += v / (double)n;
        if (var_out) var_out[l] = v;
    }
    *mean_out = est;
    if (rmse_out) *rmse_out = std::sqrt(mse);
    return MLQ_OK;
}

// ---------------------------------------------------------------------------
// Field-valued quantities of interest (the state v_h(T) of a sample, Sec. 2.4
// with a field functional; the intergrid transfer of Sec. 4 / Sec. 5 between
// nested levels).
// ---------------------------------------------------------------------------
namespace {

// axis of step q of Kuhn tetrahedron s (the mesh convention of mlq.h: the
// six axis orders (x,y,z), (x,z,y), (y,x,z), (y,z,x), (z,x,y), (z,y,x))
int kuhn_step_axis(int s, int q)
{
    static const int ax[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    return ax[s][q];
}

bool dims_ok(int dim, const int32_t *dims)
{
    if (!dims || (dim != 2 && dim != 3)) return false;
    for (int a = 0; a < (dim == 2 ? 1 : 3); ++a)
        if (dims[a] < 2 || dims[a] > 65536) return false;
    return true;
}

}  // namespace

// The P1 interpolant of a coarse field on the nested fine mesh (red
// refinement in 2D, regular refinement of the Kuhn cubes in 3D: 2m - 1 nodes
// per axis).  A fine node at a coarse node keeps its value; a fine node
// halving a coarse edge takes the mean of the edge's two ends.  In 2D the
// edges are the x, y and (1,1)-diagonal ones of the triangulation; in 3D the
// seven directions with components in {0, 1} (every such segment of a cube is
// an edge of its Kuhn tetrahedra).
extern "C" int mlq_field_prolong(int dim, const int32_t *coarse_dims, const double *vc, double *vf)
{
    if (!dims_ok(dim, coarse_dims) || !vc || !vf) return MLQ_EINVAL;
    if (dim == 2) {
        const int64_t mc = coarse_dims[0], mf = 2 * mc - 1;
        for (int64_t J = 0; J < mf; ++J)
            for (int64_t I = 0; I < mf; ++I) {
                const int64_t i = I / 2, j = J / 2, a = I & 1, b = J & 1;
                const double c0 = vc[i + mc * j];
                vf[I + mf * J] = (a | b) ? 0.5 * (c0 + vc[(i + a) + mc * (j + b)]) : c0;
            }
        return MLQ_OK;
    }
    const int64_t cx = coarse_dims[0], cy = coarse_dims[1], cz = coarse_dims[2];
    const int64_t fx = 2 * cx - 1, fy = 2 * cy - 1, fz = 2 * cz - 1;
    for (int64_t K = 0; K < fz; ++K)
        for (int64_t J = 0; J < fy; ++J)
            for (int64_t I = 0; I < fx; ++I) {
                const int64_t i = I / 2, j = J / 2, k = K / 2, a = I & 1, b = J & 1, c = K & 1;
                const double c0 = vc[i + cx * (j + cy * k)];
                vf[I + fx * (J + fy * K)] =
                    (a | b | c) ? 0.5 * (c0 + vc[(i + a) + cx * ((j + b) + cy * (k + c))]) : c0;
            }
    return MLQ_OK;
}

// ||e||_{L2(D)} and ||e||_{H1(D)} of the P1 function with nodal values e on
// a structured level (dims and lengths as in mlq_add_level; 2D: the unit
// square), summed element by element: sum |T| (sum_a e_a^2 + (sum_a e_a)^2)
// / ((d + 1)(d + 2)) (the consistent mass form) and sum |T| |grad e_h|^2.
extern "C" int mlq_field_norms(int dim, const int32_t *dims, const double *lengths, const double *e, double *l2,
                               double *h1)
{
    if (!dims_ok(dim, dims) || !e) return MLQ_EINVAL;
    double m2 = 0.0, g2 = 0.0;
    if (dim == 2) {
        const int64_t m = dims[0];
        const double h = 1.0 / (double)(m - 1), area = 0.5 * h * h;
        for (int64_t j = 0; j + 1 < m; ++j)
            for (int64_t i = 0; i + 1 < m; ++i) {
                const double u00 = e[i + m * j], u10 = e[i + 1 + m * j], u11 = e[i + 1 + m * (j + 1)],
                             u01 = e[i + m * (j + 1)];
                // lower (i,j)(i+1,j)(i+1,j+1): grad = ((u10-u00)/h, (u11-u10)/h)
                // upper (i,j)(i+1,j+1)(i,j+1): grad = ((u11-u01)/h, (u01-u00)/h)
                const double tri[2][3] = {{u00, u10, u11}, {u00, u11, u01}};
                const double gx[2] = {(u10 - u00) / h, (u11 - u01) / h}, gy[2] = {(u11 - u10) / h, (u01 - u00) / h};
                for (int t = 0; t < 2; ++t) {
                    const double s = tri[t][0] + tri[t][1] + tri[t][2];
                    m2 += area / 12.0 *
                          (tri[t][0] * tri[t][0] + tri[t][1] * tri[t][1] + tri[t][2] * tri[t][2] + s * s);
                    g2 += area * (gx[t] * gx[t] + gy[t] * gy[t]);
                }
            }
    } else {
        const int64_t mx = dims[0], my = dims[1], mz = dims[2];
        const double L[3] = {lengths ? lengths[0] : 1.0, lengths ? lengths[1] : 1.0, lengths ? lengths[2] : 0.25};
        const double h[3] = {L[0] / (mx - 1), L[1] / (my - 1), L[2] / (mz - 1)};
        const double vol = h[0] * h[1] * h[2] / 6.0;
        for (int64_t k = 0; k + 1 < mz; ++k)
            for (int64_t j = 0; j + 1 < my; ++j)
                for (int64_t i = 0; i + 1 < mx; ++i)
                    for (int s = 0; s < 6; ++s) {
                        // vertices: the path from (i,j,k) stepping along the axes of s
                        int64_t c[3] = {i, j, k};
                        double u[4];
                        u[0] = e[c[0] + mx * (c[1] + my * c[2])];
                        double grad[3];
                        for (int q = 0; q < 3; ++q) {
                            const int ax = kuhn_step_axis(s, q);
                            ++c[ax];
                            u[q + 1] = e[c[0] + mx * (c[1] + my * c[2])];
                            grad[ax] = (u[q + 1] - u[q]) / h[ax];
                        }
                        const double sum = u[0] + u[1] + u[2] + u[3];
                        m2 += vol / 20.0 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2] + u[3] * u[3] + sum * sum);
                        g2 += vol * (grad[0] * grad[0] + grad[1] * grad[1] + grad[2] * grad[2]);
                    }
    }
    if (l2) *l2 = std::sqrt(m2);
    if (h1) *h1 = std::sqrt(m2 + g2);
    return MLQ_OK;
}

// eq. PimpedML with nested sample rules (the non-nested levels of Sec. 5.4):
//   QoI = sum_{l=0}^{L} (Q_l - Q_{l-1})(F_{L-l}),  Q_{-1} = 0,
// Q_l the mean over the first N_l points (N_0 <= N_1 <= ... <= N_L).  Term l
// needs the QoI on one mesh only (mesh L-l) at the first N_l points:
// F[l][0..N_l-1].  Means are summed in index order.
extern "C" int mlq_pimped_ml_combine(int L, const int64_t *N, const double *const *F, double *est_out)
{
    if (L < 0 || !N || !F || !est_out) return MLQ_EINVAL;
    for (int l = 0; l <= L; ++l) {
        if (N[l] < 1 || !F[l]) return MLQ_EINVAL;
        if (l > 0 && N[l] < N[l - 1]) return MLQ_EINVAL;
    }
    double est = 0.0;
    for (int l = 0; l <= L; ++l) {
        double a = 0.0;
        for (int64_t i = 0; i < N[l]; ++i) a += F[l][i];
        est += a / (double)N[l];
        if (l > 0) {
            double b = 0.0;
            for (int64_t i = 0; i < N[l - 1]; ++i) b += F[l][i];
            est -= b / (double)N[l - 1];
        }
    }
    *est_out = est;
    return MLQ_OK;
}
