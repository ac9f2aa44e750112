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
