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
