// mlq_points.cuh -- point quantities of interest fused into the block loops
// of the solvers (argument block shared by the host runtime and the kernels).
#pragma once

#include <cstddef>
#include <cuda_runtime.h>

namespace mlq {

// Point QoIs of Sec. 2.4, fused into the block loop of every solver: the
// action potential u(x_p, t_n) at a few points x_p after every block (n = 0:
// the initial state) and the activation time a(x_p) = min{t : u(x_p, t) >=
// u_th}, with u(x_p, .) linear in time between block ends (-1: never
// reached).  u(x_p, t) is the P1 value, sum_a w_a v[node_a] over the simplex
// holding x_p.  One thread per point (rank 0 of the sample's cluster) reads
// v through L2 after the block's last cluster barrier.
constexpr int kMaxPoints = 32;

struct PointArgs {
    int npts;            // 0: none; at most kMaxPoints
    const int *node;     // [npts][4] simplex nodes (2D: the 4th repeats the 1st with weight 0)
    const double *w;     // [npts][4] barycentric weights
    double u_th;         // activation threshold
    double *trace;       // [S][npts][nsteps + 1], or null
    double *act;         // [S][npts], or null
};

struct PointState {
    double uprev = 0.0;
    int n = 0;
    bool hit = false;
};

__device__ __forceinline__ void point_record(const PointArgs &pa, int sample, int nsteps, double dt, const double *v,
                                             PointState &ps)
{
    const int p = threadIdx.x;
    const int *nd = pa.node + 4 * p;
    const double *wt = pa.w + 4 * p;
    double u = 0.0;
#pragma unroll
    for (int a = 0; a < 4; ++a) u += wt[a] * __ldcg(v + nd[a]);
    if (pa.trace) pa.trace[((size_t)sample * pa.npts + p) * (nsteps + 1) + ps.n] = u;
    if (!ps.hit && u >= pa.u_th) {
        ps.hit = true;
        const double t = ps.n == 0 ? 0.0 : dt * ((double)(ps.n - 1) + (pa.u_th - ps.uprev) / (u - ps.uprev));
        if (pa.act) pa.act[(size_t)sample * pa.npts + p] = t;
    }
    ps.uprev = u;
    ++ps.n;
}

// after the block loop: entries of a sample that stopped early are NaN, and
// a point that never reached u_th has a(x_p) = -1
__device__ __forceinline__ void point_finish(const PointArgs &pa, int sample, int nsteps, const PointState &ps)
{
    const int p = threadIdx.x;
    if (pa.trace)
        for (int n = ps.n; n <= nsteps; ++n)
            pa.trace[((size_t)sample * pa.npts + p) * (nsteps + 1) + n] = __longlong_as_double(0x7ff8000000000000LL);
    if (pa.act && !ps.hit) pa.act[(size_t)sample * pa.npts + p] = -1.0;
}

}  // namespace mlq
