// mlq_mesh_solver.cuh -- device-resident time-block solver for levels on
// general tetrahedral meshes (the non-nested hierarchies of Sec. 4 and the
// ventricle of Sec. 5.4).
//
// One sample per group of CTAs (a cluster of CS CTAs, or G CTAs of a
// cooperative launch when a sample wants more CTAs than a cluster holds;
// mlq_groups.cuh); CTA `rank` of the group owns the CSR rows
// [n rank / size, n (rank + 1) / size).  Every vector lives in global memory
// (sample-major); values of other CTAs' rows are read through L2 after a
// group barrier.  Per time block (Sec. 3.1-3.3, as for the structured
// levels):
//   y = v + dt R(v, w), w += dt eps (v - gam w)              (own rows)
//   b = M y, r = b - A v in FP64                             (CSR products)
//   inner solve: Jacobi-PCG in Chronopoulos-Gear form (one cluster reduction
//   per iteration) on A d = r / ||r|| in the inner precision TI, v += ||r|| d;
//   the mixed path repeats while ||b - A v|| > rtol ||b|| (iterative
//   refinement in FP64), the FP64 path solves to that tolerance in one sweep
//   Q = m^T v with m = M 1.
// The whole block loop runs in one launch: no host synchronisation per
// iteration or per block.
#pragma once

#include "mlq_groups.cuh"
#include "mlq_kernels.cuh"

namespace mlq {

template <typename TI>
struct MeshArgs {
    int n, S;
    int64_t nnz;
    const int64_t *rp;            // [n + 1] CSR rows
    const int32_t *ci;            // [nnz] columns
    const int64_t *diag;          // [n] position of the diagonal in its row
    const double *mval;           // [nnz] consistent mass
    const double *lump;           // [n] m = M 1
    const double *A64;            // [S][nnz] M + dt K(D) in FP64
    const TI *Ai;                 // [S][nnz] the same in the inner precision
    double dt;
    int nsteps;
    double a, eps, gam;           // FHN
    double rtol_out, rtol_in;
    int max_iter, max_sweeps;
    const double *v0, *w0;        // [n]; w0 may be null (0)
    double *v, *w, *b, *y;        // [S][n] FP64 state, load, reaction
    TI *r, *u, *wv, *s, *p, *x, *dinv;   // [S][n] inner vectors
    double *q;                    // [S]
    int32_t *iters, *status;      // [S]
    PointArgs pq;                 // point QoIs (npts = 0: none)
};

// Rows of a CSR product handled by groups of 8 lanes: each group takes two
// rows per round (the loads of both in flight together: the gather of x is
// bound by L2 latency), its lanes the entries t = rp[row] + lane, + 8, ...;
// the partial sums meet by butterfly inside the group.  Every lane of a warp
// runs the same number of rounds (a row past the band contributes zeros), so
// the shuffles see the whole warp.  The matrix goes through the read-only
// path (it is not written during the solve), x through L2 (other CTAs write
// it between cluster barriers).  f(row, value) consumes a row on lane 0 of
// its group.
template <typename TV, typename TX, typename F>
__device__ __forceinline__ void csr_rows(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                         const TV *__restrict__ val, const TX *x, int r0, int r1, F &&f)
{
    const int lane8 = threadIdx.x & 7, grp = threadIdx.x >> 3, ngrp = blockDim.x >> 3;
    const int rounds = (r1 - r0 + 2 * ngrp - 1) / (2 * ngrp);
    for (int k = 0; k < rounds; ++k) {
        const int ra = r0 + 2 * k * ngrp + grp, rb = ra + ngrp;
        TV acca = (TV)0, accb = (TV)0;
        int64_t ta = 0, ea = 0, tb = 0, eb = 0;
        if (ra < r1) {
            ta = __ldg(rp + ra) + lane8;
            ea = __ldg(rp + ra + 1);
        }
        if (rb < r1) {
            tb = __ldg(rp + rb) + lane8;
            eb = __ldg(rp + rb + 1);
        }
        while (ta < ea || tb < eb) {
            const bool ha = ta < ea, hb = tb < eb;
            const int32_t ca = ha ? __ldg(ci + ta) : 0, cb = hb ? __ldg(ci + tb) : 0;
            const TV va = ha ? __ldg(val + ta) : (TV)0, vb = hb ? __ldg(val + tb) : (TV)0;
            const TX xa = ha ? __ldcg(x + ca) : (TX)0, xb = hb ? __ldcg(x + cb) : (TX)0;
            acca += va * (TV)xa;
            accb += vb * (TV)xb;
            ta += 8;
            tb += 8;
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
            acca += __shfl_xor_sync(0xffffffffu, acca, o);
            accb += __shfl_xor_sync(0xffffffffu, accb, o);
        }
        if (lane8 == 0) {
            if (ra < r1) f(ra, acca);
            if (rb < r1) f(rb, accb);
        }
    }
}

// PTS: record the point QoIs of g.pq.  A separate instantiation, so that
// the solves without points carry none of the point state in registers (at
// the 64-register cap of 512 threads x 2 CTAs it adds spills).
template <typename TI, typename Grp, bool PTS>
__global__ void __launch_bounds__(512, 2) mesh_slab_kernel(MeshArgs<TI> g, Grp grp)
{
    __shared__ double wsl[32][4];
    __shared__ double csl[2][4];
    __shared__ Ctl ctl;
    const int rank = grp.rank(), gsz = grp.size();
    const int sample = grp.sample();
    const int n = g.n, tid = threadIdx.x, nt = blockDim.x;
    const int r0 = (int)(((int64_t)n * rank) / gsz), r1 = (int)(((int64_t)n * (rank + 1)) / gsz);
    constexpr bool mixed = sizeof(TI) == 4;

    const size_t so = (size_t)sample * n;
    const double *A64 = g.A64 + (size_t)sample * g.nnz;
    const TI *Ai = g.Ai + (size_t)sample * g.nnz;
    double *v = g.v + so, *w = g.w + so, *b = g.b + so, *y = g.y + so;
    TI *R = g.r + so, *U = g.u + so, *W = g.wv + so, *Sv = g.s + so, *P = g.p + so, *X = g.x + so;
    TI *Dinv = g.dinv + so;

    for (int i = r0 + tid; i < r1; i += nt) {
        v[i] = g.v0[i];
        w[i] = g.w0 ? g.w0[i] : 0.0;
        Dinv[i] = (TI)1 / Ai[g.diag[i]];
    }
    grp.sync();
    PointState pst;
    const bool pth = PTS && rank == 0 && tid < g.pq.npts;   // point QoI threads
    if constexpr (PTS) {
        if (pth) point_record(g.pq, sample, g.nsteps, g.dt, v, pst);
    }

    int par = 0;
    int64_t total_iters = 0;
    int32_t status = S_CONVERGED;
    const double dt = g.dt;
    for (int step = 0; step < g.nsteps; ++step) {
        // ---- block load (own rows): y = v + dt R(v, w), w update
        for (int i = r0 + tid; i < r1; i += nt) {
            const double vv = v[i], ww = w[i];
            y[i] = vv + dt * reaction<mixed>(vv, ww, g.a);
            w[i] = ww + dt * g.eps * recovery<mixed>(vv, ww, g.gam);
        }
        grp.sync();
        // ---- b = M y (FP64), then r = b - A v (FP64) into R
        {
            double acc[2] = {0.0, 0.0};
            csr_rows(g.rp, g.ci, g.mval, y, r0, r1, [&](int i, double bb) {
                b[i] = bb;
                acc[0] += bb * bb;
            });
            __syncthreads();   // b of the CTA's rows written before the residual reads them
            csr_rows(g.rp, g.ci, A64, v, r0, r1, [&](int i, double av) {
                const double rr = b[i] - av;
                R[i] = (TI)rr;
                acc[1] += rr * rr;
            });
            grp.template reduce<2>(acc, wsl, csl, par, [&](double(&t)[2]) {
                ctl.s0 = t[0];
                ctl.s1 = t[1];
            });
            par ^= 1;
        }
        const double bnorm2 = ctl.s0;
        double rnorm2 = ctl.s1;
        if (!(isfinite(bnorm2) && isfinite(rnorm2))) {
            status = S_NONFINITE;
            break;
        }
        const double tol_out2 = g.rtol_out * g.rtol_out * bnorm2;
        bool nonfinite = false, solved = false;
        const int sweeps = mixed ? g.max_sweeps : 1;
        for (int sweep = 0; sweep < sweeps; ++sweep) {
            if (sweep > 0) {
                double racc[1] = {0.0};
                csr_rows(g.rp, g.ci, A64, v, r0, r1, [&](int i, double av) {
                    const double rr = b[i] - av;
                    R[i] = (TI)rr;
                    racc[0] += rr * rr;
                });
                grp.template reduce<1>(racc, wsl, csl, par, [&](double(&t)[1]) { ctl.s1 = t[0]; });
                par ^= 1;
                rnorm2 = ctl.s1;
                if (!isfinite(rnorm2)) {
                    nonfinite = true;
                    break;
                }
            }
            if (rnorm2 <= tol_out2) {
                solved = true;
                break;
            }
            const double rnorm = sqrt(rnorm2);
            const TI rscale = (TI)(1.0 / rnorm);
            // inner target relative to the normalised start: rtol_in, or half
            // of what the outer test still needs when that is looser; the FP64
            // path solves to the outer target in its one sweep
            const double need = tol_out2 / rnorm2;
            const double tol_in2 = mixed ? fmax(g.rtol_in * g.rtol_in, 0.25 * need) : need;

            // init: r0 normalised, u0 = D^-1 r0, x = p = s = 0
            for (int i = r0 + tid; i < r1; i += nt) {
                const TI rv = R[i] * rscale;
                R[i] = rv;
                U[i] = Dinv[i] * rv;
                X[i] = (TI)0;
                P[i] = (TI)0;
                Sv[i] = (TI)0;
            }
            double gacc = 0.0, racc = 0.0;   // (r, u) and (r, r) of the iterate, thread partials
            for (int i = r0 + tid; i < r1; i += nt) {
                gacc += (double)(R[i] * U[i]);
                racc += (double)(R[i] * R[i]);
            }
            grp.sync();
            double gamma_prev = 1.0, eta_prev = 1.0;
            int it = 0;
            auto decide = [&](double gamma, double delta, double rr) {
                double alpha = 0.0, beta = 0.0;
                int code;
                if (!isfinite(rr) || !isfinite(gamma) || !isfinite(delta)) code = 3;
                else if (rr <= tol_in2) code = 1;
                else if (it >= g.max_iter) code = 2;
                else {
                    code = 0;
                    double eta = delta;
                    if (it > 0) {
                        beta = gamma / gamma_prev;
                        eta = delta - beta * beta * eta_prev;
                    }
                    alpha = gamma / eta;
                    gamma_prev = gamma;
                    eta_prev = eta;
                }
                ctl.alpha = alpha;
                ctl.beta = beta;
                ctl.code = code;
            };
            while (true) {
                // w = A u and (w, u); one reduction of (r, u), (w, u), (r, r)
                double pacc[3] = {gacc, 0.0, racc};
                csr_rows(g.rp, g.ci, Ai, U, r0, r1, [&](int i, TI wv) {
                    W[i] = wv;
                    pacc[1] += (double)(wv * U[i]);
                });
                grp.template reduce<3>(pacc, wsl, csl, par, [&](double(&t)[3]) { decide(t[0], t[1], t[2]); });
                par ^= 1;
                const int code = ctl.code;
                if (code != 0) {
                    if (code == 3) nonfinite = true;
                    else if (code == 2) status = status == S_CONVERGED ? S_MAXITER : status;
                    break;
                }
                const TI ta = (TI)ctl.alpha, tb = (TI)ctl.beta;
                // s = w + b s; p = u + b p; x += a p; r -= a s; u = D^-1 r
                gacc = 0.0;
                racc = 0.0;
                for (int i = r0 + tid; i < r1; i += nt) {
                    const TI ww = W[i], uu = U[i];
                    const TI sv = it == 0 ? ww : ww + tb * Sv[i];
                    const TI pv = it == 0 ? uu : uu + tb * P[i];
                    Sv[i] = sv;
                    P[i] = pv;
                    X[i] = X[i] + ta * pv;
                    const TI rv = R[i] - ta * sv;
                    R[i] = rv;
                    const TI un = Dinv[i] * rv;
                    U[i] = un;
                    gacc += (double)(rv * un);
                    racc += (double)(rv * rv);
                }
                ++it;
                grp.sync();
            }
            total_iters += it;
            if (nonfinite) break;
            for (int i = r0 + tid; i < r1; i += nt) v[i] = fma((double)X[i], rnorm, v[i]);
            grp.sync();
            if (!mixed) solved = true;
        }
        if (nonfinite) {
            status = S_NONFINITE;
            break;
        }
        if (!solved && status == S_CONVERGED) status = S_MAXITER;
        if constexpr (PTS) {
            if (pth) point_record(g.pq, sample, g.nsteps, dt, v, pst);
        }
    }
    if constexpr (PTS) {
        if (pth) point_finish(g.pq, sample, g.nsteps, pst);
    }

    double qacc[1] = {0.0};
    for (int i = r0 + tid; i < r1; i += nt) qacc[0] += g.lump[i] * v[i];
    grp.template reduce<1>(qacc, wsl, csl, par, [&](double(&t)[1]) { ctl.s0 = t[0]; });
    if (rank == 0 && tid == 0) {
        g.q[sample] = status == S_NONFINITE ? __longlong_as_double(0x7ff8000000000000LL) : ctl.s0;
        g.iters[sample] = (int32_t)(total_iters > 0x7fffffff ? 0x7fffffff : total_iters);
        g.status[sample] = status;
    }
    grp.sync();
}

}  // namespace mlq
