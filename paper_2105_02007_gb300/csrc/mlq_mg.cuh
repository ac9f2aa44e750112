// mlq_mg.cuh -- geometric multigrid preconditioner for the inner FP32 PCG.
//
// The nested hierarchy of the paper's Sec. 3.1 (red refinement, m_{c+1} =
// (m_c + 1) / 2 nodes per side) is used as a multigrid hierarchy for the block
// matrix A = M + dt K(theta):
//   * coarse operators are Galerkin, A_c = P^T A_{c-1} P with P the P1
//     interpolation.  For nested P1 spaces P^T M P is the coarse mass matrix
//     and P^T K P the coarse stiffness matrix whose conductivity on a coarse
//     triangle is the average of D over its four children (the coarse basis
//     gradients are constant on it), so A_c = M_c + dt K_c(Dbar_c), set up per
//     sample by mg_coarsen_kernel and mg_stencil_kernel;
//   * V(1,1) cycle, damped Jacobi (omega = 0.6) as pre- and post-smoother,
//     restriction P^T and interpolation P, a few damped Jacobi sweeps on the
//     coarsest level: a fixed symmetric positive definite operator, so it can
//     precondition CG.
// Every level is distributed over the cluster exactly like the fine grid: a
// CTA owns the rows J with 2J in its band of the finer level; halo rows come
// from the neighbouring CTAs' shared memory over DSMEM after a cluster
// barrier.
#pragma once

#include "mlq_kernels.cuh"

namespace mlq {

constexpr int kMgMaxLevels = 8;
constexpr float kMgOmega = 0.6f;

// Conductivity of an element as (d11, d12, d22).
struct D3 {
    float a, b, c;
};

// ---------------------------------------------------------------------------
// Level geometry shared by host and device.
//   m_c          nodes per side of level c
//   band(c,r)    rows [R0, R1) of level c owned by cluster rank r: level 0
//                splits the m rows evenly, level c takes the rows J with 2J in
//                the band of level c-1
// The hierarchy stops before a level where a band would be empty or m < 3.
// Shared layout per level (bytes, the same in every CTA): four stencil
// arrays D, E, N, NE (structure of arrays: conflict-free neighbour reads),
// each 1 + (rows_max + 1) * m floats (pad, row R0-1, own rows); tiles XA, XB,
// RR of 1 + (rows_max + 2) * m + 1 floats (pad, halo row R0-1, own rows,
// halo row R1, pad); BB, rows_max * m floats (own rows only).
// ---------------------------------------------------------------------------
struct MgLevelPlan {
    int m, rows_max;
    int off_d, off_e, off_n, off_ne, off_xa, off_xb, off_r, off_b;
    int csize, tile;
};

struct MgPlan {
    int nl;      // levels
    int total;   // bytes
    MgLevelPlan lv[kMgMaxLevels];
};

// per-sample stencils of the coarse levels (index 0 unused: the fine stencil
// is SolveArgs::Ai), each [S][5][m_c^2] FP32
struct MgPtrs {
    const float *A[kMgMaxLevels];
};

__host__ __device__ inline void mg_band(int m0, int cs, int rank, int c, int *R0, int *R1)
{
    int r0 = (int)(((int64_t)m0 * rank) / cs), r1 = (int)(((int64_t)m0 * (rank + 1)) / cs);
    for (int k = 0; k < c; ++k) {
        r0 = (r0 + 1) / 2;
        r1 = (r1 + 1) / 2;
    }
    *R0 = r0;
    *R1 = r1;
}

__host__ __device__ inline MgPlan mg_plan(int m0, int cs)
{
    MgPlan pl;
    pl.nl = 0;
    int off = 0;
    int m = m0;
    for (int c = 0; c < kMgMaxLevels; ++c) {
        int rmax = 0, rmin = 1 << 30;
        for (int r = 0; r < cs; ++r) {
            int a, b;
            mg_band(m0, cs, r, c, &a, &b);
            rmax = b - a > rmax ? b - a : rmax;
            rmin = b - a < rmin ? b - a : rmin;
        }
        if (c > 0 && (rmin < 1 || m < 3)) break;
        MgLevelPlan &L = pl.lv[c];
        L.m = m;
        L.rows_max = rmax;
        L.csize = 1 + (rmax + 1) * m;
        L.tile = 1 + (rmax + 2) * m + 1;
        const int cb = align16(L.csize * 4), tb = align16(L.tile * 4);
        L.off_d = off;
        L.off_e = off + cb;
        L.off_n = off + 2 * cb;
        L.off_ne = off + 3 * cb;
        off += 4 * cb;
        L.off_xa = off;
        L.off_xb = off + tb;
        L.off_r = off + 2 * tb;
        off += 3 * tb;
        L.off_b = off;
        off += align16(rmax * m * 4);
        pl.nl = c + 1;
        if (m < 5 || (m - 1) % 2) break;
        m = (m + 1) / 2;
    }
    pl.total = off;
    return pl;
}

template <int CS, int NPT>
__global__ void __launch_bounds__(NPT >= 12 ? 384 : 512, 1)
    slab_solve_mg_kernel(SolveArgs<float> g, MgPtrs Acoarse, MgPlan plan)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double wsl[32][4];
    __shared__ double csl[2][4];
    __shared__ Ctl ctl;
    // per-level band of this CTA and of its neighbours
    __shared__ int sR0[kMgMaxLevels], sR1[kMgMaxLevels], sLo[kMgMaxLevels];

    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int sample = blockIdx.x / CS;
    const int tid = threadIdx.x, nt = blockDim.x;
    const bool has_lo = rank > 0, has_hi = rank + 1 < CS;
    const int NL = plan.nl;
    if (tid < NL) {
        int a, b;
        mg_band(g.m, CS, rank, tid, &a, &b);
        sR0[tid] = a;
        sR1[tid] = b;
        if (has_lo) {
            mg_band(g.m, CS, rank - 1, tid, &a, &b);
            sLo[tid] = a;
        } else {
            sLo[tid] = 0;
        }
    }
    __syncthreads();

    auto F_ = [&](int off) { return reinterpret_cast<float *>(smem_raw + off); };
    const int m = g.m, n = g.n;
    const int own0 = sR0[0] * m, own1 = sR1[0] * m, nown = own1 - own0;

    const size_t so = (size_t)sample * n;
    const size_t SN = (size_t)g.S * n;
    const double *A64 = g.A64 + (size_t)sample * kSlots2D * n;
    double *v = g.v + so;
    double *wb0 = g.w + so;
    double *b = g.b + so;

    // ---- one-time set-up: stencil rows of every level, zeroed tiles
    for (int c = 0; c < NL; ++c) {
        const MgLevelPlan &P = plan.lv[c];
        const int mc = P.m, nc = mc * mc, R0 = sR0[c], R1 = sR1[c];
        const float *Ag = (c == 0 ? g.Ai + (size_t)sample * kSlots2D * n
                                  : Acoarse.A[c] + (size_t)sample * kSlots2D * nc);
        float *Dd = F_(P.off_d), *Ee = F_(P.off_e), *Nn = F_(P.off_n), *NE = F_(P.off_ne);
        const int base = (R0 - 1) * mc;   // node of index 1
        for (int t = tid; t < P.csize; t += nt) {
            const int node = base + (t - 1);
            const bool ok = t > 0 && node >= 0 && node < R1 * mc;
            Dd[t] = ok ? Ag[node] : 0.0f;
            Ee[t] = ok ? Ag[nc + node] : 0.0f;
            Nn[t] = ok ? Ag[2 * nc + node] : 0.0f;
            NE[t] = ok ? Ag[3 * nc + node] : 0.0f;
        }
        float *xa = F_(P.off_xa), *xb = F_(P.off_xb), *rr = F_(P.off_r);
        for (int t = tid; t < P.tile; t += nt) {
            xa[t] = 0.0f;
            xb[t] = 0.0f;
            rr[t] = 0.0f;
        }
    }
    for (int node = own0 + tid; node < own1; node += nt) {
        double v0, w0;
        if (g.v0) {
            v0 = g.v0[node];
            w0 = g.w0 ? g.w0[node] : 0.0;
        } else {
            const int j = node / m, i = node - j * m;
            const double xx = (double)i / (double)(m - 1), yy = (double)j / (double)(m - 1);
            v0 = (xx * xx + yy * yy <= g.radius2) ? 1.0 : 0.0;
            w0 = 0.0;
        }
        v[node] = v0;
        wb0[node] = w0;
    }
    cl.sync();

    // ---- helpers ----------------------------------------------------------
    // import the halo rows of the tile at byte offset `off` on level c
    auto exchange = [&](int c, int off) {
        if constexpr (CS == 1) {
            __syncthreads();
        } else {
            const int mc = plan.lv[c].m, R0 = sR0[c], R1 = sR1[c];
            cl.sync();
            float *T = F_(off);
            if (has_lo) {
                const float *nb = cl.map_shared_rank(T, rank - 1);
                const int src = 1 + mc + (R0 - 1 - sLo[c]) * mc;   // rank-1's last own row
                for (int i = tid; i < mc; i += nt) T[1 + i] = nb[src + i];
            }
            if (has_hi) {
                const float *nb = cl.map_shared_rank(T, rank + 1);
                const int dst = 1 + mc + (R1 - R0) * mc;
                for (int i = tid; i < mc; i += nt) T[dst + i] = nb[1 + mc + i];
            }
            __syncthreads();
        }
    };
    // (A x)_t on level c, t = tile index of an own node (= stencil index + 0)
    auto spmv = [&](const float *Dd, const float *Ee, const float *Nn, const float *NE, int mc, const float *x,
                    int t) {
        float w = Dd[t] * x[t];
        w = fmaf(Ee[t], x[t + 1], w);
        w = fmaf(Ee[t - 1], x[t - 1], w);
        w = fmaf(Nn[t], x[t + mc], w);
        w = fmaf(Nn[t - mc], x[t - mc], w);
        w = fmaf(NE[t], x[t + mc + 1], w);
        w = fmaf(NE[t - mc - 1], x[t - mc - 1], w);
        return w;
    };

    // V-cycle on BB of level 0 (own rows), result in XA of level 0
    auto vcycle = [&]() {
        for (int c = 0; c < NL; ++c) {
            const MgLevelPlan &P = plan.lv[c];
            const int mc = P.m, nown_c = (sR1[c] - sR0[c]) * mc, base = 1 + mc;
            const float *Dd = F_(P.off_d), *Ee = F_(P.off_e), *Nn = F_(P.off_n), *NE = F_(P.off_ne);
            float *xa = F_(P.off_xa), *xb = F_(P.off_xb), *rr = F_(P.off_r), *bb = F_(P.off_b);
            // pre-smoothing from zero: XA = omega D^-1 B
            for (int l = tid; l < nown_c; l += nt) xa[base + l] = kMgOmega * bb[l] / Dd[base + l];
            if (c == NL - 1) {
                // coarsest: further damped Jacobi sweeps, ping-pong XA / XB
                const int sweeps = CS == 1 ? 6 : 10;
                float *X = xa, *Y = xb;
                int ox = P.off_xa, oy = P.off_xb;
                for (int k = 1; k < sweeps; ++k) {
                    exchange(c, ox);
                    for (int l = tid; l < nown_c; l += nt) {
                        const int t = base + l;
                        Y[t] = X[t] + kMgOmega * (bb[l] - spmv(Dd, Ee, Nn, NE, mc, X, t)) / Dd[t];
                    }
                    float *tp = X;
                    X = Y;
                    Y = tp;
                    const int to = ox;
                    ox = oy;
                    oy = to;
                }
                if (X != xa)
                    for (int l = tid; l < nown_c; l += nt) xa[base + l] = X[base + l];
                break;
            }
            // residual RR = B - A XA
            exchange(c, P.off_xa);
            for (int l = tid; l < nown_c; l += nt) rr[base + l] = bb[l] - spmv(Dd, Ee, Nn, NE, mc, xa, base + l);
            exchange(c, P.off_r);
            // restriction: B_{c+1}(I, J) = R(2I, 2J) + 1/2 sum of the six neighbours
            const MgLevelPlan &Q = plan.lv[c + 1];
            const int mq = Q.m, R0q = sR0[c + 1], nown_q = (sR1[c + 1] - R0q) * mq;
            float *bq = F_(Q.off_b);
            const int R0 = sR0[c];
            for (int l = tid; l < nown_q; l += nt) {
                const int J = R0q + l / mq, I = l - (l / mq) * mq;
                const int i = 2 * I, j = 2 * J;
                const int t = 1 + (j - (R0 - 1)) * mc + i;
                float h = 0.0f;
                if (i + 1 < mc) h += rr[t + 1];
                if (i > 0) h += rr[t - 1];
                if (j + 1 < mc) h += rr[t + mc];
                if (j > 0) h += rr[t - mc];
                if (i + 1 < mc && j + 1 < mc) h += rr[t + mc + 1];
                if (i > 0 && j > 0) h += rr[t - mc - 1];
                bq[l] = rr[t] + 0.5f * h;
            }
        }
        // ascend: interpolate and post-smooth
        for (int c = NL - 2; c >= 0; --c) {
            const MgLevelPlan &P = plan.lv[c], &Q = plan.lv[c + 1];
            const int mc = P.m, R0 = sR0[c], nown_c = (sR1[c] - R0) * mc, base = 1 + mc;
            const int mq = Q.m, R0q = sR0[c + 1];
            const float *Dd = F_(P.off_d), *Ee = F_(P.off_e), *Nn = F_(P.off_n), *NE = F_(P.off_ne);
            float *xa = F_(P.off_xa), *xb = F_(P.off_xb), *bb = F_(P.off_b);
            const float *xq = F_(Q.off_xa);
            exchange(c + 1, Q.off_xa);
            // XB = XA + P X_{c+1}
            for (int l = tid; l < nown_c; l += nt) {
                const int jl = l / mc, i = l - jl * mc, j = R0 + jl;
                const int tq = 1 + ((j >> 1) - (R0q - 1)) * mq + (i >> 1);
                float pv;
                if (!(i & 1) && !(j & 1)) pv = xq[tq];
                else if ((i & 1) && !(j & 1)) pv = 0.5f * (xq[tq] + xq[tq + 1]);
                else if (!(i & 1) && (j & 1)) pv = 0.5f * (xq[tq] + xq[tq + mq]);
                else pv = 0.5f * (xq[tq] + xq[tq + mq + 1]);
                xb[base + l] = xa[base + l] + pv;
            }
            exchange(c, P.off_xb);
            // XA = XB + omega D^-1 (B - A XB)
            for (int l = tid; l < nown_c; l += nt) {
                const int t = base + l;
                xa[t] = xb[t] + kMgOmega * (bb[l] - spmv(Dd, Ee, Nn, NE, mc, xb, t)) / Dd[t];
            }
        }
    };

    const MgLevelPlan &P0 = plan.lv[0];
    const float *D0 = F_(P0.off_d), *E0 = F_(P0.off_e), *N0 = F_(P0.off_n), *NE0 = F_(P0.off_ne);
    float *XA0 = F_(P0.off_xa), *RR0 = F_(P0.off_r), *BB0 = F_(P0.off_b);
    const int FB = 1 + m;   // tile index of own local 0 on the fine level

    float r[NPT], u[NPT], w[NPT], sv[NPT], p[NPT], x[NPT];
    int wpar = 0, par = 0;
    int64_t total_iters = 0;
    int32_t status = S_CONVERGED;
    const double dt = g.dt;

    for (int step = 0; step < g.nsteps; ++step) {
        // ---- block load: b = M (v + dt R), w update, r0 = b - A v (into RR)
        const double *wcur = wb0 + wpar * SN;
        double *wnext = wb0 + (wpar ^ 1) * SN;
        {
            double acc[2] = {0.0, 0.0};
#pragma unroll 1
            for (int l = tid; l < nown; l += nt) {
                const int node = own0 + l;
                const int j = node / m, i = node - j * m;
                const double bb = mass_apply_y(m, i, j, g.h2, v, wcur, node, dt, g.a);
                b[node] = bb;
                const double vv = v[node], ww = wcur[node];
                wnext[node] = ww + dt * g.eps * (vv - g.gam * ww);
                const double rr = bb - stencil_apply_global(A64, n, m, node, i, j, v);
                RR0[FB + l] = (float)rr;
                acc[0] += bb * bb;
                acc[1] += rr * rr;
            }
            cluster_reduce<2, CS>(acc, wsl, csl, par, [&](double(&t)[2]) {
                ctl.s0 = t[0];
                ctl.s1 = t[1];
            });
            par ^= 1;
        }
        wpar ^= 1;
        const double bnorm2 = ctl.s0;
        double rnorm2 = ctl.s1;
        if (!(isfinite(bnorm2) && isfinite(rnorm2))) {
            status = S_NONFINITE;
            break;
        }
        const double tol_out2 = g.rtol_out * g.rtol_out * bnorm2;

        bool nonfinite = false, solved = false;
        for (int sweep = 0; sweep < g.max_sweeps; ++sweep) {
            if (sweep > 0) {
                double racc[1] = {0.0};
#pragma unroll 1
                for (int l = tid; l < nown; l += nt) {
                    const int node = own0 + l;
                    const int j = node / m, i = node - j * m;
                    const double rr = b[node] - stencil_apply_global(A64, n, m, node, i, j, v);
                    RR0[FB + l] = (float)rr;
                    racc[0] += rr * rr;
                }
                cluster_reduce<1, CS>(racc, wsl, csl, par, [&](double(&t)[1]) { ctl.s1 = t[0]; });
                par ^= 1;
                rnorm2 = ctl.s1;
                if (!isfinite(rnorm2)) { nonfinite = true; break; }
            }
            if (rnorm2 <= tol_out2) { solved = true; break; }
            const double rnorm = sqrt(rnorm2);
            const float rscale = (float)(1.0 / rnorm);
            const double tol_in2 = g.rtol_in * g.rtol_in;

            // ---- init: r0 (normalised), u0 = MG(r0), w0 = A u0
#pragma unroll
            for (int k = 0; k < NPT; ++k) {
                const int l = tid + k * nt;
                if (l < nown) {
                    r[k] = RR0[FB + l] * rscale;
                    BB0[l] = r[k];
                }
                x[k] = 0.0f;
                p[k] = 0.0f;
                sv[k] = 0.0f;
            }
            __syncthreads();
            vcycle();
            exchange(0, P0.off_xa);
            float iacc[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int k = 0; k < NPT; ++k) {
                const int l = tid + k * nt;
                if (l < nown) {
                    u[k] = XA0[FB + l];
                    w[k] = spmv(D0, E0, N0, NE0, m, XA0, FB + l);
                    iacc[0] = fmaf(r[k], u[k], iacc[0]);
                    iacc[1] = fmaf(w[k], u[k], iacc[1]);
                    iacc[2] = fmaf(r[k], r[k], iacc[2]);
                }
            }
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
                        beta = gamma * rcp_newton(gamma_prev);
                        eta = delta - beta * beta * eta_prev;
                    }
                    alpha = gamma * rcp_newton(eta);
                    gamma_prev = gamma;
                    eta_prev = eta;
                }
                ctl.alpha = alpha;
                ctl.beta = beta;
                ctl.code = code;
            };
            cluster_reduce<3, CS>(iacc, wsl, csl, par, [&](double(&t)[3]) { decide(t[0], t[1], t[2]); });
            par ^= 1;
            while (true) {
                const int code = ctl.code;
                if (code != 0) {
                    if (code == 3) nonfinite = true;
                    else if (code == 2) status = status == S_CONVERGED ? S_MAXITER : status;
                    break;
                }
                const float ta = (float)ctl.alpha, tb = (float)ctl.beta;
                // s_i = w_i + b s_{i-1}; p_i = u_i + b p_{i-1}; x += a p_i; r -= a s_i
#pragma unroll
                for (int k = 0; k < NPT; ++k) {
                    const int l = tid + k * nt;
                    if (l < nown) {
                        sv[k] = it == 0 ? w[k] : fmaf(tb, sv[k], w[k]);
                        p[k] = it == 0 ? u[k] : fmaf(tb, p[k], u[k]);
                        x[k] = fmaf(ta, p[k], x[k]);
                        r[k] = fmaf(-ta, sv[k], r[k]);
                        BB0[l] = r[k];
                    }
                }
                __syncthreads();
                vcycle();
                exchange(0, P0.off_xa);
                float pacc[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int k = 0; k < NPT; ++k) {
                    const int l = tid + k * nt;
                    if (l < nown) {
                        u[k] = XA0[FB + l];
                        w[k] = spmv(D0, E0, N0, NE0, m, XA0, FB + l);
                        pacc[0] = fmaf(r[k], u[k], pacc[0]);
                        pacc[1] = fmaf(w[k], u[k], pacc[1]);
                        pacc[2] = fmaf(r[k], r[k], pacc[2]);
                    }
                }
                ++it;
                cluster_reduce<3, CS>(pacc, wsl, csl, par, [&](double(&t)[3]) { decide(t[0], t[1], t[2]); });
                par ^= 1;
            }
            total_iters += it;
            if (nonfinite) break;
#pragma unroll
            for (int k = 0; k < NPT; ++k) {
                const int l = tid + k * nt;
                if (l < nown) v[own0 + l] = fma((double)x[k], rnorm, v[own0 + l]);
            }
            cl.sync();
        }
        if (nonfinite) {
            status = S_NONFINITE;
            break;
        }
        if (!solved && status == S_CONVERGED) status = S_MAXITER;
    }

    double qacc[1] = {0.0};
    for (int node = own0 + tid; node < own1; node += nt) {
        const int j = node / m, i = node - j * m;
        qacc[0] += lumped_mass(m, i, j, g.h2) * v[node];
    }
    cluster_reduce<1, CS>(qacc, wsl, csl, par, [&](double(&t)[1]) { ctl.s0 = t[0]; });
    if (rank == 0 && tid == 0) {
        g.q[sample] = status == S_NONFINITE ? __longlong_as_double(0x7ff8000000000000LL) : ctl.s0;
        g.iters[sample] = (int32_t)(total_iters > 0x7fffffff ? 0x7fffffff : total_iters);
        g.status[sample] = status;
    }
    cl.sync();
}

}  // namespace mlq
