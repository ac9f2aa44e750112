// mlq_kernels.cuh -- device code of libmlq (sm_103a).
//
// Hot path of the per-sample forward solve of the stochastic monodomain
// equation, batched over samples:
//   K1 kl_synthesis_kernel    theta_e = theta_mean_e + sum_k Phi[e,k] xi_k
//                             (eq. KLlowrank), epilogue (cos 2t, sin 2t)
//   K2 stencil_setup_kernel   A = M + dt K(theta) as a stored 7-point stencil
//                             (Sec. 3.1 mass/stiffness, eq. AdmV conductivity)
//   K3-K6 slab_solve_kernel   all time blocks of one sample in one cluster of
//                             CTAs: FHN reaction and consistent-mass load
//                             (eq. mono_disc), Jacobi-PCG per block (multiple
//                             time blocks, Sec. 3.3), FP64 refinement
//   K7 level_sums_kernel      Y = Q_l - Q_{l-1} and per-level FP64 sums
//                             (eq. StandardML)
#pragma once

#include <cooperative_groups.h>
#include <cstdint>
#include <cuda_runtime.h>

namespace cg = cooperative_groups;

namespace mlq {

// per-sample status codes (mirror mlq_sample_status)
enum : int32_t { S_CONVERGED = 0, S_MAXITER = 1, S_NONFINITE = 2 };

// Coefficient slots of the stored stencil, per node P = (i, j):
//   0 diag  A[P][P]
//   1 E     A[P][(i+1, j)]
//   2 N     A[P][(i, j+1)]
//   3 NE    A[P][(i+1, j+1)]
//   4 dinv  1 / A[P][P]  (Jacobi preconditioner)
// The W, S and SW entries of row P are the E, N, NE slots of the neighbour
// (A is symmetric).  Slots of missing neighbours hold 0.
constexpr int kSlots2D = 5;

// Fast division by a level constant: q = (n * mul) >> 40, exact for
// n * d < 2^40 (checked on the host for every divisor it sets up).
struct FastDiv {
    uint64_t mul;
    uint32_t d;
    __host__ __device__ __forceinline__ uint32_t div(uint32_t n) const {
        return (uint32_t)(((uint64_t)n * mul) >> 40);
    }
};

// ---------------------------------------------------------------------------
// K1: KL synthesis.  One thread per (element, sample); Phi rows are shared
// by all samples (L1/L2 resident), xi rows by all elements.
// out[(s*ne + e)*2 + {0,1}] = (cos 2 theta, sin 2 theta).
// ---------------------------------------------------------------------------
__global__ void kl_synthesis_kernel(const double *__restrict__ phi, const double *__restrict__ theta_mean,
                                    const double *__restrict__ xi, int K, int ne, int S,
                                    double *__restrict__ out)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (e >= ne || s >= S) return;
    const double *pr = phi + (size_t)e * K;
    const double *xr = xi + (size_t)s * K;
    double t = theta_mean ? theta_mean[e] : 0.0;
    for (int k = 0; k < K; ++k) t = fma(pr[k], xr[k], t);
    double sn, cs;
    sincos(2.0 * t, &sn, &cs);
    out[((size_t)s * ne + e) * 2 + 0] = cs;
    out[((size_t)s * ne + e) * 2 + 1] = sn;
}

// ---------------------------------------------------------------------------
// K2: stencil of A = M + dt K(theta) on the structured triangulation.
//
// With D = sbar I + (ds/2) [[c2, s2], [s2, -c2]], sbar = (s_l+s_t)/2,
// ds = s_l - s_t, (c2, s2) = (cos 2t, sin 2t):
//   d11 = sbar + ds/2 c2,  d22 = sbar - ds/2 c2,  d12 = ds/2 s2.
// P1 element stiffness (|e| = h^2/2, h cancels in 2D):
//   lower (a,b,c) = (i,j)(i+1,j)(i+1,j+1), gradients (-1,0),(1,-1),(0,1) / h
//   upper (a,c,d) = (i,j)(i+1,j+1)(i,j+1), gradients (0,-1),(1,0),(-1,1) / h
//   K_xy = (1/2) g_x^T D g_y.
// Consistent mass per element: h^2/12 on the diagonal, h^2/24 off it.
// ---------------------------------------------------------------------------
struct DTensor {
    double d11, d12, d22;
};

__device__ __forceinline__ DTensor dtensor(const double *cs, double sbar, double hds)
{
    DTensor D;
    D.d11 = sbar + hds * cs[0];
    D.d22 = sbar - hds * cs[0];
    D.d12 = hds * cs[1];
    return D;
}

__global__ void stencil_setup_kernel(const double *__restrict__ cs2, int m, double h, double dt, double s_l,
                                     double s_t, int S, double *__restrict__ A64, float *__restrict__ A32)
{
    const int n = m * m;
    const int node = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (node >= n || s >= S) return;
    const int i = node % m, j = node / m;
    const int ne = 2 * (m - 1) * (m - 1);
    const double *c = cs2 + (size_t)s * ne * 2;
    const double sbar = 0.5 * (s_l + s_t), hds = 0.5 * (s_l - s_t);
    const double mdiag = h * h / 12.0, moff = h * h / 24.0;
    const int mc = m - 1; // cells per side
    double diag = 0.0, east = 0.0, north = 0.0, ne_ = 0.0;
    auto lower = [&](int ci, int cj) { return 2 * (ci + mc * cj); };
    auto upper = [&](int ci, int cj) { return 2 * (ci + mc * cj) + 1; };
    const bool cell_ij = (i < mc && j < mc);         // square (i, j)
    const bool cell_im = (i >= 1 && j < mc);         // square (i-1, j)
    const bool cell_mm = (i >= 1 && j >= 1);         // square (i-1, j-1)
    const bool cell_jm = (i < mc && j >= 1);         // square (i, j-1)
    if (cell_ij) {
        // lower(i,j): P = a; E = b; NE = c
        DTensor D = dtensor(c + 2 * lower(i, j), sbar, hds);
        diag += 0.5 * D.d11 * dt + mdiag;
        east += -0.5 * (D.d11 - D.d12) * dt + moff;
        ne_ += -0.5 * D.d12 * dt + moff;
        // upper(i,j): P = a; NE = c; N = d
        D = dtensor(c + 2 * upper(i, j), sbar, hds);
        diag += 0.5 * D.d22 * dt + mdiag;
        ne_ += -0.5 * D.d12 * dt + moff;
        north += 0.5 * (D.d12 - D.d22) * dt + moff;
    }
    if (cell_im) {
        // lower(i-1,j): a = (i-1,j), P = b, N = c
        DTensor D = dtensor(c + 2 * lower(i - 1, j), sbar, hds);
        diag += 0.5 * (D.d11 - 2.0 * D.d12 + D.d22) * dt + mdiag;
        north += 0.5 * (D.d12 - D.d22) * dt + moff;
    }
    if (cell_mm) {
        // lower(i-1,j-1): P = c; upper(i-1,j-1): P = c
        DTensor D = dtensor(c + 2 * lower(i - 1, j - 1), sbar, hds);
        diag += 0.5 * D.d22 * dt + mdiag;
        D = dtensor(c + 2 * upper(i - 1, j - 1), sbar, hds);
        diag += 0.5 * D.d11 * dt + mdiag;
    }
    if (cell_jm) {
        // upper(i,j-1): a = (i,j-1), E = c, P = d
        DTensor D = dtensor(c + 2 * upper(i, j - 1), sbar, hds);
        diag += 0.5 * (D.d11 - 2.0 * D.d12 + D.d22) * dt + mdiag;
        east += -0.5 * (D.d11 - D.d12) * dt + moff;
    }
    double *a = A64 + (size_t)s * kSlots2D * n;
    a[node] = diag;
    a[n + node] = east;
    a[2 * n + node] = north;
    a[3 * n + node] = ne_;
    a[4 * n + node] = 1.0 / diag;
    if (A32) {
        float *f = A32 + (size_t)s * kSlots2D * n;
        f[node] = (float)diag;
        f[n + node] = (float)east;
        f[2 * n + node] = (float)north;
        f[3 * n + node] = (float)ne_;
        f[4 * n + node] = 1.0f / (float)diag;
    }
}

// ---------------------------------------------------------------------------
// Slab solver.
// ---------------------------------------------------------------------------
template <typename TI>
struct SolveArgs {
    int m, n;
    FastDiv divm;
    double h2;                    // h^2
    double dt;
    int nsteps;
    double a, eps, gam;           // FHN
    double rtol_out, rtol_in;     // FP64 residual target, inner relative target
    int max_iter, max_sweeps;
    const double *A64;            // [S][4][n]
    const TI *Ai;                 // [S][4][n] stencil in the inner precision
    double *v;                    // [S][n]
    double *w;                    // [2][S][n]
    double *b;                    // [S][n]
    TI *r, *s, *wc;               // [2][S][n] each
    TI *p, *x;                    // [S][n]
    const double *v0, *w0;        // [n] or null
    double radius2;               // initial disc, used when v0 is null
    int S;
    double *q;                    // [S]
    int32_t *iters, *status;      // [S]
};

template <typename T>
__device__ __forceinline__ T ldcg(const T *p) { return __ldcg(p); }

// Sum NV doubles over the block and then over the cluster.  Every thread of
// every CTA returns the same values: per-CTA partials are combined in rank
// order, so the result does not depend on timing.
template <int NV, int CS>
__device__ __forceinline__ void cluster_sum(double (&v)[NV], double (*warp_buf)[4], double (*slots)[4], int par)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) warp_buf[warp][k] = v[k];
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double t = 0.0;
        for (int w = 0; w < nwarp; ++w) t += warp_buf[w][threadIdx.x];
        slots[par][threadIdx.x] = t;
    }
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = 0.0;
#pragma unroll
    for (int r = 0; r < CS; ++r) {
        const double *rs = cl.map_shared_rank(&slots[par][0], r);
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] += rs[k];
    }
}

// Stencil apply at own node P = (i, j) (tile index l) for a vector held in a
// shared-memory tile; coefficients from the sample's stored stencil.
template <typename TI, typename TV>
__device__ __forceinline__ TV stencil_apply(const TI *__restrict__ A, int n, int m, int node, int i, int j,
                                            const TV *u, int l)
{
    TV acc = (TV)A[node] * u[l];
    if (i + 1 < m) acc += (TV)A[n + node] * u[l + 1];
    if (i > 0) acc += (TV)A[n + node - 1] * u[l - 1];
    if (j + 1 < m) acc += (TV)A[2 * n + node] * u[l + m];
    if (j > 0) acc += (TV)A[2 * n + node - m] * u[l - m];
    if (i + 1 < m && j + 1 < m) acc += (TV)A[3 * n + node] * u[l + m + 1];
    if (i > 0 && j > 0) acc += (TV)A[3 * n + node - m - 1] * u[l - m - 1];
    return acc;
}

// Same, reading the vector from global memory (other CTAs' rows through L2).
__device__ __forceinline__ double stencil_apply_global(const double *__restrict__ A, int n, int m, int node, int i,
                                                       int j, const double *x)
{
    double acc = A[node] * ldcg(x + node);
    if (i + 1 < m) acc += A[n + node] * ldcg(x + node + 1);
    if (i > 0) acc += A[n + node - 1] * ldcg(x + node - 1);
    if (j + 1 < m) acc += A[2 * n + node] * ldcg(x + node + m);
    if (j > 0) acc += A[2 * n + node - m] * ldcg(x + node - m);
    if (i + 1 < m && j + 1 < m) acc += A[3 * n + node] * ldcg(x + node + m + 1);
    if (i > 0 && j > 0) acc += A[3 * n + node - m - 1] * ldcg(x + node - m - 1);
    return acc;
}

// Consistent mass applied to a tile vector at own node (i, j): each existing
// incident triangle adds h^2/12 to the diagonal and h^2/24 per shared edge.
__device__ __forceinline__ double mass_apply(int m, int i, int j, double h2, const double *y, int l)
{
    const int mc = m - 1;
    const bool cij = (i < mc && j < mc), cim = (i >= 1 && j < mc), cmm = (i >= 1 && j >= 1),
               cjm = (i < mc && j >= 1);
    // incident triangles: lower/upper(i,j) [2 if cij], lower(i-1,j) [cim],
    // lower/upper(i-1,j-1) [2 if cmm], upper(i,j-1) [cjm]
    const int ninc = 2 * cij + cim + 2 * cmm + cjm;
    double acc = (double)ninc * (h2 / 12.0) * y[l];
    const double e = h2 / 24.0;
    // edge to E: lower(i,j), upper(i,j-1)
    if (i + 1 < m) acc += e * (double)(cij + cjm) * y[l + 1];
    // edge to W: lower(i-1,j) [as a-b], upper(i-1,j-1) [as c-d]
    if (i > 0) acc += e * (double)(cim + cmm) * y[l - 1];
    // edge to N: upper(i,j) [a-d], lower(i-1,j) [b-c]
    if (j + 1 < m) acc += e * (double)(cij + cim) * y[l + m];
    // edge to S: upper(i,j-1) [d-a], lower(i-1,j-1) [c-b]
    if (j > 0) acc += e * (double)(cjm + cmm) * y[l - m];
    // edge to NE: lower(i,j), upper(i,j)
    if (i + 1 < m && j + 1 < m) acc += e * (double)(2 * cij) * y[l + m + 1];
    // edge to SW: lower(i-1,j-1), upper(i-1,j-1)
    if (i > 0 && j > 0) acc += e * (double)(2 * cmm) * y[l - m - 1];
    return acc;
}

// Lumped mass m_i = sum over incident triangles |e|/3 = ninc h^2 / 6.
__device__ __forceinline__ double lumped_mass(int m, int i, int j, double h2)
{
    const int mc = m - 1;
    const int ninc = 2 * (i < mc && j < mc) + (i >= 1 && j < mc) + 2 * (i >= 1 && j >= 1) + (i < mc && j >= 1);
    return (double)ninc * h2 / 6.0;
}

// One cluster of CS CTAs per sample.  CTA `rank` owns rows [r0, r1) of the
// m x m grid; its shared tile holds rows [lo, hi) = own rows plus one halo row
// on each side.  Per time block (multiple time blocks, Sec. 3.3):
//   S1  y = v + dt R(v, w) on the tile, b = M y, w <- w + dt eps (v - gam w),
//       r = b - A v                                         (eq. mono_disc)
//   refinement sweeps: inner Jacobi-PCG on A d = r (Chronopoulos-Gear form:
//       one cluster barrier per iteration), v += d, new FP64 residual.
// In the FP64 path (TI = double) one sweep runs to rtol ||b||.
template <typename TI, int CS>
__global__ void __launch_bounds__(512, 1) slab_solve_kernel(SolveArgs<TI> g)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double warp_buf[32][4];
    __shared__ double slots[2][4];

    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int sample = blockIdx.x / CS;
    const int m = g.m, n = g.n;
    const int r0 = (int)(((int64_t)m * rank) / CS), r1 = (int)(((int64_t)m * (rank + 1)) / CS);
    const int lo = r0 > 0 ? r0 - 1 : 0, hi = r1 < m ? r1 + 1 : m;
    const int own0 = r0 * m, own1 = r1 * m, tile0 = lo * m, tile1 = hi * m;
    const int tid = threadIdx.x, nt = blockDim.x;

    double *ytile = reinterpret_cast<double *>(smem_raw);   // FP64 tile (block S1)
    TI *utile = reinterpret_cast<TI *>(smem_raw);           // inner-precision tile (PCG)

    const size_t so = (size_t)sample * n;
    const size_t SN = (size_t)g.S * n;  // stride between the two halves of a double buffer
    const double *A64 = g.A64 + (size_t)sample * kSlots2D * n;
    const TI *Ai = g.Ai + (size_t)sample * kSlots2D * n;
    const TI *Dinv = Ai + 4 * (size_t)n;
    double *v = g.v + so;
    double *wb0 = g.w + so;
    double *b = g.b + so;
    TI *rb0 = g.r + so;
    TI *sb0 = g.s + so;
    TI *wc0 = g.wc + so;
    TI *p = g.p + so;
    TI *x = g.x + so;
    int par = 0;  // parity of the reduction slots

    // initial state
    for (int node = own0 + tid; node < own1; node += nt) {
        double v0, w0;
        if (g.v0) {
            v0 = g.v0[node];
            w0 = g.w0 ? g.w0[node] : 0.0;
        } else {
            const int j = (int)g.divm.div((uint32_t)node), i = node - j * m;
            const double xx = (double)i / (double)(m - 1), yy = (double)j / (double)(m - 1);
            v0 = (xx * xx + yy * yy <= g.radius2) ? 1.0 : 0.0;
            w0 = 0.0;
        }
        v[node] = v0;
        wb0[node] = w0;
    }
    cl.sync();

    int wpar = 0;
    int64_t total_iters = 0;
    int32_t status = S_CONVERGED;
    const bool mixed = sizeof(TI) == 4;
    const double dt = g.dt;

    for (int step = 0; step < g.nsteps; ++step) {
        // ---- S1: reaction, consistent-mass load, recovery update, residual
        for (int node = tile0 + tid; node < tile1; node += nt) {
            const double vv = ldcg(v + node), ww = ldcg(wb0 + wpar * SN + node);
            const double R = vv * (vv - g.a) * (1.0 - vv) - ww;
            ytile[node - tile0] = vv + dt * R;
        }
        __syncthreads();
        double acc[2] = {0.0, 0.0};  // |b|^2, |r|^2
        double *wcur = wb0 + wpar * SN, *wnext = wb0 + (wpar ^ 1) * SN;
        for (int node = own0 + tid; node < own1; node += nt) {
            const int j = (int)g.divm.div((uint32_t)node), i = node - j * m;
            const double bb = mass_apply(m, i, j, g.h2, ytile, node - tile0);
            b[node] = bb;
            const double vv = v[node], ww = wcur[node];
            wnext[node] = ww + dt * g.eps * (vv - g.gam * ww);
            const double rr = bb - stencil_apply_global(A64, n, m, node, i, j, v);
            rb0[node] = (TI)rr;
            acc[0] += bb * bb;
            acc[1] += rr * rr;
        }
        cluster_sum<2, CS>(acc, warp_buf, slots, par);
        par ^= 1;
        wpar ^= 1;
        const double bnorm2 = acc[0];
        double rnorm2 = acc[1];
        if (!(isfinite(bnorm2) && isfinite(rnorm2))) {
            status = S_NONFINITE;
            break;
        }
        const double tol_out2 = g.rtol_out * g.rtol_out * bnorm2;

        bool nonfinite = false, solved = false;
        for (int sweep = 0; sweep < g.max_sweeps; ++sweep) {
            if (sweep > 0) {
                // ---- FP64 residual of the refined iterate
                double racc[2] = {0.0, 0.0};
                for (int node = own0 + tid; node < own1; node += nt) {
                    const int j = (int)g.divm.div((uint32_t)node), i = node - j * m;
                    const double rr = b[node] - stencil_apply_global(A64, n, m, node, i, j, v);
                    rb0[node] = (TI)rr;
                    racc[0] += rr * rr;
                }
                cluster_sum<2, CS>(racc, warp_buf, slots, par);
                par ^= 1;
                rnorm2 = racc[0];
                if (!isfinite(rnorm2)) { nonfinite = true; break; }
            }
            if (rnorm2 <= tol_out2) { solved = true; break; }
            const double tol_in2 = mixed ? g.rtol_in * g.rtol_in * rnorm2 : tol_out2;

            // ---- inner PCG init: u0 = r0 / d on the tile, w0 = A u0
            for (int node = tile0 + tid; node < tile1; node += nt)
                utile[node - tile0] = ldcg(rb0 + node) * Dinv[node];
            __syncthreads();
            double iacc[3] = {0.0, 0.0, 0.0};  // gamma, delta, |r|^2
            for (int node = own0 + tid; node < own1; node += nt) {
                const int j = (int)g.divm.div((uint32_t)node), i = node - j * m;
                const int l = node - tile0;
                const TI u0 = utile[l];
                const TI w0 = stencil_apply<TI, TI>(Ai, n, m, node, i, j, utile, l);
                wc0[node] = w0;
                x[node] = (TI)0;
                const TI r0v = rb0[node];
                iacc[0] += (double)(r0v * u0);
                iacc[1] += (double)(w0 * u0);
                iacc[2] += (double)(r0v * r0v);
            }
            cluster_sum<3, CS>(iacc, warp_buf, slots, par);
            par ^= 1;
            double gamma = iacc[0], delta = iacc[1], rr = iacc[2];
            double gamma_prev = 1.0, alpha_prev = 1.0;
            int it = 0;
            while (true) {
                if (!isfinite(rr) || !isfinite(gamma) || !isfinite(delta)) { nonfinite = true; break; }
                if (rr <= tol_in2) { solved = !mixed; break; }
                if (it >= g.max_iter) { status = status == S_CONVERGED ? S_MAXITER : status; break; }
                double alpha, beta;
                if (it == 0) {
                    beta = 0.0;
                    alpha = gamma / delta;
                } else {
                    beta = gamma / gamma_prev;
                    alpha = gamma / (delta - beta * gamma / alpha_prev);
                }
                const TI ta = (TI)alpha, tb = (TI)beta;
                const int cur = it & 1, nxt = cur ^ 1;
                const TI *rcur = rb0 + cur * SN, *wcurv = wc0 + cur * SN, *sprev = sb0 + nxt * SN;
                TI *rnext = rb0 + nxt * SN, *scur = sb0 + cur * SN, *wnextv = wc0 + nxt * SN;
                double pacc[3] = {0.0, 0.0, 0.0};
                // s_i = w_i + beta s_{i-1};  r_{i+1} = r_i - alpha s_i;  u_{i+1} = r_{i+1}/d
                // (own rows and halo rows: the halo is recomputed from the
                // neighbours' previous-iteration vectors, double-buffered)
                for (int node = tile0 + tid; node < tile1; node += nt) {
                    const TI ri = ldcg(rcur + node), wi = ldcg(wcurv + node);
                    const TI sp = it == 0 ? (TI)0 : ldcg(sprev + node);
                    const TI si = wi + tb * sp;
                    const TI rn = ri - ta * si;
                    const TI di = Dinv[node];
                    const TI un = rn * di;
                    utile[node - tile0] = un;
                    if (node >= own0 && node < own1) {
                        const TI ui = ri * di;
                        const TI pi = it == 0 ? ui : ui + tb * p[node];
                        x[node] = x[node] + ta * pi;
                        p[node] = pi;
                        scur[node] = si;
                        rnext[node] = rn;
                        pacc[0] += (double)(rn * un);
                        pacc[2] += (double)(rn * rn);
                    }
                }
                __syncthreads();
                for (int node = own0 + tid; node < own1; node += nt) {
                    const int j = (int)g.divm.div((uint32_t)node), i = node - j * m;
                    const int l = node - tile0;
                    const TI wn = stencil_apply<TI, TI>(Ai, n, m, node, i, j, utile, l);
                    wnextv[node] = wn;
                    pacc[1] += (double)(wn * utile[l]);
                }
                cluster_sum<3, CS>(pacc, warp_buf, slots, par);
                par ^= 1;
                gamma_prev = gamma;
                alpha_prev = alpha;
                gamma = pacc[0];
                delta = pacc[1];
                rr = pacc[2];
                ++it;
            }
            total_iters += it;
            if (nonfinite) break;
            // ---- v += d
            for (int node = own0 + tid; node < own1; node += nt)
                v[node] = v[node] + (double)x[node];
            cl.sync();
            if (!mixed) break;  // FP64: a single sweep solves to rtol ||b||
        }
        if (nonfinite) {
            status = S_NONFINITE;
            break;
        }
        if (!solved && status == S_CONVERGED) status = S_MAXITER;
    }

    // ---- QoI: Q = m^T v, m = M 1
    double qacc[1] = {0.0};
    for (int node = own0 + tid; node < own1; node += nt) {
        const int j = (int)g.divm.div((uint32_t)node), i = node - j * m;
        qacc[0] += lumped_mass(m, i, j, g.h2) * v[node];
    }
    cluster_sum<1, CS>(qacc, warp_buf, slots, par);
    if (rank == 0 && tid == 0) {
        g.q[sample] = status == S_NONFINITE ? __longlong_as_double(0x7ff8000000000000LL) : qacc[0];
        g.iters[sample] = (int32_t)(total_iters > 0x7fffffff ? 0x7fffffff : total_iters);
        g.status[sample] = status;
    }
    // keep every CTA's shared memory alive until all remote reads are done
    cl.sync();
}

// ---------------------------------------------------------------------------
// Shared-memory-resident variant of the slab solver.
//
// Same algorithm and the same cluster decomposition as slab_solve_kernel, but
// every PCG vector of a CTA's rows lives in its shared memory for the whole
// run, and the halo rows of the next iterate are recomputed from the
// neighbouring CTAs' shared memory over DSMEM (distributed shared memory of
// the thread-block cluster).  The CG loop then touches global memory only for
// the read-only stencil coefficients (L1 resident).  The FP64 state (v, w, b)
// stays in global memory: it is read once per refinement sweep.
//
// Shared layout, identical in every CTA of the cluster (so that a neighbour's
// array is the same offset in its window):
//   utile  (rows_max + 2) * m   TI   tile rows [lo, hi) of the next iterate
//   R0 R1 W0 W1 S0 S1 P X       nmax TI each, own nodes, local index
//   ytile  (rows_max + 2) * m   FP64, aliases S0..X (dead while a block's
//          load vector is formed)
// ---------------------------------------------------------------------------
struct SmemPlan {
    int nmax;       // rows_max * m
    int tile;       // (rows_max + 2) * m, capped at m * m
    int off_vec;    // byte offset of R0
    int vec_bytes;  // bytes per own-node vector (16-byte multiple)
    int off_y;      // byte offset of ytile
    int total;      // dynamic shared bytes
};

__host__ __device__ inline int align16(int b) { return (b + 15) & ~15; }

__host__ __device__ inline SmemPlan smem_plan(int m, int cs, int ti_bytes)
{
    SmemPlan pl;
    const int rows = (m + cs - 1) / cs;
    pl.nmax = rows * m;
    pl.tile = (rows + 2 < m ? rows + 2 : m) * m;
    pl.off_vec = align16(pl.tile * ti_bytes);
    pl.vec_bytes = align16(pl.nmax * ti_bytes);
    pl.off_y = pl.off_vec + 4 * pl.vec_bytes;
    const int end_vec = pl.off_vec + 8 * pl.vec_bytes;
    const int end_y = pl.off_y + align16(pl.tile * 8);
    pl.total = end_vec > end_y ? end_vec : end_y;
    return pl;
}

template <typename TI, int CS>
__global__ void __launch_bounds__(512, 1) slab_solve_smem_kernel(SolveArgs<TI> g)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double warp_buf[32][4];
    __shared__ double slots[2][4];

    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int sample = blockIdx.x / CS;
    const int m = g.m, n = g.n;
    const int r0 = (int)(((int64_t)m * rank) / CS), r1 = (int)(((int64_t)m * (rank + 1)) / CS);
    const int lo = r0 > 0 ? r0 - 1 : 0, hi = r1 < m ? r1 + 1 : m;
    const int own0 = r0 * m, own1 = r1 * m, tile0 = lo * m, tile1 = hi * m;
    const int nown = own1 - own0;
    const int tid = threadIdx.x, nt = blockDim.x;
    const SmemPlan pl = smem_plan(m, CS, (int)sizeof(TI));

    TI *utile = reinterpret_cast<TI *>(smem_raw);
    TI *vec0 = reinterpret_cast<TI *>(smem_raw + pl.off_vec);
    const int vstride = pl.vec_bytes / (int)sizeof(TI);
    TI *Rv = vec0;                 // R0, R1 at Rv, Rv + vstride
    TI *Wv = vec0 + 2 * vstride;   // W0, W1
    TI *Sv = vec0 + 4 * vstride;   // S0, S1
    TI *P = vec0 + 6 * vstride;
    TI *X = vec0 + 7 * vstride;
    double *ytile = reinterpret_cast<double *>(smem_raw + pl.off_y);
    const int ushift = own0 - tile0;  // tile index of own local index 0

    // neighbours' windows (their arrays sit at the same offsets)
    const bool has_lo = rank > 0, has_hi = rank + 1 < CS;
    const int r0_lo = has_lo ? (int)(((int64_t)m * (rank - 1)) / CS) : 0;
    TI *vec_lo = has_lo ? cl.map_shared_rank(vec0, rank - 1) : nullptr;
    TI *vec_hi = has_hi ? cl.map_shared_rank(vec0, rank + 1) : nullptr;
    // local index, in the neighbour's numbering, of our halo rows' first node
    const int lo_base = (r0 - 1 - r0_lo) * m;  // row r0-1 in rank-1
    const int hi_base = 0;                     // row r1 is rank+1's first row

    const size_t so = (size_t)sample * n;
    const double *A64 = g.A64 + (size_t)sample * kSlots2D * n;
    const TI *Ai = g.Ai + (size_t)sample * kSlots2D * n;
    const TI *Dinv = Ai + 4 * (size_t)n;
    double *v = g.v + so;
    double *wb0 = g.w + so;
    const size_t SN = (size_t)g.S * n;
    double *b = g.b + so;
    int par = 0;

    for (int node = own0 + tid; node < own1; node += nt) {
        double v0, w0;
        if (g.v0) {
            v0 = g.v0[node];
            w0 = g.w0 ? g.w0[node] : 0.0;
        } else {
            const int j = (int)g.divm.div((uint32_t)node), i = node - j * m;
            const double xx = (double)i / (double)(m - 1), yy = (double)j / (double)(m - 1);
            v0 = (xx * xx + yy * yy <= g.radius2) ? 1.0 : 0.0;
            w0 = 0.0;
        }
        v[node] = v0;
        wb0[node] = w0;
    }
    cl.sync();

    int wpar = 0;
    int64_t total_iters = 0;
    int32_t status = S_CONVERGED;
    const bool mixed = sizeof(TI) == 4;
    const double dt = g.dt;

    for (int step = 0; step < g.nsteps; ++step) {
        // ---- block load: y = v + dt R(v, w) on the tile, b = M y, w update,
        //      r0 = b - A v into R0 (own rows)
        const double *wcur = wb0 + wpar * SN;
        double *wnext = wb0 + (wpar ^ 1) * SN;
        for (int node = tile0 + tid; node < tile1; node += nt) {
            const double vv = ldcg(v + node), ww = ldcg(wcur + node);
            const double R = vv * (vv - g.a) * (1.0 - vv) - ww;
            ytile[node - tile0] = vv + dt * R;
        }
        __syncthreads();
        double acc[2] = {0.0, 0.0};
        for (int node = own0 + tid; node < own1; node += nt) {
            const int j = (int)g.divm.div((uint32_t)node), i = node - j * m;
            const double bb = mass_apply(m, i, j, g.h2, ytile, node - tile0);
            b[node] = bb;
            const double vv = v[node], ww = wcur[node];
            wnext[node] = ww + dt * g.eps * (vv - g.gam * ww);
            const double rr = bb - stencil_apply_global(A64, n, m, node, i, j, v);
            Rv[node - own0] = (TI)rr;
            acc[0] += bb * bb;
            acc[1] += rr * rr;
        }
        cluster_sum<2, CS>(acc, warp_buf, slots, par);
        par ^= 1;
        wpar ^= 1;
        const double bnorm2 = acc[0];
        double rnorm2 = acc[1];
        if (!(isfinite(bnorm2) && isfinite(rnorm2))) {
            status = S_NONFINITE;
            break;
        }
        const double tol_out2 = g.rtol_out * g.rtol_out * bnorm2;

        bool nonfinite = false, solved = false;
        for (int sweep = 0; sweep < g.max_sweeps; ++sweep) {
            if (sweep > 0) {
                double racc[2] = {0.0, 0.0};
                for (int node = own0 + tid; node < own1; node += nt) {
                    const int j = (int)g.divm.div((uint32_t)node), i = node - j * m;
                    const double rr = b[node] - stencil_apply_global(A64, n, m, node, i, j, v);
                    Rv[node - own0] = (TI)rr;
                    racc[0] += rr * rr;
                }
                cluster_sum<2, CS>(racc, warp_buf, slots, par);
                par ^= 1;
                rnorm2 = racc[0];
                if (!isfinite(rnorm2)) { nonfinite = true; break; }
            }
            if (rnorm2 <= tol_out2) { solved = true; break; }
            const double tol_in2 = mixed ? g.rtol_in * g.rtol_in * rnorm2 : tol_out2;

            // ---- inner PCG init: u0 = r0 d^-1 on the tile, w0 = A u0, x = 0
            for (int l = tid; l < nown; l += nt) utile[l + ushift] = Rv[l] * Dinv[own0 + l];
            if (has_lo)
                for (int i = tid; i < m; i += nt)
                    utile[i] = vec_lo[lo_base + i] * Dinv[tile0 + i];
            if (has_hi)
                for (int i = tid; i < m; i += nt)
                    utile[own1 - tile0 + i] = vec_hi[hi_base + i] * Dinv[own1 + i];
            __syncthreads();
            double iacc[3] = {0.0, 0.0, 0.0};
            for (int l = tid; l < nown; l += nt) {
                const int node = own0 + l;
                const int j = (int)g.divm.div((uint32_t)node), i = node - j * m;
                const TI u0 = utile[l + ushift];
                const TI w0 = stencil_apply<TI, TI>(Ai, n, m, node, i, j, utile, l + ushift);
                Wv[l] = w0;
                X[l] = (TI)0;
                const TI r0v = Rv[l];
                iacc[0] += (double)(r0v * u0);
                iacc[1] += (double)(w0 * u0);
                iacc[2] += (double)(r0v * r0v);
            }
            cluster_sum<3, CS>(iacc, warp_buf, slots, par);
            par ^= 1;
            double gamma = iacc[0], delta = iacc[1], rr = iacc[2];
            double gamma_prev = 1.0, alpha_prev = 1.0;
            int it = 0;
            while (true) {
                if (!isfinite(rr) || !isfinite(gamma) || !isfinite(delta)) { nonfinite = true; break; }
                if (rr <= tol_in2) { solved = !mixed; break; }
                if (it >= g.max_iter) { status = status == S_CONVERGED ? S_MAXITER : status; break; }
                double alpha, beta;
                if (it == 0) {
                    beta = 0.0;
                    alpha = gamma / delta;
                } else {
                    beta = gamma / gamma_prev;
                    alpha = gamma / (delta - beta * gamma / alpha_prev);
                }
                const TI ta = (TI)alpha, tb = (TI)beta;
                const int cur = it & 1, nxt = cur ^ 1;
                TI *Rc = Rv + cur * vstride, *Rn = Rv + nxt * vstride;
                TI *Wc = Wv + cur * vstride, *Wn = Wv + nxt * vstride;
                TI *Sc = Sv + cur * vstride, *Sp = Sv + nxt * vstride;
                double pacc[3] = {0.0, 0.0, 0.0};
                // own rows
                for (int l = tid; l < nown; l += nt) {
                    const TI ri = Rc[l], wi = Wc[l];
                    const TI si = it == 0 ? wi : wi + tb * Sp[l];
                    const TI rn = ri - ta * si;
                    const TI di = Dinv[own0 + l];
                    const TI un = rn * di;
                    utile[l + ushift] = un;
                    const TI ui = ri * di;
                    const TI pi = it == 0 ? ui : ui + tb * P[l];
                    X[l] += ta * pi;
                    P[l] = pi;
                    Sc[l] = si;
                    Rn[l] = rn;
                    pacc[0] += (double)(rn * un);
                    pacc[2] += (double)(rn * rn);
                }
                // halo rows: the neighbours' r_i, w_i, s_{i-1} over DSMEM
                if (has_lo) {
                    const TI *rr_ = vec_lo + cur * vstride, *ww_ = vec_lo + (2 + cur) * vstride;
                    const TI *ss_ = vec_lo + (4 + nxt) * vstride;
                    for (int i = tid; i < m; i += nt) {
                        const int k = lo_base + i;
                        const TI si = it == 0 ? ww_[k] : ww_[k] + tb * ss_[k];
                        utile[i] = (rr_[k] - ta * si) * Dinv[tile0 + i];
                    }
                }
                if (has_hi) {
                    const TI *rr_ = vec_hi + cur * vstride, *ww_ = vec_hi + (2 + cur) * vstride;
                    const TI *ss_ = vec_hi + (4 + nxt) * vstride;
                    for (int i = tid; i < m; i += nt) {
                        const int k = hi_base + i;
                        const TI si = it == 0 ? ww_[k] : ww_[k] + tb * ss_[k];
                        utile[own1 - tile0 + i] = (rr_[k] - ta * si) * Dinv[own1 + i];
                    }
                }
                __syncthreads();
                for (int l = tid; l < nown; l += nt) {
                    const int node = own0 + l;
                    const int j = (int)g.divm.div((uint32_t)node), i = node - j * m;
                    const TI wn = stencil_apply<TI, TI>(Ai, n, m, node, i, j, utile, l + ushift);
                    Wn[l] = wn;
                    pacc[1] += (double)(wn * utile[l + ushift]);
                }
                cluster_sum<3, CS>(pacc, warp_buf, slots, par);
                par ^= 1;
                gamma_prev = gamma;
                alpha_prev = alpha;
                gamma = pacc[0];
                delta = pacc[1];
                rr = pacc[2];
                ++it;
            }
            total_iters += it;
            if (nonfinite) break;
            for (int l = tid; l < nown; l += nt) v[own0 + l] = v[own0 + l] + (double)X[l];
            cl.sync();
            if (!mixed) break;
        }
        if (nonfinite) {
            status = S_NONFINITE;
            break;
        }
        if (!solved && status == S_CONVERGED) status = S_MAXITER;
    }

    double qacc[1] = {0.0};
    for (int node = own0 + tid; node < own1; node += nt) {
        const int j = (int)g.divm.div((uint32_t)node), i = node - j * m;
        qacc[0] += lumped_mass(m, i, j, g.h2) * v[node];
    }
    cluster_sum<1, CS>(qacc, warp_buf, slots, par);
    if (rank == 0 && tid == 0) {
        g.q[sample] = status == S_NONFINITE ? __longlong_as_double(0x7ff8000000000000LL) : qacc[0];
        g.iters[sample] = (int32_t)(total_iters > 0x7fffffff ? 0x7fffffff : total_iters);
        g.status[sample] = status;
    }
    cl.sync();
}

// ---------------------------------------------------------------------------
// K7: Y = Q_l - Q_{l-1} and per-level sums in FP64.  One block, two passes
// (mean, then centred squares); the tree is fixed by blockDim, so the sums do
// not depend on how samples were batched.
// sums[0] = sum Y, sums[1] = sum (Y - mean Y)^2.
// ---------------------------------------------------------------------------
__global__ void level_sums_kernel(const double *__restrict__ qf, const double *__restrict__ qc, int64_t S,
                                  double *__restrict__ y, double *__restrict__ sums)
{
    __shared__ double buf[1024];
    __shared__ double mean_sh;
    double s1 = 0.0;
    for (int64_t k = threadIdx.x; k < S; k += blockDim.x) {
        const double yy = qc ? qf[k] - qc[k] : qf[k];
        if (y) y[k] = yy;
        s1 += yy;
    }
    buf[threadIdx.x] = s1;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) buf[threadIdx.x] += buf[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        sums[0] = buf[0];
        mean_sh = buf[0] / (double)S;
    }
    __syncthreads();
    const double mu = mean_sh;
    double s2 = 0.0;
    for (int64_t k = threadIdx.x; k < S; k += blockDim.x) {
        const double d = (qc ? qf[k] - qc[k] : qf[k]) - mu;
        s2 += d * d;
    }
    __syncthreads();
    buf[threadIdx.x] = s2;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) buf[threadIdx.x] += buf[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[1] = buf[0];
}

// worst-of status merge of the fine and coarse members
__global__ void merge_status_kernel(const int32_t *__restrict__ a, const int32_t *__restrict__ c, int64_t S,
                                    int32_t *__restrict__ out)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= S) return;
    out[k] = c ? (a[k] > c[k] ? a[k] : c[k]) : a[k];
}

}  // namespace mlq
