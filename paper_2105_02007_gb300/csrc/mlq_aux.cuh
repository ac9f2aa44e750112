// mlq_aux.cuh -- the non-solver kernels of libmlq (sm_103a):
//   K1 kl_synthesis_kernel    theta_e = theta_mean_e + sum_k Phi[e,k] xi_k
//                             (eq. KLlowrank), epilogue (cos 2t, sin 2t)
//   K2 stencil_setup_kernel   A = M + dt K(theta) as a stored 7-point stencil
//                             (Sec. 3.1 mass/stiffness, eq. AdmV conductivity)
//   K7 level_sums_kernel      Y = Q_l - Q_{l-1} and per-level FP64 sums
//                             (eq. StandardML)
// Included by the host runtime only (one definition per library).
#pragma once

#include "mlq_kernels.cuh"
#include "mlq_mg.cuh"

namespace mlq {

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

// ---------------------------------------------------------------------------
// Multigrid set-up (see mlq_mg.cuh): coarse conductivities and stencils.
// ---------------------------------------------------------------------------
// Dbar of level c >= 1 from level c-1 (level 0 given as cos/sin(2 theta)).
// The four children of coarse square (I, J) in the finer mesh:
//   lower(I,J): lower(2I,2J), lower(2I+1,2J), lower(2I+1,2J+1), upper(2I+1,2J)
//   upper(I,J): upper(2I,2J), upper(2I,2J+1), upper(2I+1,2J+1), lower(2I,2J+1)
__global__ void mg_coarsen_kernel(const double *__restrict__ cs2, const D3 *__restrict__ dfine, int mf, int S,
                                  double s_l, double s_t, D3 *__restrict__ dcoarse)
{
    const int mc = (mf + 1) / 2;
    const int nec = 2 * (mc - 1) * (mc - 1), nef = 2 * (mf - 1) * (mf - 1);
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (e >= nec || s >= S) return;
    const int cell = e >> 1, up = e & 1;
    const int I = cell % (mc - 1), J = cell / (mc - 1);
    const int cf = mf - 1;
    auto el = [&](int ci, int cj, int u) { return 2 * (ci + cf * cj) + u; };
    int ch[4];
    if (!up) {
        ch[0] = el(2 * I, 2 * J, 0);
        ch[1] = el(2 * I + 1, 2 * J, 0);
        ch[2] = el(2 * I + 1, 2 * J + 1, 0);
        ch[3] = el(2 * I + 1, 2 * J, 1);
    } else {
        ch[0] = el(2 * I, 2 * J, 1);
        ch[1] = el(2 * I, 2 * J + 1, 1);
        ch[2] = el(2 * I + 1, 2 * J + 1, 1);
        ch[3] = el(2 * I, 2 * J + 1, 0);
    }
    double a = 0.0, b = 0.0, c = 0.0;
    if (cs2) {
        const double sbar = 0.5 * (s_l + s_t), hds = 0.5 * (s_l - s_t);
        for (int k = 0; k < 4; ++k) {
            const double *q = cs2 + ((size_t)s * nef + ch[k]) * 2;
            a += sbar + hds * q[0];
            b += hds * q[1];
            c += sbar - hds * q[0];
        }
    } else {
        for (int k = 0; k < 4; ++k) {
            const D3 d = dfine[(size_t)s * nef + ch[k]];
            a += d.a;
            b += d.b;
            c += d.c;
        }
    }
    dcoarse[(size_t)s * nec + e] = D3{(float)(0.25 * a), (float)(0.25 * b), (float)(0.25 * c)};
}

// FP32 stencil (diag, E, N, NE, 1/diag) of A_c = M_c + dt K_c(Dbar_c) on the
// m x m level (same element formulas as stencil_setup_kernel).
__global__ void mg_stencil_kernel(const D3 *__restrict__ dbar, int m, double dt, int S, float *__restrict__ A)
{
    const int n = m * m;
    const int node = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (node >= n || s >= S) return;
    const int i = node % m, j = node / m;
    const int mc = m - 1, ne = 2 * mc * mc;
    const double h = 1.0 / (double)(m - 1);
    const double mdiag = h * h / 12.0, moff = h * h / 24.0;
    const D3 *d = dbar + (size_t)s * ne;
    auto el = [&](int ci, int cj, int u) { return d[2 * (ci + mc * cj) + u]; };
    double diag = 0.0, east = 0.0, north = 0.0, nea = 0.0;
    if (i < mc && j < mc) {
        D3 D = el(i, j, 0);
        diag += 0.5 * D.a * dt + mdiag;
        east += -0.5 * (D.a - D.b) * dt + moff;
        nea += -0.5 * D.b * dt + moff;
        D = el(i, j, 1);
        diag += 0.5 * D.c * dt + mdiag;
        nea += -0.5 * D.b * dt + moff;
        north += 0.5 * (D.b - D.c) * dt + moff;
    }
    if (i >= 1 && j < mc) {
        const D3 D = el(i - 1, j, 0);
        diag += 0.5 * (D.a - 2.0 * D.b + D.c) * dt + mdiag;
        north += 0.5 * (D.b - D.c) * dt + moff;
    }
    if (i >= 1 && j >= 1) {
        D3 D = el(i - 1, j - 1, 0);
        diag += 0.5 * D.c * dt + mdiag;
        D = el(i - 1, j - 1, 1);
        diag += 0.5 * D.a * dt + mdiag;
    }
    if (i < mc && j >= 1) {
        const D3 D = el(i, j - 1, 1);
        diag += 0.5 * (D.a - 2.0 * D.b + D.c) * dt + mdiag;
        east += -0.5 * (D.a - D.b) * dt + moff;
    }
    float *a = A + (size_t)s * kSlots2D * n;
    a[node] = (float)diag;
    a[n + node] = (float)east;
    a[2 * n + node] = (float)north;
    a[3 * n + node] = (float)nea;
    a[4 * n + node] = (float)(1.0 / diag);
}

}  // namespace mlq
