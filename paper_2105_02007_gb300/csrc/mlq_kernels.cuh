// mlq_kernels.cuh -- device code of the slab solvers of libmlq (sm_103a).
//
// The per-sample forward solve of the stochastic monodomain equation: all
// time blocks of one sample run inside one cluster of CTAs -- FHN reaction
// and consistent-mass load (eq. mono_disc), Jacobi-PCG per block (multiple
// time blocks, Sec. 3.3) with FP64 iterative refinement in the mixed path,
// and the QoI m^T v.  The set-up and reduction kernels are in mlq_aux.cuh.
#pragma once

#include <cooperative_groups.h>
#include <cstdint>
#include <cuda_runtime.h>

#include "mlq_points.cuh"

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
// Slab solver.
// ---------------------------------------------------------------------------

// Solutions of the last blocks kept for the initial guess of the next one
// (multigrid kernels): v_j lives in buffer j mod kVRing of [kVRing][S][n].
// The guess of block `step` (from v_step, v_step-1, ...) is the polynomial
// extrapolation of order guess_order(step): the value at t + dt of the
// polynomial through the last p + 1 solutions.  The order starts at 0 and
// rises by one every two blocks: the first blocks follow a discontinuous
// initial state, and a stencil reaching back to it or to the first rough
// solutions makes a worse guess than v_step itself.
constexpr int kVRing = 5;
constexpr int kGuessOrderMax = kVRing - 1;

__host__ __device__ inline int guess_order(int step)
{
    return step < 3 ? 0 : ((step - 1) / 2 < kGuessOrderMax ? (step - 1) / 2 : kGuessOrderMax);
}

// value at t_{n+1} of the polynomial of order p through v0 = v_n, v1 =
// v_{n-1}, ... (binomial weights: the p+1-th difference vanishes)
__host__ __device__ inline double extrapolate(int p, double v0, double v1, double v2, double v3, double v4)
{
    switch (p) {
    case 0: return v0;
    case 1: return 2.0 * v0 - v1;
    case 2: return 3.0 * v0 - 3.0 * v1 + v2;
    case 3: return 4.0 * v0 - 6.0 * v1 + 4.0 * v2 - v3;
    default: return 5.0 * v0 - 10.0 * v1 + 10.0 * v2 - 5.0 * v3 + v4;
    }
}

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
    double *v;                    // [S][n]; [kVRing][S][n] for the multigrid kernel
    double *w;                    // [2][S][n]
    double *b;                    // [S][n]
    double *y;                    // [S][n] v + dt R(v, w) per node (multigrid kernel), else null
    TI *r, *s, *wc;               // [2][S][n] each
    TI *p, *x;                    // [S][n]
    const double *v0, *w0;        // [n] or null
    double radius2;               // initial disc, used when v0 is null
    int S;
    double *q;                    // [S]
    int32_t *iters, *status;      // [S]
    PointArgs pq;                 // point QoIs (npts = 0: none)
    // time scheme: 0 = the two-variable FHN with the reaction explicit per
    // block (backward Euler); 1 = the paper's scheme (PaperScheme below)
    int scheme;
    double theta;                 // 1 backward Euler, 0.5 Crank-Nicolson (the stencil holds M + theta dt K)
    double alpha, u_rest, u_th, u_peak;       // I_ion(u) = alpha (u - u_rest)(u - u_th)(u - u_peak)
    double amp, sigma2, t1, x0, y0;           // I_app = (u_rest + amp exp(-|x - x0|^2 / sigma2)) on [0, t1)
};

// The paper's time scheme (Sec. 3.1 eq. st-system with eq. mono_disc, the
// current of eq. ionic_term, the stimulus of Sec. 5.1), per block k -> k+1:
//   (M + theta dt K) u + dt M I_ion(u) = c,
//   c = (M - (1 - theta) dt K) u_k + dt M (theta g(t_{k+1}) + (1 - theta) g(t_k)),
// g the nodal stimulus.  With A = M + theta dt K the kernels form
// c = M y - ((1 - theta) / theta) A u_k, y = u_k / theta + dt (theta g_{k+1} +
// (1 - theta) g_k), and solve the nonlinear system by chord-Newton sweeps:
// the FP64 residual F = c - A u - dt M I_ion(u) of the current iterate, an
// inner PCG on A d = F, u += d, until ||F|| <= rtol ||c||.  A stays the SPD
// matrix of the set-up, so the inner solver is CG; the sweeps converge
// linearly with the factor ~ dt max |I_ion'| (about 0.07 at the paper's
// dt and constants) to the same root as Newton with the full Jacobian.
template <typename A>
__device__ __forceinline__ double paper_ionic(const A &g, double u)
{
    return g.alpha * (u - g.u_rest) * (u - g.u_th) * (u - g.u_peak);
}

template <typename A>
__device__ __forceinline__ double paper_stimulus(const A &g, double x, double y, double t)
{
    if (!(t >= 0.0 && t < g.t1)) return 0.0;
    const double dx = x - g.x0, dy = y - g.y0;
    return g.u_rest + g.amp * exp(-(dx * dx + dy * dy) / g.sigma2);
}

template <typename T>
__device__ __forceinline__ T ldcg(const T *p) { return __ldcg(p); }

// ---------------------------------------------------------------------------
// Cluster-wide sums.
//
// Each thread passes NV partial sums in its own precision TA (FP32 in the
// mixed path: the thread's own few products).  They are summed over the warp
// in TA and converted to FP64;
// warp 0 adds the per-warp values with a butterfly over its lanes (FP64),
// giving the CTA's total; with CS > 1 the CTA totals are exchanged over DSMEM
// after a cluster barrier and added with a butterfly over CS lanes.  Every
// CTA therefore gets bit-identical totals, independent of timing.  Thread 0
// hands the totals to `fin`; its writes to shared memory are visible to the
// whole CTA on return.
//   wsl: [32][4] doubles (per-warp values), csl: [2][4] doubles (CTA totals,
//   alternating by `par` so that a slow reader never sees the next round).
// ---------------------------------------------------------------------------
template <int NV, int CS, typename TA, typename F>
__device__ __forceinline__ void cluster_reduce(TA (&v)[NV], double (*wsl)[4], double (*csl)[4], int par, F &&fin)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    // a thread's partial (its own few products) and the warp butterfly in the
    // thread precision, every sum above the warp in FP64 (widening before the
    // butterfly measured 6 % more time for the estimate, with the same result
    // to 2e-14: the sums only set the scalars of the FP32 inner solve, whose
    // FP64 refinement decides the accuracy)
    double dv[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
        dv[k] = (double)v[k];
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) wsl[warp][k] = dv[k];
    }
    __syncthreads();
    double acc[NV];
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] = lane < nwarp ? wsl[lane][k] : 0.0;
        for (int o = 1; o < nwarp; o <<= 1) {
#pragma unroll
            for (int k = 0; k < NV; ++k) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
        }
    }
    if constexpr (CS == 1) {
        if (threadIdx.x == 0) fin(acc);
    } else {
        if (threadIdx.x == 0) {
#pragma unroll
            for (int k = 0; k < NV; ++k) csl[par][k] = acc[k];
        }
        cg::cluster_group cl = cg::this_cluster();
        cl.sync();
        if (warp == 0) {
            double t[NV];
            const double *rs = lane < CS ? cl.map_shared_rank(&csl[par][0], lane) : nullptr;
#pragma unroll
            for (int k = 0; k < NV; ++k) t[k] = lane < CS ? rs[k] : 0.0;
#pragma unroll
            for (int o = 1; o < CS; o <<= 1) {
#pragma unroll
                for (int k = 0; k < NV; ++k) t[k] += __shfl_xor_sync(0xffffffffu, t[k], o);
            }
            if (lane == 0) fin(t);
        }
    }
    __syncthreads();
}

// The FitzHugh-Nagumo terms of a time block: the ionic current R(v, w) =
// v (v - a)(1 - v) - w and the recovery increment v - gam w, added times dt
// to the FP64 state.  F32 evaluates them in FP32: the increments are O(dt)
// against O(1) state values, so their rounding moves y and w by ~1e-10
// absolute per block, and GB300 issues FP64 at 1/64 of the FP32 rate.  The
// Jacobi kernels of the mixed path (each block starts from v^n) use it; the
// multigrid kernels keep FP64, because their initial guess extrapolates the
// last five block solutions with weights of magnitude up to 10 (sum 31),
// which amplifies that rounding noise into the first residual of every block
// (measured: twice the CG iterations per block at 257 x 257).
template <bool F32>
__device__ __forceinline__ double reaction(double v, double w, double a)
{
    if constexpr (F32) {
        const float vf = (float)v, af = (float)a;
        return (double)(vf * (vf - af) * (1.0f - vf) - (float)w);
    } else {
        return v * (v - a) * (1.0 - v) - w;
    }
}
template <bool F32>
__device__ __forceinline__ double recovery(double v, double w, double gam)
{
    if constexpr (F32) return (double)((float)v - (float)gam * (float)w);
    else return v - gam * w;
}

// 1/d in FP64 from an FP32 reciprocal and one Newton-Raphson step
// r <- r + r (1 - d r) (the error squares: ~2^-46 relative), for d well
// inside the FP32 range; used for the PCG scalars of the normalised inner
// problem, whose magnitudes are bounded away from FP32 limits.
__device__ __forceinline__ double rcp_newton(double d)
{
    double r = (double)(1.0f / (float)d);
    return fma(r, fma(-d, r, 1.0), r);
}

// Walks the nodes own0 + tid, own0 + tid + nt, ... keeping (i, j) without
// a division per node.
struct NodeWalk {
    int i, j, di, dj, m;
    __device__ __forceinline__ void init(int node, int nt, int m_)
    {
        m = m_;
        j = node / m;
        i = node - j * m;
        dj = nt / m;
        di = nt - dj * m;
    }
    __device__ __forceinline__ void next()
    {
        i += di;
        j += dj;
        if (i >= m) {
            i -= m;
            ++j;
        }
    }
};

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
    // one path for every node (boundary nodes do not split their warp): a
    // coupling across the boundary has a zero slot (the stencil set-up adds
    // nothing for a missing neighbour), so wrapping to the next row adds
    // exactly nothing; an index outside the array is replaced by the node
    // and its slot by 0
    (void)i;
    (void)j;
    const bool e = node + 1 < n, w = node >= 1, no = node + m < n, so = node >= m, ne = node + m + 1 < n,
               sw = node >= m + 1;
    const double ce = e ? A[n + node] : 0.0, cw = w ? A[n + node - 1] : 0.0;
    const double cn = no ? A[2 * n + node] : 0.0, cs = so ? A[2 * n + node - m] : 0.0;
    const double cne = ne ? A[3 * n + node] : 0.0, csw = sw ? A[3 * n + node - m - 1] : 0.0;
    const double x0 = ldcg(x + node), xe = ldcg(x + (e ? node + 1 : node)), xw = ldcg(x + (w ? node - 1 : node));
    const double xn = ldcg(x + (no ? node + m : node)), xs = ldcg(x + (so ? node - m : node));
    const double xne = ldcg(x + (ne ? node + m + 1 : node)), xsw = ldcg(x + (sw ? node - m - 1 : node));
    double acc = A[node] * x0;
    acc += ce * xe;
    acc += cw * xw;
    acc += cn * xn;
    acc += cs * xs;
    acc += cne * xne;
    acc += csw * xsw;
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

// ---------------------------------------------------------------------------
// Slab solver: every time block of one sample in one cluster of CS CTAs.
//
// CTA `rank` owns rows [r0, r1) of the m x m grid.  Per time block (multiple
// time blocks of the paper's Sec. 3.3, one backward-Euler step each):
//   load   y = v + dt R(v, w) on the rows [r0-1, r1+1), b = M y,
//          w <- w + dt eps (v - gam w), r = b - A v            (eq. mono_disc)
//   sweeps inner Jacobi-PCG on A d = r from d = 0, then v += d and a new FP64
//          residual; the mixed path repeats until ||b - A v|| <= rtol ||b||,
//          the FP64 path runs one sweep to that tolerance.
// The PCG is the Chronopoulos-Gear form (one reduction per iteration):
//   s_i = w_i + b_i s_{i-1},  r_{i+1} = r_i - a_i s_i,  u_{i+1} = D^-1 r_{i+1},
//   w_{i+1} = A u_{i+1},  g = (r, u),  d = (w, u),
//   b_i = g_i / g_{i-1},  a_i = g_i / (d_i - b_i g_i / a_{i-1}).
// The halo rows of u_{i+1} are recomputed from the neighbours' r_i, w_i,
// s_{i-1} (double-buffered), so an iteration needs one cluster barrier.
//
// RES = true: the PCG vectors of a CTA's rows live in its shared memory and
// the neighbours' rows are read over DSMEM; RES = false: they live in global
// memory (halo rows through L2).  The FP64 state v, w, b is in global memory.
//
// Shared layout (RES), identical in every CTA of the cluster:
//   utile  (rows_max + 2) * m   TI   rows [lo, hi) of the next iterate
//   R0 R1 W0 W1 S0 S1 P X       nmax TI each, own nodes, local index
//   ytile  (rows_max + 2) * m   FP64, aliases S0..X (dead while a block's load
//          vector is formed)
// Without RES only utile / ytile (aliased) are in shared memory.
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

__host__ __device__ inline SmemPlan smem_plan(int m, int cs, int ti_bytes, bool resident)
{
    SmemPlan pl;
    const int rows = (m + cs - 1) / cs;
    pl.nmax = rows * m;
    pl.tile = (rows + 2 < m ? rows + 2 : m) * m;
    if (!resident) {
        pl.off_vec = 0;
        pl.vec_bytes = 0;
        pl.off_y = 0;
        pl.total = align16(pl.tile * 8);
        return pl;
    }
    pl.off_vec = align16(pl.tile * ti_bytes);
    pl.vec_bytes = align16(pl.nmax * ti_bytes);
    pl.off_y = pl.off_vec + 4 * pl.vec_bytes;
    const int end_vec = pl.off_vec + 8 * pl.vec_bytes;
    const int end_y = pl.off_y + align16(pl.tile * 8);
    pl.total = end_vec > end_y ? end_vec : end_y;
    return pl;
}

// control words written by thread 0, read by every thread
struct Ctl {
    double alpha, beta;
    double s0, s1;      // broadcast sums (load / residual phases)
    int code;           // 0 continue, 1 converged, 2 max_iter, 3 non-finite
};

template <bool RES, typename T>
__device__ __forceinline__ T ld_halo(const T *p)
{
    if constexpr (RES) return *p;   // neighbour's shared memory over DSMEM
    else return __ldcg(p);          // another CTA's rows: bypass L1
}

template <typename TI, int CS, bool RES>
__global__ void __launch_bounds__(512, 1) slab_solve_kernel(SolveArgs<TI> g)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double wsl[32][4];
    __shared__ double csl[2][4];
    __shared__ Ctl ctl;

    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int sample = blockIdx.x / CS;
    const int m = g.m, n = g.n;
    const int r0 = (int)(((int64_t)m * rank) / CS), r1 = (int)(((int64_t)m * (rank + 1)) / CS);
    const int lo = r0 > 0 ? r0 - 1 : 0, hi = r1 < m ? r1 + 1 : m;
    const int own0 = r0 * m, own1 = r1 * m, tile0 = lo * m, tile1 = hi * m;
    const int nown = own1 - own0;
    const int tid = threadIdx.x, nt = blockDim.x;
    const bool has_lo = rank > 0, has_hi = rank + 1 < CS;
    const SmemPlan pl = smem_plan(m, CS, (int)sizeof(TI), RES);

    TI *utile = reinterpret_cast<TI *>(smem_raw);
    double *ytile = reinterpret_cast<double *>(smem_raw + pl.off_y);
    const int ushift = own0 - tile0;

    const size_t so = (size_t)sample * n;
    const size_t SN = (size_t)g.S * n;
    const double *A64 = g.A64 + (size_t)sample * kSlots2D * n;
    const TI *Ai = g.Ai + (size_t)sample * kSlots2D * n;
    const TI *Dinv = Ai + 4 * (size_t)n;
    double *v = g.v + so;
    double *wb0 = g.w + so;
    double *b = g.b + so;

    // PCG vectors: own rows (local index) and the neighbours' boundary rows
    TI *R, *W, *Sv, *P, *X;
    const TI *Rlo = nullptr, *Wlo = nullptr, *Slo = nullptr, *Rhi = nullptr, *Whi = nullptr, *Shi = nullptr;
    size_t vs;  // stride between the two halves of a double buffer
    if constexpr (RES) {
        TI *vec0 = reinterpret_cast<TI *>(smem_raw + pl.off_vec);
        vs = (size_t)(pl.vec_bytes / (int)sizeof(TI));
        R = vec0;
        W = vec0 + 2 * vs;
        Sv = vec0 + 4 * vs;
        P = vec0 + 6 * vs;
        X = vec0 + 7 * vs;
        if (has_lo) {
            const int r0_lo = (int)(((int64_t)m * (rank - 1)) / CS);
            const TI *nb = cl.map_shared_rank(vec0, rank - 1) + (r0 - 1 - r0_lo) * m;
            Rlo = nb;
            Wlo = nb + 2 * vs;
            Slo = nb + 4 * vs;
        }
        if (has_hi) {
            const TI *nb = cl.map_shared_rank(vec0, rank + 1);
            Rhi = nb;
            Whi = nb + 2 * vs;
            Shi = nb + 4 * vs;
        }
    } else {
        vs = SN;
        R = g.r + so + own0;
        W = g.wc + so + own0;
        Sv = g.s + so + own0;
        P = g.p + so + own0;
        X = g.x + so + own0;
        Rlo = g.r + so + tile0;
        Wlo = g.wc + so + tile0;
        Slo = g.s + so + tile0;
        Rhi = g.r + so + own1;
        Whi = g.wc + so + own1;
        Shi = g.s + so + own1;
    }
    int par = 0;

    for (int node = own0 + tid; node < own1; node += nt) {
        double v0, w0;
        if (g.v0) {
            v0 = g.v0[node];
            w0 = g.w0 ? g.w0[node] : 0.0;
        } else if (g.scheme == 1) {
            v0 = g.u_rest;   // the paper's scheme starts at rest; the stimulus excites
            w0 = 0.0;
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
    PointState pst;
    const bool pth = rank == 0 && tid < g.pq.npts;   // point QoI threads
    if (pth) point_record(g.pq, sample, g.nsteps, g.dt, v, pst);
    const bool paper = g.scheme == 1;
    const double hgrid = 1.0 / (double)(m - 1);

    int wpar = 0;
    int64_t total_iters = 0;     // thread 0's count
    int32_t status = S_CONVERGED;
    constexpr bool mixed = sizeof(TI) == 4;
    const double dt = g.dt;

    for (int step = 0; step < g.nsteps; ++step) {
        // ---- block load
        const double *wcur = wb0 + wpar * SN;
        double *wnext = wb0 + (wpar ^ 1) * SN;
        const double cpre = paper ? (1.0 - g.theta) / g.theta : 0.0;
        for (int node = tile0 + tid; node < tile1; node += nt) {
            const double vv = ldcg(v + node), ww = ldcg(wcur + node);
            if (paper) {
                const int j = node / m, i = node - j * m;
                const double x = i * hgrid, y = j * hgrid;
                ytile[node - tile0] = vv / g.theta + dt * (g.theta * paper_stimulus(g, x, y, (step + 1) * dt) +
                                                           (1.0 - g.theta) * paper_stimulus(g, x, y, step * dt));
            } else {
                ytile[node - tile0] = vv + dt * reaction<mixed>(vv, ww, g.a);
            }
        }
        __syncthreads();
        if (paper) {
            // c = M y - ((1 - theta) / theta) A u_k, then the ionic current of the
            // iterate (u_k) into the tile for the first residual
            NodeWalk nw;
            nw.init(own0 + tid, nt, m);
            for (int l = tid; l < nown; l += nt, nw.next()) {
                const int node = own0 + l;
                double bb = mass_apply(m, nw.i, nw.j, g.h2, ytile, node - tile0);
                if (cpre != 0.0) bb -= cpre * stencil_apply_global(A64, n, m, node, nw.i, nw.j, v);
                b[node] = bb;
            }
            __syncthreads();
            for (int node = tile0 + tid; node < tile1; node += nt) ytile[node - tile0] = paper_ionic(g, ldcg(v + node));
            __syncthreads();
        }
        {
            double acc[2] = {0.0, 0.0};
            NodeWalk nw;
            nw.init(own0 + tid, nt, m);
            for (int l = tid; l < nown; l += nt, nw.next()) {
                const int node = own0 + l;
                double bb, rr;
                if (paper) {
                    bb = b[node];
                    rr = bb - stencil_apply_global(A64, n, m, node, nw.i, nw.j, v) -
                         dt * mass_apply(m, nw.i, nw.j, g.h2, ytile, node - tile0);
                } else {
                    bb = mass_apply(m, nw.i, nw.j, g.h2, ytile, node - tile0);
                    b[node] = bb;
                    const double vv = v[node], ww = wcur[node];
                    wnext[node] = ww + dt * g.eps * recovery<mixed>(vv, ww, g.gam);
                    rr = bb - stencil_apply_global(A64, n, m, node, nw.i, nw.j, v);
                }
                R[l] = (TI)rr;
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
                if (paper) {
                    // the ionic current of the iterate (the tile's FP64 slots are
                    // free between inner solves)
                    for (int node = tile0 + tid; node < tile1; node += nt)
                        ytile[node - tile0] = paper_ionic(g, ldcg(v + node));
                    __syncthreads();
                }
                NodeWalk nw;
                nw.init(own0 + tid, nt, m);
                for (int l = tid; l < nown; l += nt, nw.next()) {
                    const int node = own0 + l;
                    double rr = b[node] - stencil_apply_global(A64, n, m, node, nw.i, nw.j, v);
                    if (paper) rr -= dt * mass_apply(m, nw.i, nw.j, g.h2, ytile, node - tile0);
                    R[l] = (TI)rr;
                    racc[0] += rr * rr;
                }
                cluster_reduce<1, CS>(racc, wsl, csl, par, [&](double(&t)[1]) { ctl.s1 = t[0]; });
                par ^= 1;
                rnorm2 = ctl.s1;
                if (!isfinite(rnorm2)) { nonfinite = true; break; }
            }
            if (rnorm2 <= tol_out2) { solved = true; break; }
            // the paper's scheme: each sweep is one chord-Newton step, whose
            // linear system needs no more than the contraction of the step
            const double tol_in2 = paper ? fmax((mixed ? g.rtol_in * g.rtol_in : 1e-12) * rnorm2, 0.25 * tol_out2)
                                         : (mixed ? g.rtol_in * g.rtol_in * rnorm2 : tol_out2);

            // ---- inner PCG init: u0 = D^-1 r0 on the tile, w0 = A u0, x = 0
            for (int l = tid; l < nown; l += nt) utile[l + ushift] = R[l] * Dinv[own0 + l];
            if (has_lo)
                for (int i = tid; i < m; i += nt) utile[i] = ld_halo<RES>(Rlo + i) * Dinv[tile0 + i];
            if (has_hi)
                for (int i = tid; i < m; i += nt)
                    utile[own1 - tile0 + i] = ld_halo<RES>(Rhi + i) * Dinv[own1 + i];
            __syncthreads();
            // thread 0's recurrence state: eta_i = (p_i, A p_i) = delta_i - beta_i^2 eta_{i-1}
            double gamma_prev = 1.0, eta_prev = 1.0;
            int it = 0;
            auto decide = [&](double gamma, double delta, double rr) {
                // runs on thread 0 only
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
            {
                TI iacc[3] = {(TI)0, (TI)0, (TI)0};
                NodeWalk nw;
                nw.init(own0 + tid, nt, m);
                for (int l = tid; l < nown; l += nt, nw.next()) {
                    const TI u0 = utile[l + ushift];
                    const TI w0 = stencil_apply<TI, TI>(Ai, n, m, own0 + l, nw.i, nw.j, utile, l + ushift);
                    W[l] = w0;
                    X[l] = (TI)0;
                    const TI r0v = R[l];
                    iacc[0] += r0v * u0;
                    iacc[1] += w0 * u0;
                    iacc[2] += r0v * r0v;
                }
                cluster_reduce<3, CS>(iacc, wsl, csl, par, [&](double(&t)[3]) { decide(t[0], t[1], t[2]); });
                par ^= 1;
            }
            while (true) {
                const int code = ctl.code;
                if (code != 0) {
                    if (code == 3) nonfinite = true;
                    else if (code == 1) solved = !mixed;
                    else status = status == S_CONVERGED ? S_MAXITER : status;
                    break;
                }
                const TI ta = (TI)ctl.alpha, tb = (TI)ctl.beta;
                const int cur = it & 1, nxt = cur ^ 1;
                TI *Rc = R + cur * vs, *Rn = R + nxt * vs;
                TI *Wc = W + cur * vs, *Wn = W + nxt * vs;
                TI *Sc = Sv + cur * vs, *Sp = Sv + nxt * vs;
                TI pacc[3] = {(TI)0, (TI)0, (TI)0};
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
                    pacc[0] += rn * un;
                    pacc[2] += rn * rn;
                }
                if (has_lo) {
                    const TI *rr_ = Rlo + cur * vs, *ww_ = Wlo + cur * vs, *ss_ = Slo + nxt * vs;
                    for (int i = tid; i < m; i += nt) {
                        const TI wi = ld_halo<RES>(ww_ + i);
                        const TI si = it == 0 ? wi : wi + tb * ld_halo<RES>(ss_ + i);
                        utile[i] = (ld_halo<RES>(rr_ + i) - ta * si) * Dinv[tile0 + i];
                    }
                }
                if (has_hi) {
                    const TI *rr_ = Rhi + cur * vs, *ww_ = Whi + cur * vs, *ss_ = Shi + nxt * vs;
                    for (int i = tid; i < m; i += nt) {
                        const TI wi = ld_halo<RES>(ww_ + i);
                        const TI si = it == 0 ? wi : wi + tb * ld_halo<RES>(ss_ + i);
                        utile[own1 - tile0 + i] = (ld_halo<RES>(rr_ + i) - ta * si) * Dinv[own1 + i];
                    }
                }
                __syncthreads();
                {
                    NodeWalk nw;
                    nw.init(own0 + tid, nt, m);
                    for (int l = tid; l < nown; l += nt, nw.next()) {
                        const TI wn = stencil_apply<TI, TI>(Ai, n, m, own0 + l, nw.i, nw.j, utile, l + ushift);
                        Wn[l] = wn;
                        pacc[1] += wn * utile[l + ushift];
                    }
                }
                ++it;
                cluster_reduce<3, CS>(pacc, wsl, csl, par, [&](double(&t)[3]) { decide(t[0], t[1], t[2]); });
                par ^= 1;
            }
            total_iters += it;
            if (nonfinite) break;
            for (int l = tid; l < nown; l += nt) v[own0 + l] = v[own0 + l] + (double)X[l];
            cl.sync();
            if (!mixed && !paper) break;
        }
        if (nonfinite) {
            status = S_NONFINITE;
            break;
        }
        if (!solved && status == S_CONVERGED) status = S_MAXITER;
        if (pth) point_record(g.pq, sample, g.nsteps, dt, v, pst);
    }
    if (pth) point_finish(g.pq, sample, g.nsteps, pst);

    double qacc[1] = {0.0};
    {
        NodeWalk nw;
        nw.init(own0 + tid, nt, m);
        for (int l = tid; l < nown; l += nt, nw.next()) qacc[0] += lumped_mass(m, nw.i, nw.j, g.h2) * v[own0 + l];
    }
    cluster_reduce<1, CS>(qacc, wsl, csl, par, [&](double(&t)[1]) { ctl.s0 = t[0]; });
    if (rank == 0 && tid == 0) {
        g.q[sample] = status == S_NONFINITE ? __longlong_as_double(0x7ff8000000000000LL) : ctl.s0;
        g.iters[sample] = (int32_t)(total_iters > 0x7fffffff ? 0x7fffffff : total_iters);
        g.status[sample] = status;
    }
    // keep every CTA's shared memory alive until all remote reads are done
    cl.sync();
}

// ---------------------------------------------------------------------------
// Register-resident slab solver (mixed path: FP32 inner PCG).
//
// Same algorithm and decomposition as slab_solve_kernel, laid out for the
// SM: thread t of a CTA owns the nodes l = t + k*nt (k < NPT) of the CTA's
// rows and keeps their PCG vectors r, w, s, p, x in registers for the whole
// run.  Shared memory holds, per node, the stencil row (diag, E, N, NE) as a
// float4 and D^-1; the W, S, SW entries of a row are the E, N, NE entries of
// the neighbouring nodes (A is symmetric), so the float4 array also covers
// the row below the CTA's band.  The iterate u goes through a zero-padded
// shared tile, so the stencil apply has no boundary branches (missing
// neighbours have zero coefficients).  The first and last own row of r, w, s
// are exported, double-buffered, for the neighbouring CTAs, which rebuild
// their halo rows of u from them over DSMEM.  The block load vector
// b = M (v + dt R(v, w)) is formed from the FP64 state in global memory,
// evaluating y = v + dt R at each stencil point.
//
// Shared layout (bytes), identical in every CTA of the cluster:
//   c0     1 + (rows_max + 1) * m  float4   (pad, row r0-1, own rows)
//   dinv   rows_max * m            float
//   utile  1 + (rows_max + 2) * m + 1 float  (pad, rows r0-1 .. r1, pad)
//   ex     [2 parity][2 rows: first, last][3: r, w, s][m] floats
// ---------------------------------------------------------------------------
struct RegPlan {
    int nmax, rows;
    int off_dinv, off_u, off_ex, total;
    int csize, usize;
};

__host__ __device__ inline RegPlan reg_plan(int m, int cs)
{
    RegPlan pl;
    pl.rows = (m + cs - 1) / cs;
    pl.nmax = pl.rows * m;
    pl.csize = 1 + (pl.rows + 1) * m;
    pl.off_dinv = align16(pl.csize * 16);
    pl.off_u = pl.off_dinv + align16(pl.nmax * 4);
    pl.usize = 1 + (pl.rows + 2) * m + 1;
    pl.off_ex = pl.off_u + align16(pl.usize * 4);
    pl.total = pl.off_ex + align16(2 * 2 * 3 * m * 4);
    return pl;
}

// y = v + dt R(v, w) at node q (FP64 state in global memory, through L2)
template <bool F32 = false>
__device__ __forceinline__ double load_y(const double *v, const double *w, int q, double dt, double a)
{
    const double vv = __ldcg(v + q), ww = __ldcg(w + q);
    return vv + dt * reaction<F32>(vv, ww, a);
}

// b_P = (M y)_P with y evaluated at the stencil points (see mass_apply)
template <bool F32>
__device__ __forceinline__ double mass_apply_y(int m, int i, int j, double h2, const double *v, const double *w,
                                               int node, double dt, double a)
{
    const int mc = m - 1;
    const bool cij = (i < mc && j < mc), cim = (i >= 1 && j < mc), cmm = (i >= 1 && j >= 1),
               cjm = (i < mc && j >= 1);
    const int ninc = 2 * cij + cim + 2 * cmm + cjm;
    double acc = (double)ninc * (h2 / 12.0) * load_y<F32>(v, w, node, dt, a);
    const double e = h2 / 24.0;
    if (i + 1 < m) acc += e * (double)(cij + cjm) * load_y<F32>(v, w, node + 1, dt, a);
    if (i > 0) acc += e * (double)(cim + cmm) * load_y<F32>(v, w, node - 1, dt, a);
    if (j + 1 < m) acc += e * (double)(cij + cim) * load_y<F32>(v, w, node + m, dt, a);
    if (j > 0) acc += e * (double)(cjm + cmm) * load_y<F32>(v, w, node - m, dt, a);
    if (i + 1 < m && j + 1 < m) acc += e * (double)(2 * cij) * load_y<F32>(v, w, node + m + 1, dt, a);
    if (i > 0 && j > 0) acc += e * (double)(2 * cmm) * load_y<F32>(v, w, node - m - 1, dt, a);
    return acc;
}

template <int CS, int NPT>
__global__ void __launch_bounds__(NPT >= 12 ? (NPT >= 16 ? 512 : 384) : 512, 1)
    slab_solve_reg_kernel(SolveArgs<float> g)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double wsl[32][4];
    __shared__ double csl[2][4];
    __shared__ Ctl ctl;

    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int sample = blockIdx.x / CS;
    const int m = g.m, n = g.n;
    const int r0 = (int)(((int64_t)m * rank) / CS), r1 = (int)(((int64_t)m * (rank + 1)) / CS);
    const int own0 = r0 * m, own1 = r1 * m;
    const int nown = own1 - own0;
    const int tid = threadIdx.x, nt = blockDim.x;
    const bool has_lo = rank > 0, has_hi = rank + 1 < CS;
    const RegPlan pl = reg_plan(m, CS);

    float4 *c0 = reinterpret_cast<float4 *>(smem_raw);                 // index 1 + m + l for own l
    float *dv = reinterpret_cast<float *>(smem_raw + pl.off_dinv);      // own l
    float *ut = reinterpret_cast<float *>(smem_raw + pl.off_u);         // index 1 + m + l for own l
    float *ex = reinterpret_cast<float *>(smem_raw + pl.off_ex);        // [par][row][var][m]
    const int UB = 1 + m;                 // c0 / utile index of own local index 0
    const int Uhi = 1 + m + nown;         // utile index of the upper halo row
    const float *ex_lo = has_lo ? cl.map_shared_rank(ex, rank - 1) : nullptr;
    const float *ex_hi = has_hi ? cl.map_shared_rank(ex, rank + 1) : nullptr;
    auto exi = [m](int par, int row, int var) { return ((par * 2 + row) * 3 + var) * m; };

    const size_t so = (size_t)sample * n;
    const size_t SN = (size_t)g.S * n;
    const double *A64 = g.A64 + (size_t)sample * kSlots2D * n;
    const float *Ai = g.Ai + (size_t)sample * kSlots2D * n;
    double *v = g.v + so;
    double *wb0 = g.w + so;
    double *b = g.b + so;

    // ---- one-time setup: stencil rows (own rows and the row below) into
    //      shared memory, D^-1, zeroed u tile
    for (int t = tid; t < pl.csize; t += nt) {
        const int node = own0 - m + (t - 1);   // t = 0 is the pad
        float4 c = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (t > 0 && node >= 0 && node < own1) c = make_float4(Ai[node], Ai[n + node], Ai[2 * n + node], Ai[3 * n + node]);
        c0[t] = c;
    }
    for (int l = tid; l < nown; l += nt) dv[l] = Ai[4 * n + own0 + l];
    for (int t = tid; t < pl.usize; t += nt) ut[t] = 0.0f;
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
    PointState pst;
    const bool pth = rank == 0 && tid < g.pq.npts;   // point QoI threads
    if (pth) point_record(g.pq, sample, g.nsteps, g.dt, v, pst);

    float r[NPT], w[NPT], sv[NPT], p[NPT], x[NPT];
    int wpar = 0, par = 0;
    int64_t total_iters = 0;
    int32_t status = S_CONVERGED;
    const double dt = g.dt;
    const int last0 = nown - m;   // local index of the first node of the last own row

    for (int step = 0; step < g.nsteps; ++step) {
        // ---- block load: b = M (v + dt R), w update, r0 = b - A v
        const double *wcur = wb0 + wpar * SN;
        double *wnext = wb0 + (wpar ^ 1) * SN;
        {
            // (the FP32 residual is staged in the u tile, which is free here;
            //  the init below moves it into registers)
            double acc[2] = {0.0, 0.0};
#pragma unroll 1
            for (int l = tid; l < nown; l += nt) {
                const int node = own0 + l;
                const int j = node / m, i = node - j * m;
                const double bb = mass_apply_y<true>(m, i, j, g.h2, v, wcur, node, dt, g.a);
                b[node] = bb;
                const double vv = v[node], ww = wcur[node];
                wnext[node] = ww + dt * g.eps * recovery<true>(vv, ww, g.gam);
                const double rr = bb - stencil_apply_global(A64, n, m, node, i, j, v);
                const float rf = (float)rr;
                ut[UB + l] = rf;
                acc[0] += bb * bb;
                acc[1] += rr * rr;
                if (l < m) ex[exi(0, 0, 0) + l] = rf;
                if (l >= last0) ex[exi(0, 1, 0) + l - last0] = rf;
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
                // FP64 residual b - A v of the refined iterate, exported as r_0
                double racc[1] = {0.0};
#pragma unroll 1
                for (int l = tid; l < nown; l += nt) {
                    const int node = own0 + l;
                    const int j = node / m, i = node - j * m;
                    const double rr = b[node] - stencil_apply_global(A64, n, m, node, i, j, v);
                    const float rf = (float)rr;
                    ut[UB + l] = rf;
                    racc[0] += rr * rr;
                    if (l < m) ex[exi(0, 0, 0) + l] = rf;
                    if (l >= last0) ex[exi(0, 1, 0) + l - last0] = rf;
                }
                cluster_reduce<1, CS>(racc, wsl, csl, par, [&](double(&t)[1]) { ctl.s1 = t[0]; });
                par ^= 1;
                rnorm2 = ctl.s1;
                if (!isfinite(rnorm2)) { nonfinite = true; break; }
            }
            if (rnorm2 <= tol_out2) { solved = true; break; }
            // The inner problem is solved for r / ||r|| (and the correction
            // scaled back): FP32 squares of late-sweep residuals would
            // otherwise underflow.  The neighbours apply the same factor to
            // the r_0 rows they import.
            const double rnorm = sqrt(rnorm2);
            const float rscale = (float)(1.0 / rnorm);
            const double tol_in2 = g.rtol_in * g.rtol_in;

            // ---- init: u0 = D^-1 r0 (own + halo), w0 = A u0, x = 0
#pragma unroll
            for (int k = 0; k < NPT; ++k) {
                const int l = tid + k * nt;
                if (l < nown) {
                    r[k] = ut[UB + l] * rscale;
                    ut[UB + l] = r[k] * dv[l];
                }
            }
            if (has_lo)
                for (int i = tid; i < m; i += nt)
                    ut[1 + i] = (ex_lo[exi(0, 1, 0) + i] * rscale) * Ai[4 * n + own0 - m + i];
            if (has_hi)
                for (int i = tid; i < m; i += nt)
                    ut[Uhi + i] = (ex_hi[exi(0, 0, 0) + i] * rscale) * Ai[4 * n + own1 + i];
            __syncthreads();
            // thread 0's recurrence state: eta_i = (p_i, A p_i) = delta_i - beta_i^2 eta_{i-1}
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
            // w = A u for own local index l (u read from the tile)
            auto apply = [&](int l) {
                const int t = UB + l;
                const float4 a = c0[t];
                float wn = a.x * ut[t];
                wn = fmaf(a.y, ut[t + 1], wn);
                wn = fmaf(c0[t - 1].y, ut[t - 1], wn);
                wn = fmaf(a.z, ut[t + m], wn);
                wn = fmaf(c0[t - m].z, ut[t - m], wn);
                wn = fmaf(a.w, ut[t + m + 1], wn);
                wn = fmaf(c0[t - m - 1].w, ut[t - m - 1], wn);
                return wn;
            };
            {
                float iacc[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int k = 0; k < NPT; ++k) {
                    const int l = tid + k * nt;
                    x[k] = 0.0f;
                    p[k] = 0.0f;
                    sv[k] = 0.0f;
                    if (l < nown) {
                        const float u0 = ut[UB + l];
                        const float wn = apply(l);
                        w[k] = wn;
                        iacc[0] = fmaf(r[k], u0, iacc[0]);
                        iacc[1] = fmaf(wn, u0, iacc[1]);
                        iacc[2] = fmaf(r[k], r[k], iacc[2]);
                        if (l < m) ex[exi(0, 0, 1) + l] = wn;
                        if (l >= last0) ex[exi(0, 1, 1) + l - last0] = wn;
                    }
                }
                cluster_reduce<3, CS>(iacc, wsl, csl, par, [&](double(&t)[3]) { decide(t[0], t[1], t[2]); });
                par ^= 1;
            }
            while (true) {
                const int code = ctl.code;
                if (code != 0) {
                    if (code == 3) nonfinite = true;
                    else if (code == 2) status = status == S_CONVERGED ? S_MAXITER : status;
                    break;
                }
                const float ta = (float)ctl.alpha, tb = (float)ctl.beta;
                const int cur = it & 1, nxt = cur ^ 1;
                float pacc[3] = {0.0f, 0.0f, 0.0f};
                // own nodes: s_i, r_{i+1}, u_{i+1}, p_i, x_{i+1}
#pragma unroll
                for (int k = 0; k < NPT; ++k) {
                    const int l = tid + k * nt;
                    if (l < nown) {
                        const float di = dv[l];
                        const float si = it == 0 ? w[k] : fmaf(tb, sv[k], w[k]);
                        const float rn = fmaf(-ta, si, r[k]);
                        const float uk = rn * di;
                        ut[UB + l] = uk;
                        const float ui = r[k] * di;
                        p[k] = it == 0 ? ui : fmaf(tb, p[k], ui);
                        x[k] = fmaf(ta, p[k], x[k]);
                        sv[k] = si;
                        r[k] = rn;
                        pacc[0] = fmaf(rn, uk, pacc[0]);
                        pacc[2] = fmaf(rn, rn, pacc[2]);
                        if (l < m) {
                            ex[exi(nxt, 0, 0) + l] = rn;
                            ex[exi(nxt, 0, 2) + l] = si;
                        }
                        if (l >= last0) {
                            ex[exi(nxt, 1, 0) + l - last0] = rn;
                            ex[exi(nxt, 1, 2) + l - last0] = si;
                        }
                    }
                }
                // halo rows from the neighbours' exports of r_i, w_i, s_{i-1}
                if (has_lo) {
                    const float *er = ex_lo + exi(cur, 1, 0), *ew = ex_lo + exi(cur, 1, 1),
                                *es = ex_lo + exi(cur, 1, 2);
                    for (int i = tid; i < m; i += nt) {
                        // at it = 0 the exported r_0 rows are still unscaled
                        const float ri = it == 0 ? er[i] * rscale : er[i];
                        const float si = it == 0 ? ew[i] : fmaf(tb, es[i], ew[i]);
                        ut[1 + i] = fmaf(-ta, si, ri) * Ai[4 * n + own0 - m + i];
                    }
                }
                if (has_hi) {
                    const float *er = ex_hi + exi(cur, 0, 0), *ew = ex_hi + exi(cur, 0, 1),
                                *es = ex_hi + exi(cur, 0, 2);
                    for (int i = tid; i < m; i += nt) {
                        const float ri = it == 0 ? er[i] * rscale : er[i];
                        const float si = it == 0 ? ew[i] : fmaf(tb, es[i], ew[i]);
                        ut[Uhi + i] = fmaf(-ta, si, ri) * Ai[4 * n + own1 + i];
                    }
                }
                __syncthreads();
                // w_{i+1} = A u_{i+1}
#pragma unroll
                for (int k = 0; k < NPT; ++k) {
                    const int l = tid + k * nt;
                    if (l < nown) {
                        const float wn = apply(l);
                        w[k] = wn;
                        pacc[1] = fmaf(wn, ut[UB + l], pacc[1]);
                        if (l < m) ex[exi(nxt, 0, 1) + l] = wn;
                        if (l >= last0) ex[exi(nxt, 1, 1) + l - last0] = wn;
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
        if (pth) point_record(g.pq, sample, g.nsteps, dt, v, pst);
    }
    if (pth) point_finish(g.pq, sample, g.nsteps, pst);

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
