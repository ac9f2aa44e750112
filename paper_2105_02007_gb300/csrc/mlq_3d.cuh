// mlq_3d.cuh -- P1 on Kuhn tetrahedra of a structured box (the 3D slab of
// the configurations), Sec. 3.1: set-up of the 15-point stencils and the
// batched time-block solver.
//
// Mesh convention (the same as the library's documented mesh, include/mlq.h):
//   nodes   (i, j, k), node = i + mx (j + my k), x = Lx i / (mx - 1), ...
//   cells   c = i + (mx - 1)(j + (my - 1) k), six tetrahedra e = 6 c + s;
//           tetrahedron s walks from corner (i, j, k) to (i+1, j+1, k+1) along
//           the unit steps perm[s][0], perm[s][1], perm[s][2] (Kuhn / Freudenthal
//           splitting, nested under regular refinement)
//   barycentric coordinates on tetrahedron s, xi = local coordinates in [0,1]^3
//   along the steps: lambda_0 = 1 - xi_a, lambda_1 = xi_a - xi_b,
//   lambda_2 = xi_b - xi_c, lambda_3 = xi_c (a, b, c = the step axes in order).
// Every edge of a tetrahedron joins its vertices q < q' along a direction with
// components in {0, 1}: the stencil of a node P is its diagonal plus the
// couplings to P + d for the seven such directions d (slot = dx + 2 dy + 4 dz);
// the coupling to P - d is slot d of node P - d (the matrices are symmetric).
//
// Solver (one sample per cluster of CS CTAs, everything in global memory and
// L2; the 3D levels outgrow the shared memory of a cluster):
//   per time block  y = v + dt R(v, w); b = M y; w <- w + dt eps (v - gam w);
//                   r = b - A v in FP64 from the guess v extrapolated
//                   from the last block solutions (guess_order)
//   inner solve     Jacobi-preconditioned CG (Chronopoulos-Gear: one cluster
//                   reduction per iteration) on A d = r / ||r|| from d = 0 in
//                   the inner precision TI, v += ||r|| d; the mixed path
//                   repeats while ||b - A v|| > rtol ||b|| (iterative
//                   refinement in FP64), the FP64 path runs one sweep to that
//                   tolerance
//   QoI             Q = sum_P m_P v_P with the lumped mass m = M 1.
// CTA `rank` owns the grid lines j0 <= j < j1 of every plane k (on every
// level); another CTA's values are read through L2 (ld.cg) after a cluster
// barrier.
#pragma once

#include "mlq_3d_types.cuh"
#include "mlq_kernels.cuh"

namespace mlq {

constexpr int kMgCoarsestSweeps3D = 6;  // damped Jacobi sweeps on the coarsest 3D level

// ---------------------------------------------------------------------------
// Level set-up (sample independent): FP64 mass stencil [8][n] and lumped mass
// m_P = (incident tetrahedra) |e| / 4.  Gathers over the (up to) 24
// tetrahedra at the node in a fixed order.
// ---------------------------------------------------------------------------
__global__ void level3d_setup_kernel(Grid3 g, double *__restrict__ M3, double *__restrict__ lump)
{
    const int64_t P = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= g.n) return;
    const int i = (int)(P % g.mx), j = (int)((P / g.mx) % g.my), k = (int)(P / ((int64_t)g.mx * g.my));
    const double vol = g.hx * g.hy * g.hz / 6.0;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int cnt = 0;
    for (int d = 0; d < 8; ++d) {   // cell with P at corner d
        const int ci = i - (d & 1), cj = j - ((d >> 1) & 1), ck = k - ((d >> 2) & 1);
        if (ci < 0 || cj < 0 || ck < 0 || ci >= g.mx - 1 || cj >= g.my - 1 || ck >= g.mz - 1) continue;
        for (int s = 0; s < 6; ++s) {
            int q = -1;
            for (int t = 0; t < 4; ++t)
                if (kuhn_vertex(s, t) == d) q = t;
            if (q < 0) continue;
            ++cnt;
            acc[0] += vol / 10.0;
            for (int t = q + 1; t < 4; ++t) acc[kuhn_vertex(s, t) ^ d] += vol / 20.0;
        }
    }
    for (int sl = 0; sl < 8; ++sl) M3[(int64_t)sl * g.n + P] = acc[sl];
    lump[P] = cnt * vol / 4.0;
}

// Gather of the stencil of M + dt K(D) at node P over the (up to) 24
// tetrahedra at P, in a fixed order; getD(e, d11, d12, d22) gives the
// in-plane block of D on tetrahedron e (d33 = s_t).
template <typename GetD>
__device__ __forceinline__ void stencil3d_gather(const Grid3 &g, int64_t P, double dt, double s_t, GetD getD,
                                                 double (&acc)[8])
{
    const int i = (int)(P % g.mx), j = (int)((P / g.mx) % g.my), k = (int)(P / ((int64_t)g.mx * g.my));
    const double vol = g.hx * g.hy * g.hz / 6.0;
    for (int sl = 0; sl < 8; ++sl) acc[sl] = 0.0;
    for (int d = 0; d < 8; ++d) {
        const int ci = i - (d & 1), cj = j - ((d >> 1) & 1), ck = k - ((d >> 2) & 1);
        if (ci < 0 || cj < 0 || ck < 0 || ci >= g.mx - 1 || cj >= g.my - 1 || ck >= g.mz - 1) continue;
        const int64_t cell = ci + (int64_t)(g.mx - 1) * (cj + (int64_t)(g.my - 1) * ck);
        for (int s = 0; s < 6; ++s) {
            int q = -1;
            for (int t = 0; t < 4; ++t)
                if (kuhn_vertex(s, t) == d) q = t;
            if (q < 0) continue;
            double d11, d12, d22;
            getD(6 * cell + s, d11, d12, d22);
            const double d33 = s_t;
            double G[4][3];
            kuhn_grads(g, s, G);
            const double Dq[3] = {d11 * G[q][0] + d12 * G[q][1], d12 * G[q][0] + d22 * G[q][1], d33 * G[q][2]};
            for (int t = q; t < 4; ++t) {
                const double kq = vol * (Dq[0] * G[t][0] + Dq[1] * G[t][1] + Dq[2] * G[t][2]);
                const double mq = vol / 20.0 * (t == q ? 2.0 : 1.0);
                acc[kuhn_vertex(s, t) ^ d] += mq + dt * kq;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// K2 (3D): per sample the stencil of A = M + dt K(theta): A64 [S][9][n] FP64
// (slot 8 = 1 / diagonal) and, when Ai is not null, the same in FP32.
// D = s_t I + (s_l - s_t) f f^T with f f^T = (1/2)[[1 + c, sn, 0], [sn, 1 - c, 0], [0, 0, 0]]
// from (c, sn) = (cos 2t, sin 2t) per tetrahedron.
// ---------------------------------------------------------------------------
__global__ void stencil3d_setup_kernel(const double *__restrict__ cs2, Grid3 g, double dt, double s_l, double s_t,
                                       int S, double *__restrict__ A64, float *__restrict__ A32)
{
    const int64_t P = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int smp = blockIdx.y;
    if (P >= g.n || smp >= S) return;
    const int64_t ne = 6LL * (g.mx - 1) * (g.my - 1) * (g.mz - 1);
    const double *c2 = cs2 + (size_t)smp * ne * 2;
    const double hds = 0.5 * (s_l - s_t);
    double acc[8];
    stencil3d_gather(g, P, dt, s_t, [&](int64_t e, double &d11, double &d12, double &d22) {
        const double c = c2[e * 2], sn = c2[e * 2 + 1];
        d11 = s_t + hds * (1.0 + c);
        d22 = s_t + hds * (1.0 - c);
        d12 = hds * sn;
    }, acc);
    double *a = A64 + (size_t)smp * kSlots3D * g.n;
    for (int sl = 0; sl < 8; ++sl) a[(int64_t)sl * g.n + P] = acc[sl];
    a[8LL * g.n + P] = 1.0 / acc[0];
    if (A32) {
        float *f = A32 + (size_t)smp * kSlots3D * g.n;
        for (int sl = 0; sl < 8; ++sl) f[(int64_t)sl * g.n + P] = (float)acc[sl];
        f[8LL * g.n + P] = (float)(1.0 / acc[0]);
    }
}

// ---------------------------------------------------------------------------
// Multigrid set-up, per sample and coarse level c: the mean in-plane D over
// the eight children of every coarse tetrahedron (the fine tetrahedra of its
// 2 x 2 x 2 fine cells whose centroid lies in it: the centroid's coarse-local
// coordinates follow the coarse tetrahedron's step order), read from
// (cos 2t, sin 2t) on the fine mesh (c = 1) or from the previous level's means.
// ---------------------------------------------------------------------------
__global__ void coarsen3d_kernel(const double *__restrict__ cs2, const float *__restrict__ dfine, Grid3 gf,
                                 Grid3 gc, int S, double s_l, double s_t, float *__restrict__ dc)
{
    const int64_t E = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int smp = blockIdx.y;
    const int64_t nec = 6LL * (gc.mx - 1) * (gc.my - 1) * (gc.mz - 1);
    const int64_t nef = 6LL * (gf.mx - 1) * (gf.my - 1) * (gf.mz - 1);
    if (E >= nec || smp >= S) return;
    const int64_t C = E / 6;
    const int Sx = (int)(E % 6);
    const int I = (int)(C % (gc.mx - 1)), J = (int)((C / (gc.mx - 1)) % (gc.my - 1)),
              K = (int)(C / ((int64_t)(gc.mx - 1) * (gc.my - 1)));
    const int a0 = kuhn_axis(Sx, 0), a1 = kuhn_axis(Sx, 1), a2 = kuhn_axis(Sx, 2);
    const double hds = 0.5 * (s_l - s_t);
    double d11 = 0.0, d12 = 0.0, d22 = 0.0;
    for (int o = 0; o < 8; ++o) {
        const int ox = o & 1, oy = (o >> 1) & 1, oz = (o >> 2) & 1;
        const int64_t cf = (2 * I + ox) + (int64_t)(gf.mx - 1) * ((2 * J + oy) + (int64_t)(gf.my - 1) * (2 * K + oz));
        for (int s = 0; s < 6; ++s) {
            double cen[3] = {(double)ox, (double)oy, (double)oz};
            for (int q = 0; q < 3; ++q) cen[kuhn_axis(s, q)] += (3.0 - q) / 4.0;
            if (!(cen[a0] > cen[a1] && cen[a1] > cen[a2])) continue;
            const int64_t e = 6 * cf + s;
            if (cs2) {
                const double c = cs2[((size_t)smp * nef + e) * 2], sn = cs2[((size_t)smp * nef + e) * 2 + 1];
                d11 += s_t + hds * (1.0 + c);
                d22 += s_t + hds * (1.0 - c);
                d12 += hds * sn;
            } else {
                const float *q = dfine + ((size_t)smp * nef + e) * 3;
                d11 += q[0];
                d12 += q[1];
                d22 += q[2];
            }
        }
    }
    float *out = dc + ((size_t)smp * nec + E) * 3;
    out[0] = (float)(d11 / 8.0);
    out[1] = (float)(d12 / 8.0);
    out[2] = (float)(d22 / 8.0);
}

// coarse-level stencil (FP32, 9 slots with 1 / diagonal) from the mean D
__global__ void stencil3d_from_d_kernel(const float *__restrict__ dbar, Grid3 g, double dt, double s_t, int S,
                                        float *__restrict__ A32)
{
    const int64_t P = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int smp = blockIdx.y;
    if (P >= g.n || smp >= S) return;
    const int64_t ne = 6LL * (g.mx - 1) * (g.my - 1) * (g.mz - 1);
    const float *d = dbar + (size_t)smp * ne * 3;
    double acc[8];
    stencil3d_gather(g, P, dt, s_t, [&](int64_t e, double &d11, double &d12, double &d22) {
        d11 = d[e * 3];
        d12 = d[e * 3 + 1];
        d22 = d[e * 3 + 2];
    }, acc);
    float *f = A32 + (size_t)smp * kSlots3D * g.n;
    for (int sl = 0; sl < 8; ++sl) f[(int64_t)sl * g.n + P] = (float)acc[sl];
    f[8LL * g.n + P] = (float)(1.0 / acc[0]);
}

// (C x)_P for a symmetric 15-point stencil C [8][n]: slot d at P couples to
// P + d, slot d at P - d couples to P - d.  x read through L2.
// One path for every node, so boundary nodes do not split their warp: a
// coupling that does not exist (P on the boundary, P +- d wrapping to
// another line or plane) has a zero slot, set up so by the gather over the
// incident tetrahedra, and adds exactly nothing; a neighbour index outside
// the array (first and last planes) is replaced by P and its slot by 0.
// Every load is issued before the first product so that they are in
// flight together.
template <typename T, typename TX>
__device__ __forceinline__ T apply15(const T *__restrict__ C, const Grid3 &g, const TX *x, int P, int, int, int)
{
    const int n = g.n;
    T c[15], xv[15];
    c[0] = C[P];
    xv[0] = (T)__ldcg(x + P);
#pragma unroll
    for (int sl = 1; sl < 8; ++sl) {
        const int off = dir_offset32(g, sl);
        const bool up = P + off < n, dn = P >= off;
        const T cu = C[sl * n + P], cd = C[sl * n + (dn ? P - off : P)];
        c[2 * sl - 1] = up ? cu : (T)0;
        c[2 * sl] = dn ? cd : (T)0;
        xv[2 * sl - 1] = (T)__ldcg(x + (up ? P + off : P));
        xv[2 * sl] = (T)__ldcg(x + (dn ? P - off : P));
    }
    T acc = c[0] * xv[0];
#pragma unroll
    for (int q = 1; q < 15; ++q) acc += c[q] * xv[q];
    return acc;
}

// The nodes a CTA owns on one level: grid lines j0 <= j < j0 + nj of every
// plane k.  They are visited line by line, j fastest inside the band and
// then k, so that the nodes a 15-point product reads in the planes k +- 1
// were visited one band of lines earlier (nj x mx nodes) rather than one
// whole plane earlier: the reuse stays inside L2 when every SM streams.
struct Band3 {
    int mx, my, j0, nj;
    int cnt;
};

__device__ __forceinline__ Band3 band3(const Grid3 &g, int rank, int cs)
{
    Band3 b;
    b.mx = g.mx;
    b.my = g.my;
    b.j0 = (int)(g.my * rank / cs);
    b.nj = (int)(g.my * (rank + 1) / cs) - b.j0;
    b.cnt = b.nj * g.mx * g.mz;
    return b;
}

// a thread's position (i, j0 + jl, k) in its band, advanced by a fixed
// stride of band-local indices without a division per node (nj > 0)
struct Walk3 {
    int i, jl, k, di, dj, dk;
    __device__ void init(const Band3 &b, int f, int stride)
    {
        i = (int)(f % b.mx);
        const int line = f / b.mx;
        jl = (int)(line % b.nj);
        k = (int)(line / b.nj);
        di = (int)(stride % b.mx);
        const int lines = stride / b.mx;
        dj = (int)(lines % b.nj);
        dk = (int)(lines / b.nj);
    }
    __device__ void next(const Band3 &b)
    {
        i += di;
        jl += dj;
        k += dk;
        if (i >= b.mx) {
            i -= b.mx;
            ++jl;
        }
        if (jl >= b.nj) {
            jl -= b.nj;
            ++k;
        }
    }
    __device__ int j(const Band3 &b) const { return b.j0 + jl; }
    __device__ int node(const Band3 &b) const { return i + b.mx * (b.j0 + jl + b.my * k); }
};

template <typename T, int N>
struct Vals {
    T v[N];
};

// L2 prefetch (one bulk request, TMA unit) of the 16-byte aligned part of
// elements [lo, hi) of an array
template <typename T>
__device__ __forceinline__ void prefetch_l2(const T *a, int lo, int hi)
{
    const uintptr_t s = ((uintptr_t)(a + lo) + 15) & ~(uintptr_t)15;
    const uintptr_t e = (uintptr_t)(a + hi) & ~(uintptr_t)15;
    if (e > s) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(s), "r"((uint32_t)(e - s)) : "memory");
}

struct NoPrefetch {
    __device__ void operator()(int, int) const {}
};

// For every node of the band: r = ld(P, i, j, k), then st(P, r).  U nodes
// per thread and round, the loads of all U issued before the first store,
// so that a pass with few loads per node still keeps U times the bytes in
// flight (HBM latency, not bandwidth, bounds a pass with one node per round).
// pf(lo, hi) prefetches the node range [lo, hi) of the pass's streamed
// arrays into L2: thread 0 hands it the band of the plane after the one it
// is in (one contiguous range of nj x mx nodes per plane), so the CTA's
// loads find their lines in L2.
template <int U, typename Ld, typename St, typename Pf = NoPrefetch>
__device__ __forceinline__ void sweep3(const Band3 &b, int tid, int nt, Ld &&ld, St &&st, Pf &&pf = Pf{})
{
    if (b.cnt <= 0) return;
    using R = decltype(ld(0, 0, 0, 0));
    const int plane = b.mx * b.my, band = b.mx * b.nj, base = b.mx * b.j0;
    const int planes = (int)(b.cnt / band);
    int ahead = 0;   // planes handed to pf so far (thread 0)
    Walk3 wk;
    wk.init(b, tid, nt);
    for (int f = tid; f < b.cnt; f += U * nt) {
        if (tid == 0)
            for (; ahead < planes && ahead <= wk.k + 1; ++ahead) pf(base + plane * ahead, base + plane * ahead + band);
        R r[U];
        int P[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            P[u] = wk.node(b);
            if (f + u * nt < b.cnt) r[u] = ld(P[u], wk.i, wk.j(b), wk.k);
            wk.next(b);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (f + u * nt < b.cnt) st(P[u], r[u]);
    }
}

// nodes per thread and round: streaming passes with a few loads per node,
// and passes with a 15-point product (thirty loads of their own)
constexpr int kU3 = 4, kU15 = 1;

template <typename TI, int CS>
__global__ void __launch_bounds__(512, 2) slab_solve_3d_kernel(Solve3Args<TI> g)
{
    __shared__ double wsl[32][4];
    __shared__ double csl[2][4];
    __shared__ Ctl ctl;
    // the multigrid level table, indexed by the level at run time: a copy in
    // shared memory keeps those reads out of local memory
    __shared__ Mg3Args sM;
    if (threadIdx.x == 0) sM = g.mg;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int sample = blockIdx.x / CS;
    const Grid3 G = g.g;
    const int n = G.n;
    const Band3 B0 = band3(G, rank, CS);
    const int tid = threadIdx.x, nt = blockDim.x;
    constexpr bool mixed = sizeof(TI) == 4;

    const size_t so = (size_t)sample * n;
    const size_t SN = (size_t)g.S * n;
    const double *A64 = g.A64 + (size_t)sample * kSlots3D * n;
    const TI *Ai = g.Ai + (size_t)sample * kSlots3D * n;
    const TI *__restrict__ Dinv = Ai + 8 * n;
    // v: [kVRing][S][n], the solutions of the last blocks and the guess of the next
    double *vb0 = g.v + so, *wb0 = g.w + so, *b = g.b + so, *yb = g.y + so;
    TI *__restrict__ R = g.r + so;
    TI *__restrict__ U = g.u + so;
    TI *__restrict__ W = g.wv + so;
    TI *__restrict__ Sv = g.s + so;
    TI *__restrict__ Pv = g.p + so;
    TI *__restrict__ X = g.x + so;
    // L2 prefetch sets of the streaming passes: the eight stencil slots of a
    // level, and single vectors
    auto pf_slots = [](const auto *A, int nn, int lo, int hi) {
#pragma unroll 1
        for (int sl = 0; sl < 8; ++sl) prefetch_l2(A + sl * nn, lo, hi);
    };

    sweep3<1>(
        B0, tid, nt,
        [&](int P, int i, int j, int k) {
            Vals<double, 2> s0;
            if (g.v0) {
                s0.v[0] = g.v0[P];
                s0.v[1] = g.w0 ? g.w0[P] : 0.0;
            } else {
                const double xx = g.Lx * i / (G.mx - 1), yy = g.Ly * j / (G.my - 1), zz = g.Lz * k / (G.mz - 1);
                s0.v[0] = (xx * xx + yy * yy + zz * zz <= g.radius2) ? 1.0 : 0.0;
                s0.v[1] = 0.0;
            }
            return s0;
        },
        [&](int P, const Vals<double, 2> &s0) {
            vb0[P] = s0.v[0];
            wb0[P] = s0.v[1];
        });
    cl.sync();
    PointState pst;
    const bool pth = rank == 0 && tid < g.pq.npts;   // point QoI threads
    if (pth) point_record(g.pq, sample, g.nsteps, g.dt, vb0, pst);

    int wpar = 0, par = 0;
    int64_t total_iters = 0;
    int32_t status = S_CONVERGED;
    const double dt = g.dt;

    // ---- multigrid preconditioner u = MG(r) (FP32 inner path, nl > 1):
    // V(1,1) with damped Jacobi, P^T restriction (the fine node 2I plus half
    // of the fourteen edge midpoints 2I +- d), P1 interpolation (a fine node
    // takes the mean of the coarse ends of the coarse edge it halves),
    // Jacobi sweeps on the coarsest level.  Every level is split over the
    // cluster by grid lines; values of other CTAs are read through L2 after a
    // cluster barrier.  Input: R (level 0 right-hand side) and its
    // pre-smoothed XA_0 = omega D^-1 R, written by the pass that formed R;
    // result in U.  Returns (r, u) and (r, r) (the thread's partial sums),
    // formed in the level-0 post-smoothing.
    constexpr bool kMg = sizeof(TI) == 4;
    const bool mgp = kMg && g.mg.nl > 1;
    float *const xa0 = mgp ? g.mg.xa[0] + so : nullptr;
    const TI om0 = (TI)g.mg.omega;
    auto vcycle = [&]() {
        Vals<double, 2> sums;
        sums.v[0] = 0.0;
        sums.v[1] = 0.0;
        if constexpr (kMg) {
            const Mg3Args &M = sM;
            const int NL = M.nl;
            const float om = M.omega;
            auto Aof = [&](int c) -> const float * {
                return c == 0 ? (const float *)Ai : M.A[c] + (size_t)sample * kSlots3D * M.g[c].n;
            };
            auto vec = [&](float *const *base, int c) { return base[c] + (size_t)sample * M.g[c].n; };
            auto BB = [&](int c) -> float * { return c == 0 ? (float *)R : vec(M.bb, c); };
            auto RR = [&](int c) -> float * { return c == 0 ? (float *)U : vec(M.rr, c); };
            for (int c = 0; c < NL - 1; ++c) {
                const Grid3 &Gc = M.g[c];
                const Band3 Bc = band3(Gc, rank, CS);
                const float *A = Aof(c), *Dv = A + 8 * (size_t)Gc.n;
                float *xa = vec(M.xa, c), *rr = RR(c), *bb = BB(c);
                // pre-smoothing from zero: XA = omega D^-1 B (level 0: done)
                if (c > 0) {
                    sweep3<kU3>(
                        Bc, tid, nt, [&](int P, int, int, int) { return om * Dv[P] * __ldcg(bb + P); },
                        [&](int P, float x) { xa[P] = x; },
                        [&](int lo, int hi) {
                            prefetch_l2(Dv, lo, hi);
                            prefetch_l2(bb, lo, hi);
                        });
                    cl.sync();
                }
                // residual RR = B - A XA
                sweep3<kU15>(
                    Bc, tid, nt,
                    [&](int P, int i, int j, int k) {
                        return __ldcg(bb + P) - apply15<float, float>(A, Gc, xa, P, i, j, k);
                    },
                    [&](int P, float r) { rr[P] = r; },
                    [&](int lo, int hi) {
                        pf_slots(A, Gc.n, lo, hi);
                        prefetch_l2(xa, lo, hi);
                        prefetch_l2(bb, lo, hi);
                    });
                cl.sync();
                // restriction into level c+1
                const Grid3 &Gq = M.g[c + 1];
                float *bq = BB(c + 1);
                sweep3<kU15>(
                    band3(Gq, rank, CS), tid, nt,
                    [&](int, int ci, int cj, int ck) {
                        const int fi = 2 * ci, fj = 2 * cj, fk = 2 * ck;
                        const int f = fi + Gc.mx * (fj + Gc.my * fk);
                        // branch-free: a missing neighbour loads the centre
                        // and enters with weight 0 (h + 0 v = h exactly), so
                        // boundary nodes do not split their warp
                        float v[15], wgt[15];
                        v[0] = __ldcg(rr + f);
#pragma unroll
                        for (int sl = 1; sl < 8; ++sl) {
                            const int dx = sl & 1, dy = (sl >> 1) & 1, dz = (sl >> 2) & 1;
                            const int off = dir_offset32(Gc, sl);
                            const bool up = fi + dx < Gc.mx && fj + dy < Gc.my && fk + dz < Gc.mz;
                            const bool dn = fi >= dx && fj >= dy && fk >= dz;
                            v[2 * sl - 1] = __ldcg(rr + (up ? f + off : f));
                            v[2 * sl] = __ldcg(rr + (dn ? f - off : f));
                            wgt[2 * sl - 1] = up ? 1.0f : 0.0f;
                            wgt[2 * sl] = dn ? 1.0f : 0.0f;
                        }
                        float h = 0.0f;
#pragma unroll
                        for (int q = 1; q < 15; ++q) h += wgt[q] * v[q];
                        return v[0] + 0.5f * h;
                    },
                    [&](int Q, float v) { bq[Q] = v; });
                cl.sync();
            }
            // coarsest: damped Jacobi sweeps, ping-pong XA / XB
            {
                const int c = NL - 1;
                const Grid3 &Gc = M.g[c];
                const Band3 Bc = band3(Gc, rank, CS);
                const float *A = Aof(c), *Dv = A + 8 * (size_t)Gc.n;
                float *X0 = vec(M.xa, c), *Y0 = vec(M.xb, c), *bb = BB(c);
                sweep3<kU3>(
                    Bc, tid, nt, [&](int P, int, int, int) { return om * Dv[P] * __ldcg(bb + P); },
                    [&](int P, float x) { X0[P] = x; });
                for (int k = 1; k < kMgCoarsestSweeps3D; ++k) {
                    cl.sync();
                    sweep3<kU15>(
                        Bc, tid, nt,
                        [&](int P, int i, int j, int kk) {
                            return __ldcg(X0 + P) +
                                   om * Dv[P] * (__ldcg(bb + P) - apply15<float, float>(A, Gc, X0, P, i, j, kk));
                        },
                        [&](int P, float x) { Y0[P] = x; });
                    float *t = X0;
                    X0 = Y0;
                    Y0 = t;
                }
                cl.sync();
            }
            // ascend
            for (int c = NL - 2; c >= 0; --c) {
                const Grid3 &Gc = M.g[c], &Gq = M.g[c + 1];
                const Band3 Bc = band3(Gc, rank, CS);
                const float *A = Aof(c), *Dv = A + 8 * (size_t)Gc.n;
                const float *xq = (c + 1 == NL - 1) ? ((kMgCoarsestSweeps3D - 1) % 2 ? vec(M.xb, c + 1) : vec(M.xa, c + 1))
                                                    : RR(c + 1);
                float *xa = vec(M.xa, c), *xb = vec(M.xb, c), *rr = RR(c), *bb = BB(c);
                // XB = XA + P X_{c+1}
                sweep3<kU3>(
                    Bc, tid, nt,
                    [&](int P, int i, int j, int k) {
                        const int ci = i >> 1, cj = j >> 1, ck = k >> 1;
                        const int qa = ci + Gq.mx * (cj + Gq.my * ck);
                        const int qb = qa + (i & 1) + Gq.mx * ((j & 1) + Gq.my * (k & 1));
                        return __ldcg(xa + P) + 0.5f * (__ldcg(xq + qa) + __ldcg(xq + qb));
                    },
                    [&](int P, float x) { xb[P] = x; }, [&](int lo, int hi) { prefetch_l2(xa, lo, hi); });
                cl.sync();
                // post-smoothing X_c = XB + omega D^-1 (B - A XB), into RR
                auto pf_post = [&](int lo, int hi) {
                    pf_slots(A, Gc.n, lo, hi);
                    prefetch_l2(Dv, lo, hi);
                    prefetch_l2(xb, lo, hi);
                    prefetch_l2(bb, lo, hi);
                };
                if (c > 0) {
                    sweep3<kU15>(
                        Bc, tid, nt,
                        [&](int P, int i, int j, int k) {
                            return __ldcg(xb + P) +
                                   om * Dv[P] * (__ldcg(bb + P) - apply15<float, float>(A, Gc, xb, P, i, j, k));
                        },
                        [&](int P, float x) { rr[P] = x; }, pf_post);
                } else {
                    sweep3<kU15>(
                        Bc, tid, nt,
                        [&](int P, int i, int j, int k) {
                            Vals<float, 2> o;
                            o.v[1] = __ldcg(bb + P);
                            o.v[0] = __ldcg(xb + P) + om * Dv[P] * (o.v[1] - apply15<float, float>(A, Gc, xb, P, i, j, k));
                            return o;
                        },
                        [&](int P, const Vals<float, 2> &o) {
                            rr[P] = o.v[0];
                            sums.v[0] += (double)(o.v[1] * o.v[0]);
                            sums.v[1] += (double)(o.v[1] * o.v[1]);
                        },
                        pf_post);
                }
                cl.sync();
            }
        }
        return sums;
    };

    auto vring = [&](int j) { return vb0 + (size_t)(((j % kVRing) + kVRing) % kVRing) * SN; };
    for (int step = 0; step < g.nsteps; ++step) {
        // the block starts from the extrapolation of order guess_order(step)
        // over v_n, v_{n-1}, ..., kept in the buffer of v_{n+1} (which held
        // v_{n-4})
        const double *vcur = vring(step);
        const double *vm1 = vring(step - 1), *vm2 = vring(step - 2), *vm3 = vring(step - 3);
        double *v = vring(step + 1);
        const int gp = guess_order(step);
        const double *wcur = wb0 + wpar * SN;
        double *wnext = wb0 + (wpar ^ 1) * SN;
        sweep3<2>(
            B0, tid, nt,
            [&](int P, int, int, int) {
                const double vv = vcur[P], ww = wcur[P];
                Vals<double, 3> o;
                // FP64 in both paths: the extrapolated guess amplifies the
                // rounding noise of an FP32 reaction (see reaction())
                o.v[0] = vv + dt * reaction<false>(vv, ww, g.a);
                o.v[1] = ww + dt * g.eps * recovery<false>(vv, ww, g.gam);
                o.v[2] = extrapolate(gp, vv, gp >= 1 ? vm1[P] : 0.0, gp >= 2 ? vm2[P] : 0.0, gp >= 3 ? vm3[P] : 0.0,
                                     gp >= 4 ? v[P] : 0.0);
                return o;
            },
            [&](int P, const Vals<double, 3> &o) {
                yb[P] = o.v[0];
                wnext[P] = o.v[1];
                v[P] = o.v[2];
            });
        wpar ^= 1;
        cl.sync();
        {
            double acc[2] = {0.0, 0.0};
            sweep3<1>(
                B0, tid, nt,
                [&](int P, int i, int j, int k) {
                    Vals<double, 2> o;
                    o.v[0] = apply15<double, double>(g.M3, G, yb, P, i, j, k);
                    o.v[1] = o.v[0] - apply15<double, double>(A64, G, v, P, i, j, k);
                    return o;
                },
                [&](int P, const Vals<double, 2> &o) {
                    b[P] = o.v[0];
                    R[P] = (TI)o.v[1];
                    acc[0] += o.v[0] * o.v[0];
                    acc[1] += o.v[1] * o.v[1];
                });
            cluster_reduce<2, CS>(acc, wsl, csl, par, [&](double(&t)[2]) {
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
                sweep3<1>(
                    B0, tid, nt,
                    [&](int P, int i, int j, int k) {
                        return b[P] - apply15<double, double>(A64, G, v, P, i, j, k);
                    },
                    [&](int P, double rr) {
                        R[P] = (TI)rr;
                        racc[0] += rr * rr;
                    });
                cluster_reduce<1, CS>(racc, wsl, csl, par, [&](double(&t)[1]) { ctl.s1 = t[0]; });
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
            // of what the outer test still needs when that is looser (the
            // FP64 check after the sweep decides); the FP64 path solves to the
            // outer target in this one sweep
            const double need = tol_out2 / rnorm2;
            const double tol_in2 = mixed ? fmax(g.rtol_in * g.rtol_in, 0.25 * need) : need;

            // init: r0 normalised, x = p = s = 0; u0 = D^-1 r0 (Jacobi) or the
            // multigrid's pre-smoothed XA_0 = omega D^-1 r0
            sweep3<kU3>(
                B0, tid, nt,
                [&](int P, int, int, int) {
                    Vals<TI, 2> o;
                    o.v[0] = R[P] * rscale;
                    o.v[1] = mgp ? om0 * Dinv[P] * o.v[0] : Dinv[P] * o.v[0];
                    return o;
                },
                [&](int P, const Vals<TI, 2> &o) {
                    R[P] = o.v[0];
                    if (mgp) xa0[P] = (float)o.v[1];
                    else U[P] = o.v[1];
                    X[P] = (TI)0;
                    Pv[P] = (TI)0;
                    Sv[P] = (TI)0;
                });
            cl.sync();
            // (r, u) and (r, r) of the current iterate
            double gacc = 0.0, racc = 0.0;
            if (mgp) {
                const Vals<double, 2> t = vcycle();
                gacc = t.v[0];
                racc = t.v[1];
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
            if (!mgp) {
                sweep3<kU3>(
                    B0, tid, nt,
                    [&](int P, int, int, int) {
                        Vals<TI, 2> o;
                        o.v[0] = R[P];
                        o.v[1] = __ldcg(U + P);
                        return o;
                    },
                    [&](int, const Vals<TI, 2> &o) {
                        gacc += (double)(o.v[0] * o.v[1]);
                        racc += (double)(o.v[0] * o.v[0]);
                    },
                    [&](int lo, int hi) {
                        prefetch_l2(R, lo, hi);
                        prefetch_l2(U, lo, hi);
                    });
            }
            while (true) {
                // w = A u, (w, u); one reduction of (r, u), (w, u), (r, r)
                double pacc[3] = {gacc, 0.0, racc};
                sweep3<kU15>(
                    B0, tid, nt,
                    [&](int P, int i, int j, int k) {
                        Vals<TI, 2> o;
                        o.v[0] = apply15<TI, TI>(Ai, G, U, P, i, j, k);
                        o.v[1] = __ldcg(U + P);
                        return o;
                    },
                    [&](int P, const Vals<TI, 2> &o) {
                        W[P] = o.v[0];
                        pacc[1] += (double)(o.v[0] * o.v[1]);
                    },
                    [&](int lo, int hi) {
                        pf_slots(Ai, n, lo, hi);
                        prefetch_l2(U, lo, hi);
                    });
                cluster_reduce<3, CS>(pacc, wsl, csl, par, [&](double(&t)[3]) { decide(t[0], t[1], t[2]); });
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
                sweep3<2>(
                    B0, tid, nt,
                    [&](int P, int, int, int) {
                        const TI ww = W[P], uu = __ldcg(U + P);
                        Vals<TI, 5> o;
                        o.v[0] = it == 0 ? ww : ww + tb * Sv[P];
                        o.v[1] = it == 0 ? uu : uu + tb * Pv[P];
                        o.v[2] = X[P] + ta * o.v[1];
                        o.v[3] = R[P] - ta * o.v[0];
                        o.v[4] = mgp ? om0 * Dinv[P] * o.v[3] : Dinv[P] * o.v[3];
                        return o;
                    },
                    [&](int P, const Vals<TI, 5> &o) {
                        Sv[P] = o.v[0];
                        Pv[P] = o.v[1];
                        X[P] = o.v[2];
                        R[P] = o.v[3];
                        racc += (double)(o.v[3] * o.v[3]);
                        if (mgp) {
                            xa0[P] = (float)o.v[4];
                        } else {
                            U[P] = o.v[4];
                            gacc += (double)(o.v[3] * o.v[4]);
                        }
                    },
                    [&](int lo, int hi) {
                        prefetch_l2(W, lo, hi);
                        prefetch_l2(U, lo, hi);
                        prefetch_l2(Sv, lo, hi);
                        prefetch_l2(Pv, lo, hi);
                        prefetch_l2(X, lo, hi);
                        prefetch_l2(R, lo, hi);
                        prefetch_l2(Dinv, lo, hi);
                    });
                ++it;
                cl.sync();
                if (mgp) gacc = vcycle().v[0];
            }
            total_iters += it;
            if (nonfinite) break;
            sweep3<2>(
                B0, tid, nt, [&](int P, int, int, int) { return fma((double)X[P], rnorm, v[P]); },
                [&](int P, double t) { v[P] = t; });
            cl.sync();
            if (!mixed) solved = true;
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
    const double *vfin = vring(g.nsteps);   // solution of the last block
    sweep3<1>(
        B0, tid, nt, [&](int P, int, int, int) { return g.lump[P] * vfin[P]; },
        [&](int, double t) { qacc[0] += t; });
    cluster_reduce<1, CS>(qacc, wsl, csl, par, [&](double(&t)[1]) { ctl.s0 = t[0]; });
    if (rank == 0 && tid == 0) {
        g.q[sample] = status == S_NONFINITE ? __longlong_as_double(0x7ff8000000000000LL) : ctl.s0;
        g.iters[sample] = (int32_t)(total_iters > 0x7fffffff ? 0x7fffffff : total_iters);
        g.status[sample] = status;
    }
    cl.sync();
}

}  // namespace mlq
