// mlq_3d_types.cuh -- geometry of the structured Kuhn-tetrahedra meshes and
// the argument block of the 3D time-block solver (shared by the host runtime
// and the kernels in mlq_3d.cuh).
#pragma once

#include <cstdint>

#include "mlq_points.cuh"

namespace mlq {

constexpr int kSlots3D = 9;  // diagonal, seven couplings, 1 / diagonal

// Node (i, j, k) of an mx x my x mz grid is stored at i + px (j + my k): rows
// are padded to px = mx rounded up to a multiple of 4, so that every row and
// plane starts on a 16-byte boundary of an FP32 array and the solver moves
// four consecutive nodes with one 16-byte access.  The pad entries (i >= mx)
// of every stencil slot, mass and vector are zero; a stencil slot that
// couples a node to a pad entry is zero as well (no such edge), so the pads
// take part in the passes and stay zero.  n counts the stored entries.
struct Grid3 {
    int mx, my, mz;
    int px;      // row pitch (multiple of 4)
    int n;       // px * my * mz stored entries
    double hx, hy, hz;
};

__host__ __device__ inline Grid3 make_grid3(int mx, int my, int mz, double hx, double hy, double hz)
{
    Grid3 g;
    g.mx = mx;
    g.my = my;
    g.mz = mz;
    g.px = (mx + 3) & ~3;
    g.n = g.px * my * mz;
    g.hx = hx;
    g.hy = hy;
    g.hz = hz;
    return g;
}

// stored index of node (i, j, k)
__host__ __device__ inline int64_t grid3_index(const Grid3 &g, int i, int j, int k)
{
    return (int64_t)i + (int64_t)g.px * (j + (int64_t)g.my * k);
}

// Kuhn steps: tetrahedron s of a cell steps along axes perm[s][0..2]
__host__ __device__ inline int kuhn_axis(int s, int q)
{
    // {0,1,2} {0,2,1} {1,0,2} {1,2,0} {2,0,1} {2,1,0}
    switch (s) {
    case 0: return q;                                   // 0 1 2
    case 1: return q == 0 ? 0 : (q == 1 ? 2 : 1);       // 0 2 1
    case 2: return q == 0 ? 1 : (q == 1 ? 0 : 2);       // 1 0 2
    case 3: return q == 0 ? 1 : (q == 1 ? 2 : 0);       // 1 2 0
    case 4: return q == 0 ? 2 : (q == 1 ? 0 : 1);       // 2 0 1
    default: return q == 0 ? 2 : (q == 1 ? 1 : 0);      // 2 1 0
    }
}

// vertex q of tetrahedron s as a corner bitmask of its cell (bit a = +1 along axis a)
__host__ __device__ inline int kuhn_vertex(int s, int q)
{
    int mask = 0;
    for (int t = 0; t < q; ++t) mask |= 1 << kuhn_axis(s, t);
    return mask;
}

__host__ __device__ inline int64_t dir_offset(const Grid3 &g, int slot)
{
    return (int64_t)(slot & 1) + (int64_t)g.px * (((slot >> 1) & 1) + (int64_t)g.my * ((slot >> 2) & 1));
}

// the same in 32 bits: the solver indexes a sample's arrays (at most nine
// slots of n nodes, n <= 2^27) with int
__host__ __device__ inline int dir_offset32(const Grid3 &g, int slot)
{
    return (slot & 1) + g.px * (((slot >> 1) & 1) + g.my * ((slot >> 2) & 1));
}

// Element matrices of tetrahedron s (|e| = hx hy hz / 6):
//   M_e[a][b] = |e| / 20 (1 + delta_ab),  K_e[a][b] = |e| g_a^T D g_b,
// D = s_t I + (s_l - s_t) f f^T, f = (cos t, sin t, 0), given (cos 2t, sin 2t).
// grad lambda_q in local coordinates: -e_a, e_a - e_b, e_b - e_c, e_c
// (a, b, c the step axes); divided by h per axis for physical gradients.
__host__ __device__ inline void kuhn_grads(const Grid3 &g, int s, double (&G)[4][3])
{
    const double ih[3] = {1.0 / g.hx, 1.0 / g.hy, 1.0 / g.hz};
    for (int q = 0; q < 4; ++q)
        for (int c = 0; c < 3; ++c) G[q][c] = 0.0;
    for (int t = 0; t < 3; ++t) {
        const int ax = kuhn_axis(s, t);
        G[t][ax] -= ih[ax];       // lambda_t loses xi_ax
        G[t + 1][ax] += ih[ax];   // lambda_{t+1} gains it
    }
}

// Geometric multigrid on the nested Kuhn hierarchy (regular refinement of
// the box: m_{c+1} = (m_c + 1) / 2 nodes per axis while every axis has an odd
// count >= 3).  Level 0 is the fine mesh; per sample and coarse level the
// stencil of A_c = M_c + dt K_c(Dbar_c) (Dbar_c the mean of D over the eight
// children of a coarse tetrahedron, which makes A_c = P^T A_{c-1} P for P1)
// and four work vectors.
constexpr int kMg3MaxLevels = 8;

struct Mg3Args {
    int nl;                           // levels including the fine one (1: Jacobi)
    float omega;                      // damped-Jacobi weight
    Grid3 g[kMg3MaxLevels];
    const float *A[kMg3MaxLevels];    // [S][9][n_c] (index 0 unused: the fine Ai)
    float *xa[kMg3MaxLevels], *xb[kMg3MaxLevels], *rr[kMg3MaxLevels], *bb[kMg3MaxLevels];  // [S][n_c]
};

// the hierarchy below a fine grid; returns the number of levels
__host__ __device__ inline int mg3_hierarchy(const Grid3 &g0, Grid3 *out, int max_levels)
{
    out[0] = g0;
    int nl = 1;
    while (nl < max_levels) {
        const Grid3 &f = out[nl - 1];
        if (f.mx < 3 || f.my < 3 || f.mz < 3 || (f.mx - 1) % 2 || (f.my - 1) % 2 || (f.mz - 1) % 2) break;
        out[nl++] = make_grid3((f.mx + 1) / 2, (f.my + 1) / 2, (f.mz + 1) / 2, 2.0 * f.hx, 2.0 * f.hy, 2.0 * f.hz);
    }
    return nl;
}

template <typename TI>
struct Solve3Args {
    Grid3 g;
    double Lx, Ly, Lz;
    double dt;
    int nsteps;
    double a, eps, gam;
    double rtol_out, rtol_in;
    int max_iter, max_sweeps;
    // every array below is in the padded layout of Grid3 (n stored entries
    // per sample and slot), except v0 and w0
    const double *M3, *lump;      // [8][n], [n] (level)
    const double *A64;            // [S][9][n]
    const TI *Ai;                 // [S][9][n] (the FP64 path: A64)
    double *v, *w, *b, *y;        // [kVRing][S][n], [2][S][n], [S][n], [S][n]
    TI *r, *u, *wv, *s, *p, *x;   // [S][n] each
    const double *v0, *w0;        // [mx my mz] unpadded, node i + mx (j + my k), or null
    double radius2;
    int S;
    double *q;
    int32_t *iters, *status;
    Mg3Args mg;                   // nl > 1: multigrid preconditioner (FP32 inner only)
    PointArgs pq;                 // point QoIs (npts = 0: none)
};

}  // namespace mlq
