// mlq_3d_types.cuh -- geometry of the structured Kuhn-tetrahedra meshes and
// the argument block of the 3D time-block solver (shared by the host runtime
// and the kernels in mlq_3d.cuh).
#pragma once

#include <cstdint>

namespace mlq {

constexpr int kSlots3D = 9;  // diagonal, seven couplings, 1 / diagonal

struct Grid3 {
    int mx, my, mz, n;
    double hx, hy, hz;
};

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
    return (int64_t)(slot & 1) + (int64_t)g.mx * (((slot >> 1) & 1) + (int64_t)g.my * ((slot >> 2) & 1));
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

template <typename TI>
struct Solve3Args {
    Grid3 g;
    double Lx, Ly, Lz;
    double dt;
    int nsteps;
    double a, eps, gam;
    double rtol_out, rtol_in;
    int max_iter, max_sweeps;
    const double *M3, *lump;      // [8][n], [n] (level)
    const double *A64;            // [S][9][n]
    const TI *Ai;                 // [S][9][n] (the FP64 path: A64)
    double *v, *w, *b, *y;        // [S][n], [2][S][n], [S][n], [S][n]
    TI *r, *u, *wv, *s, *p, *x;   // [S][n] each
    const double *v0, *w0;        // [n] or null
    double radius2;
    int S;
    double *q;
    int32_t *iters, *status;
};

}  // namespace mlq
