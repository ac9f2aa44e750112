// mlq_3d_inst.cu -- instantiations and launchers of the 3D (Kuhn tetrahedra)
// kernels.
#include "mlq_3d.cuh"
#include "mlq_launch.cuh"

namespace mlq {

template <typename TI>
cudaError_t launch_3d(int cs, const Solve3Args<TI> &a, int nclusters, int threads, cudaStream_t st)
{
    switch (cs) {
    case 1: return cluster_launch<1>(slab_solve_3d_kernel<TI, 1>, nclusters, threads, 0, st, a);
    case 2: return cluster_launch<2>(slab_solve_3d_kernel<TI, 2>, nclusters, threads, 0, st, a);
    case 4: return cluster_launch<4>(slab_solve_3d_kernel<TI, 4>, nclusters, threads, 0, st, a);
    case 8: return cluster_launch<8>(slab_solve_3d_kernel<TI, 8>, nclusters, threads, 0, st, a);
    case 16: return cluster_launch<16>(slab_solve_3d_kernel<TI, 16>, nclusters, threads, 0, st, a);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_3d_f32(int cs, const Solve3Args<float> &a, int nclusters, int threads, cudaStream_t st)
{
    return launch_3d<float>(cs, a, nclusters, threads, st);
}

cudaError_t launch_3d_f64(int cs, const Solve3Args<double> &a, int nclusters, int threads, cudaStream_t st)
{
    return launch_3d<double>(cs, a, nclusters, threads, st);
}

cudaError_t launch_level3d_setup(const Grid3 &g, double *M3, double *lump, cudaStream_t st)
{
    const int64_t nb = (g.n + 255) / 256;
    level3d_setup_kernel<<<(unsigned)nb, 256, 0, st>>>(g, M3, lump);
    return cudaGetLastError();
}

cudaError_t launch_stencil3d_setup(const double *cs2, const Grid3 &g, double dt, double s_l, double s_t, int S,
                                   double *A64, float *A32, cudaStream_t st)
{
    const int64_t nb = (g.n + 255) / 256;
    stencil3d_setup_kernel<<<dim3((unsigned)nb, (unsigned)S), 256, 0, st>>>(cs2, g, dt, s_l, s_t, S, A64, A32);
    return cudaGetLastError();
}

cudaError_t launch_mg3_setup(const double *cs2, const float *dfine, const Grid3 &gf, const Grid3 &gc, int S,
                             double dt, double s_l, double s_t, float *dc, float *Ac, cudaStream_t st)
{
    const int64_t nec = 6LL * (gc.mx - 1) * (gc.my - 1) * (gc.mz - 1);
    coarsen3d_kernel<<<dim3((unsigned)((nec + 255) / 256), (unsigned)S), 256, 0, st>>>(cs2, dfine, gf, gc, S, s_l,
                                                                                      s_t, dc);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    stencil3d_from_d_kernel<<<dim3((unsigned)((gc.n + 255) / 256), (unsigned)S), 256, 0, st>>>(dc, gc, dt, s_t, S,
                                                                                               Ac);
    return cudaGetLastError();
}

}  // namespace mlq
