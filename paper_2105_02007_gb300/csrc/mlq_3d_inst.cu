// mlq_3d_inst.cu -- instantiations and launchers of the 3D (Kuhn tetrahedra)
// kernels.  Compiled twice: MLQ_F64 = 0 (FP32 inner solve, with the level
// set-up kernels) and MLQ_F64 = 1 (FP64 inner solve), so that the two build
// in parallel.
#ifndef MLQ_F64
#define MLQ_F64 0
#endif
#if !MLQ_F64
#define MLQ_3D_SETUP
#endif

#include "mlq_3d.cuh"
#include "mlq_launch.cuh"

#include <type_traits>

namespace mlq {

namespace {

#if MLQ_F64
using TI3 = double;
#else
using TI3 = float;
#endif

template <typename F>
cudaError_t with_cs(int cs, F &&f)
{
    switch (cs) {
    case 1: return f(std::integral_constant<int, 1>{});
    case 2: return f(std::integral_constant<int, 2>{});
    case 4: return f(std::integral_constant<int, 4>{});
    case 6: return f(std::integral_constant<int, 6>{});
    case 8: return f(std::integral_constant<int, 8>{});
    case 12: return f(std::integral_constant<int, 12>{});
    case 16: return f(std::integral_constant<int, 16>{});
    default: return cudaErrorInvalidValue;
    }
}

// CTAs of the 3D solver resident at once on the device
int64_t resident_3d(int threads)
{
    int dev = 0, nsm = 1, nb = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, slab_solve_3d_kernel<TI3, GridGroup>, threads, 0) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return (int64_t)nb * nsm;
}

}  // namespace

// cs <= 16: one cluster of cs CTAs per sample; cs > 16: cs CTAs per sample
// in one cooperative launch (bar: [S][2] zeroed here, part: [S][2][cs][4])
#if MLQ_F64
cudaError_t launch_3d_f64(int cs, const Solve3Args<double> &a, int nsamples, int threads, cudaStream_t st,
                          unsigned *bar, double *part, int *err)
#else
cudaError_t launch_3d_f32(int cs, const Solve3Args<float> &a, int nsamples, int threads, cudaStream_t st,
                          unsigned *bar, double *part, int *err)
#endif
{
    if (cs > 16) {
        if (!bar || !part || !err) return cudaErrorInvalidValue;
        cudaError_t e = cudaMemsetAsync(bar, 0, (size_t)nsamples * 2 * sizeof(unsigned), st);
        if (e != cudaSuccess) return e;
        int prio = 0;
        if ((e = cudaStreamGetPriority(st, &prio)) != cudaSuccess) return e;
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)(nsamples * cs));
        cfg.blockDim = dim3((unsigned)threads);
        cfg.stream = st;
        cudaLaunchAttribute attr[2];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        attr[1].id = cudaLaunchAttributePriority;
        attr[1].val.priority = prio;
        cfg.attrs = attr;
        cfg.numAttrs = 2;
        const GridGroup grp{cs, bar, part, err};
        return cudaLaunchKernelEx(&cfg, slab_solve_3d_kernel<TI3, GridGroup>, a, grp);
    }
    return with_cs(cs, [&](auto c) {
        constexpr int CS = decltype(c)::value;
        return cluster_launch<CS>(slab_solve_3d_kernel<TI3, ClusterGroup<CS>>, nsamples, threads, 0, st, a,
                                  ClusterGroup<CS>{});
    });
}

#if MLQ_F64
int64_t resident_3d_f64(int threads)
#else
int64_t resident_3d_f32(int threads)
#endif
{
    return resident_3d(threads);
}

// samples whose groups can be resident at once: clusters for cs <= 16, the
// CTAs of a cooperative launch over cs for cs > 16
#if MLQ_F64
int active_3d_f64(int cs, int threads)
#else
int active_3d_f32(int cs, int threads)
#endif
{
    if (cs > 16) return (int)(resident_3d(threads) / cs);
    int nc = 0;
    with_cs(cs, [&](auto c) {
        constexpr int CS = decltype(c)::value;
        nc = cluster_occupancy<CS>(slab_solve_3d_kernel<TI3, ClusterGroup<CS>>, threads, 0);
        return cudaSuccess;
    });
    return nc;
}

#if !MLQ_F64

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

#endif

}  // namespace mlq
