// mlq_launch.cuh -- launch entry points of the slab-solver kernels.
//
// The kernel templates are instantiated in separate translation units
// (mlq_reg_inst.cu once per cluster size, mlq_slab_inst.cu once per inner
// precision) so that the library builds in parallel; the host runtime calls
// them through these functions.
#pragma once

#include <cstddef>
#include <cuda_runtime.h>

#include "mlq_3d_types.cuh"
#include "mlq_kernels.cuh"
#include "mlq_mg.cuh"

namespace mlq {

#define MLQ_DECLARE_REG(CS)                                                                                   \
    cudaError_t launch_reg_cs##CS(int npt, const SolveArgs<float> &a, int nclusters, int threads, size_t smem, \
                                  cudaStream_t st);                                                           \
    int active_reg_cs##CS(int npt, int threads, size_t smem);                                                  \
    cudaError_t launch_mg_cs##CS(int npt, const SolveArgs<float> &a, const MgPtrs &ptrs, const MgPlan &plan,  \
                                 int nclusters, int threads, cudaStream_t st);
MLQ_DECLARE_REG(1)
MLQ_DECLARE_REG(2)
MLQ_DECLARE_REG(4)
MLQ_DECLARE_REG(8)
MLQ_DECLARE_REG(16)
#undef MLQ_DECLARE_REG

// 3D (Kuhn tetrahedra), mlq_3d_inst.cu
// cs <= 16: one cluster of cs CTAs per sample (sizes 1, 2, 4, 6, 8, 12,
// 16); cs > 16: cs CTAs per sample in one cooperative launch whose
// per-sample barriers live in bar ([S][2], zeroed by the call) and part
// ([S][2][cs][4]), err set when a barrier wait runs out
cudaError_t launch_3d_f32(int cs, const Solve3Args<float> &a, int nsamples, int threads, cudaStream_t st,
                          unsigned *bar = nullptr, double *part = nullptr, int *err = nullptr);
cudaError_t launch_3d_f64(int cs, const Solve3Args<double> &a, int nsamples, int threads, cudaStream_t st,
                          unsigned *bar = nullptr, double *part = nullptr, int *err = nullptr);
// samples of the 3D solver resident at once (clusters for cs <= 16, 0: the
// size is not built or does not fit; cooperative CTAs / cs for cs > 16)
int active_3d_f32(int cs, int threads);
int active_3d_f64(int cs, int threads);
// CTAs of the 3D solver resident at once
int64_t resident_3d_f32(int threads);
int64_t resident_3d_f64(int threads);
cudaError_t launch_level3d_setup(const Grid3 &g, double *M3, double *lump, cudaStream_t st);
cudaError_t launch_stencil3d_setup(const double *cs2, const Grid3 &g, double dt, double s_l, double s_t, int S,
                                   double *A64, float *A32, cudaStream_t st);
cudaError_t launch_mg3_setup(const double *cs2, const float *dfine, const Grid3 &gf, const Grid3 &gc, int S,
                             double dt, double s_l, double s_t, float *dc, float *Ac, cudaStream_t st);

cudaError_t launch_slab_f32(int cs, bool resident, const SolveArgs<float> &a, int nclusters, int threads,
                            size_t smem, cudaStream_t st);
cudaError_t launch_slab_f64(int cs, bool resident, const SolveArgs<double> &a, int nclusters, int threads,
                            size_t smem, cudaStream_t st);

// cluster launch of `kern` with CS CTAs per cluster
template <int CS, typename K, typename... A>
cudaError_t cluster_launch(K kern, int nclusters, int threads, size_t smem, cudaStream_t st, const A &...args)
{
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (CS > 8) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(nclusters * CS));
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    // the stream's priority as a launch attribute: a captured graph node
    // keeps it
    int prio = 0;
    e = cudaStreamGetPriority(st, &prio);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributePriority;
    attr[1].val.priority = prio;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// clusters of `kern` that can be resident at once (0 if none / on error)
template <int CS, typename K>
int cluster_occupancy(K kern, int threads, size_t smem)
{
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (CS > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)CS);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, kern, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nc;
}

}  // namespace mlq
