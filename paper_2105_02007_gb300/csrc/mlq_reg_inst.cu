// mlq_reg_inst.cu -- instantiations of the register-resident slab solver for
// one cluster size, MLQ_CS (set on the compiler command line).
#include "mlq_launch.cuh"

#ifndef MLQ_CS
#error "compile with -DMLQ_CS=<cluster size>"
#endif

#define MLQ_CAT2(a, b) a##b
#define MLQ_CAT(a, b) MLQ_CAT2(a, b)

namespace mlq {

cudaError_t MLQ_CAT(launch_reg_cs, MLQ_CS)(int npt, const SolveArgs<float> &a, int nclusters, int threads,
                                           size_t smem, cudaStream_t st)
{
    switch (npt) {
    case 4: return cluster_launch<MLQ_CS>(slab_solve_reg_kernel<MLQ_CS, 4>, nclusters, threads, smem, st, a);
    case 8: return cluster_launch<MLQ_CS>(slab_solve_reg_kernel<MLQ_CS, 8>, nclusters, threads, smem, st, a);
    case 12: return cluster_launch<MLQ_CS>(slab_solve_reg_kernel<MLQ_CS, 12>, nclusters, threads, smem, st, a);
    case 17: return cluster_launch<MLQ_CS>(slab_solve_reg_kernel<MLQ_CS, 17>, nclusters, threads, smem, st, a);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t MLQ_CAT(launch_mg_cs, MLQ_CS)(int npt, const SolveArgs<float> &a, const MgPtrs &ptrs,
                                          const MgPlan &plan, int nclusters, int threads, cudaStream_t st)
{
    const size_t smem = (size_t)plan.total;
    switch (npt) {
    case 4: return cluster_launch<MLQ_CS>(slab_solve_mg_kernel<MLQ_CS, 4>, nclusters, threads, smem, st, a, ptrs, plan);
    case 8: return cluster_launch<MLQ_CS>(slab_solve_mg_kernel<MLQ_CS, 8>, nclusters, threads, smem, st, a, ptrs, plan);
    case 12:
        return cluster_launch<MLQ_CS>(slab_solve_mg_kernel<MLQ_CS, 12>, nclusters, threads, smem, st, a, ptrs, plan);
    default: return cudaErrorInvalidValue;
    }
}

int MLQ_CAT(active_reg_cs, MLQ_CS)(int npt, int threads, size_t smem)
{
    switch (npt) {
    case 4: return cluster_occupancy<MLQ_CS>(slab_solve_reg_kernel<MLQ_CS, 4>, threads, smem);
    case 8: return cluster_occupancy<MLQ_CS>(slab_solve_reg_kernel<MLQ_CS, 8>, threads, smem);
    case 12: return cluster_occupancy<MLQ_CS>(slab_solve_reg_kernel<MLQ_CS, 12>, threads, smem);
    case 17: return cluster_occupancy<MLQ_CS>(slab_solve_reg_kernel<MLQ_CS, 17>, threads, smem);
    default: return 0;
    }
}

}  // namespace mlq
