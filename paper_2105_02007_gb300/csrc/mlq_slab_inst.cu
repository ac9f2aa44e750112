// mlq_slab_inst.cu -- instantiations of the general slab solver (vectors in
// shared or global memory) for one inner precision: MLQ_F64 = 1 (FP64 path)
// or 0 (FP32 inner solves of the mixed path), set on the command line.
#include "mlq_launch.cuh"

#ifndef MLQ_F64
#error "compile with -DMLQ_F64=0 or 1"
#endif

namespace mlq {

#if MLQ_F64
using TI = double;
#define MLQ_LAUNCH_SLAB launch_slab_f64
#else
using TI = float;
#define MLQ_LAUNCH_SLAB launch_slab_f32
#endif

template <int CS>
static cudaError_t launch_cs(bool resident, const SolveArgs<TI> &a, int nclusters, int threads, size_t smem,
                             cudaStream_t st)
{
    if (resident) return cluster_launch<CS>(slab_solve_kernel<TI, CS, true>, nclusters, threads, smem, st, a);
    return cluster_launch<CS>(slab_solve_kernel<TI, CS, false>, nclusters, threads, smem, st, a);
}

cudaError_t MLQ_LAUNCH_SLAB(int cs, bool resident, const SolveArgs<TI> &a, int nclusters, int threads, size_t smem,
                            cudaStream_t st)
{
    switch (cs) {
    case 1: return launch_cs<1>(resident, a, nclusters, threads, smem, st);
    case 2: return launch_cs<2>(resident, a, nclusters, threads, smem, st);
    case 4: return launch_cs<4>(resident, a, nclusters, threads, smem, st);
    case 8: return launch_cs<8>(resident, a, nclusters, threads, smem, st);
    case 16: return launch_cs<16>(resident, a, nclusters, threads, smem, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace mlq
