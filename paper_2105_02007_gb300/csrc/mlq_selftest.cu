// mlq_selftest.cu -- self-test of the global-memory group barrier and sums
// of the cooperative launch shapes (mlq_groups.cuh), with a bounded wait.
#include "mlq.h"
#include "mlq_groups.cuh"

#include <cuda_runtime.h>

#include <algorithm>

namespace {

// `rounds` barrier-and-sum rounds over the group: CTA r contributes r + 1,
// so every CTA must see G (G + 1) / 2; a wrong sum counts in *bad
__global__ void group_selftest_kernel(mlq::GridGroup grp, int rounds, int expect_G, int *bad)
{
    __shared__ double wsl[32][4];
    __shared__ double csl[2][4];
    int par = 0;
    const double expect = 0.5 * expect_G * (expect_G + 1.0);
    for (int r = 0; r < rounds; ++r) {
        double v[1] = {threadIdx.x == 0 ? (double)(grp.rank() + 1) : 0.0};
        grp.template reduce<1>(v, wsl, csl, par, [&](double(&t)[1]) {
            if (!(t[0] == expect)) atomicAdd(bad, 1);
        });
        par ^= 1;
    }
}

}  // namespace

extern "C" {

int mlq_group_selftest(int device, int ctas, int rounds, int missing, int64_t max_polls)
{
    if (ctas < 1 || ctas > 64 || rounds < 1 || rounds > 1000 || missing < 0 || missing > 64 || max_polls < 1)
        return MLQ_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return MLQ_ECUDA;
    const int G = ctas + missing;   // the group counts CTAs that never arrive when missing > 0
    char *blk = nullptr;
    const size_t part_b = (size_t)2 * G * 4 * sizeof(double);
    if (cudaMalloc(&blk, 256 + part_b) != cudaSuccess) {
        cudaGetLastError();
        return MLQ_ENOMEM;
    }
    unsigned *bar = (unsigned *)blk;                 // [1][2]
    int *err = (int *)(blk + 64), *bad = (int *)(blk + 128);
    double *part = (double *)(blk + 256);
    bool ok = cudaMemset(blk, 0, 256) == cudaSuccess;
    mlq::GridGroup grp{G, bar, part, err};
    grp.limit = max_polls;
    if (ok) {
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)ctas);
        cfg.blockDim = dim3(128);
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        ok = cudaLaunchKernelEx(&cfg, group_selftest_kernel, grp, rounds, G, bad) == cudaSuccess;
        ok = ok && cudaDeviceSynchronize() == cudaSuccess;
    }
    int h[2] = {0, 0};
    ok = ok && cudaMemcpy(&h[0], err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess;
    ok = ok && cudaMemcpy(&h[1], bad, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess;
    cudaFree(blk);
    if (!ok) return MLQ_ECUDA;
    if (h[0]) return MLQ_ETIMEOUT;
    return h[1] ? MLQ_EINVAL : MLQ_OK;
}

}  // extern "C"
