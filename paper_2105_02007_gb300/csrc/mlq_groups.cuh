// mlq_groups.cuh -- the CTAs that work on one sample, and how they meet.
//
// ClusterGroup<CS>: a thread-block cluster of CS CTAs (hardware cluster
//   barrier, sums exchanged through distributed shared memory).
// GridGroup: G CTAs of a cooperative launch (every CTA of the grid resident
//   at once), for samples that want more CTAs than a cluster holds.  The
//   CTAs of sample s are blocks s G .. s G + G - 1.  They meet at a barrier
//   in global memory (an arrival counter and a generation word per sample)
//   whose wait is bounded: after kGridWaitLimit polls the CTA records
//   MLQ error 1 in *err, marks the sample's barrier broken and returns; every
//   later barrier of that sample returns at once and every later sum is NaN,
//   so the solver's non-finite test ends the sample instead of a hang.
// Both give every CTA of the sample bit-identical sums: per-warp partials
// in the thread precision, FP64 above the warp, the CTA totals added in
// rank order.
#pragma once

#include <cooperative_groups.h>
#include <cstdint>

#include "mlq_kernels.cuh"

namespace mlq {

template <int CS>
struct ClusterGroup {
    static constexpr bool kCluster = true;
    __device__ int rank() const { return (int)cg::this_cluster().block_rank(); }
    __device__ int size() const { return CS; }
    __device__ int sample() const { return blockIdx.x / CS; }
    __device__ void sync() const { cg::this_cluster().sync(); }
    template <int NV, typename TA, typename F>
    __device__ void reduce(TA (&v)[NV], double (*wsl)[4], double (*csl)[4], int par, F &&fin) const
    {
        cluster_reduce<NV, CS>(v, wsl, csl, par, fin);
    }
};

constexpr long long kGridWaitLimit = 1LL << 24;   // polls of ~0.1-0.2 us: a few seconds

struct GridGroup {
    static constexpr bool kCluster = false;
    int G;
    unsigned *bar;    // [S][2]: arrivals, generation (zero before the launch)
    double *part;     // [S][2][G][4]: CTA totals of the two alternating sums
    int *err;         // set to 1 when a wait runs out
    long long limit = kGridWaitLimit;   // polls before a wait gives up
    __device__ int rank() const { return blockIdx.x % G; }
    __device__ int size() const { return G; }
    __device__ int sample() const { return blockIdx.x / G; }

    // every CTA of the sample has arrived (and its global writes are
    // visible); false once the sample's barrier is broken
    __device__ bool sync() const
    {
        __shared__ int s_ok;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned *cnt = bar + 2 * sample(), *gen = cnt + 1;
            volatile unsigned *vgen = gen;
            int ok = 1;
            const unsigned g0 = *vgen;
            if (g0 == 0xffffffffu) {
                ok = 0;   // broken by an earlier time-out
            } else {
                __threadfence();
                const unsigned a = atomicAdd(cnt, 1u);
                if (a == (unsigned)G - 1) {
                    atomicExch(cnt, 0u);
                    __threadfence();
                    atomicExch(gen, g0 + 1 == 0xffffffffu ? 0u : g0 + 1);
                } else {
                    long long it = 0;
                    while (*vgen == g0) {
                        if (++it > limit) {
                            atomicExch(err, 1);
                            atomicExch(gen, 0xffffffffu);
                            ok = 0;
                            break;
                        }
                        __nanosleep(100);
                    }
                    if (ok && *vgen == 0xffffffffu) ok = 0;
                }
                __threadfence();
            }
            s_ok = ok;
        }
        __syncthreads();
        return s_ok != 0;
    }

    template <int NV, typename TA, typename F>
    __device__ void reduce(TA (&v)[NV], double (*wsl)[4], double (*)[4], int par, F &&fin) const
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
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
        double *slot = part + ((size_t)sample() * 2 + par) * G * 4;
        if (warp == 0) {
            double acc[NV];
#pragma unroll
            for (int k = 0; k < NV; ++k) acc[k] = lane < nwarp ? wsl[lane][k] : 0.0;
            for (int o = 1; o < nwarp; o <<= 1) {
#pragma unroll
                for (int k = 0; k < NV; ++k) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
            }
            if (lane == 0) {
#pragma unroll
                for (int k = 0; k < NV; ++k) __stcg(slot + rank() * 4 + k, acc[k]);
            }
        }
        const bool ok = sync();
        if (warp == 0) {
            // lane l adds the CTA totals of ranks l, l + 32, ... in order, then
            // a butterfly over the lanes: the same order in every CTA
            double t[NV];
#pragma unroll
            for (int k = 0; k < NV; ++k) t[k] = 0.0;
            for (int r = lane; r < G; r += 32) {
#pragma unroll
                for (int k = 0; k < NV; ++k) t[k] += __ldcg(slot + r * 4 + k);
            }
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
                for (int k = 0; k < NV; ++k) t[k] += __shfl_xor_sync(0xffffffffu, t[k], o);
            }
            if (!ok) {
#pragma unroll
                for (int k = 0; k < NV; ++k) t[k] = __longlong_as_double(0x7ff8000000000000LL);
            }
            if (lane == 0) fin(t);
        }
        __syncthreads();
    }
};

}  // namespace mlq
