// mlq_kl_tc.cuh -- KL synthesis on the 5th-generation tensor cores (tcgen05).
//
// theta[s, e] = theta_mean[e] + sum_k Phi[e, k] xi[s, k]          (eq. KLlowrank)
// as a GEMM D (128 elements x NT samples) = A (128 x K) . B^T (NT x K) per CTA
// tile, accumulated in FP32 in tensor memory.  Operands are FP32 split into
// two TF32 parts, x = x_hi + x_lo (x_hi = x with the low 13 mantissa bits
// cleared), and the product is formed as A_hi B_hi + A_hi B_lo + A_lo B_hi
// (the split-precision scheme of Markidis et al., IPDPSW 2018), which keeps
// about 21 bits: the angle error stays near 1e-6 of |theta|.  Epilogue:
// (cos 2 theta, sin 2 theta) for the stencil set-up (K2).
//
// Shared-memory operand layout (K-major, no swizzle): 8-row x 16-byte core
// matrices; element (r, k) of a tile sits at
//   (r / 8) * SBO + (k / 4) * LBO + (r % 8) * 16 + (k % 4) * 4
// with LBO = 128 B (next 4 k) and SBO = Kp / 4 * 128 B (next 8 rows).
// One thread issues the MMAs; completion is signalled through an mbarrier
// (tcgen05.commit) whose wait is bounded: on time-out the kernel records an
// error, waits (bounded) once more for the MMAs, frees its tensor memory and
// returns.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mlq {

constexpr int kTcM = 128;   // elements per tile (MMA M)

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor (tcgen05): start, leading / stride byte
// offsets (>> 4), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor, kind::tf32: D F32, A and B TF32, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t tc_idesc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t addr, uint32_t phase)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred P1;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, P1;\n\t}\n"
        : "=r"(done)
        : "r"(addr), "r"(phase)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ uint32_t tf32_hi(float x) { return __float_as_uint(x) & 0xFFFFE000u; }

// grid (ceil(ne / 128), ceil(S / NT)); 128 threads; dynamic shared memory
// 2 * (128 + NT) * Kp * 4 bytes + 64.  Kp = K rounded up to 8; NT in
// {16, 32, ..., 256}.  phi_hi / phi_lo: ne x Kp FP32 (zero padded).
// err: device int, set to 1 if a wait timed out.
__global__ void __launch_bounds__(128) kl_synthesis_tc_kernel(const float *__restrict__ phi_hi,
                                                               const float *__restrict__ phi_lo,
                                                               const double *__restrict__ theta_mean,
                                                               const double *__restrict__ xi, int K, int Kp, int ne,
                                                               int S, int NT, double *__restrict__ out, int *err)
{
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int e0 = blockIdx.x * kTcM, s0 = blockIdx.y * NT;
    const uint32_t LBO = 128, SBO = (uint32_t)(Kp / 4) * 128;
    unsigned char *A_hi = sm, *A_lo = sm + kTcM * Kp * 4;
    unsigned char *B_hi = A_lo + kTcM * Kp * 4, *B_lo = B_hi + NT * Kp * 4;
    auto off = [&](int r, int k) { return (r >> 3) * SBO + (k >> 2) * LBO + (r & 7) * 16 + (k & 3) * 4; };

    // ---- operands into shared memory (zero beyond ne / S / K)
    for (int idx = tid; idx < kTcM * Kp; idx += blockDim.x) {
        const int r = idx / Kp, k = idx - r * Kp;
        const int e = e0 + r;
        float h = 0.0f, l = 0.0f;
        if (e < ne) {
            h = phi_hi[(size_t)e * Kp + k];
            l = phi_lo[(size_t)e * Kp + k];
        }
        *reinterpret_cast<float *>(A_hi + off(r, k)) = h;
        *reinterpret_cast<float *>(A_lo + off(r, k)) = l;
    }
    for (int idx = tid; idx < NT * Kp; idx += blockDim.x) {
        const int r = idx / Kp, k = idx - r * Kp;
        const int s = s0 + r;
        const float x = (s < S && k < K) ? (float)xi[(size_t)s * K + k] : 0.0f;
        const uint32_t hb = tf32_hi(x);
        const float h = __uint_as_float(hb);
        *reinterpret_cast<float *>(B_hi + off(r, k)) = h;
        *reinterpret_cast<float *>(B_lo + off(r, k)) = x - h;
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&mbar)), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // make the generic-proxy stores visible to the tensor core's async proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    uint32_t ncols = 32;
    while ((int)ncols < NT) ncols <<= 1;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t mb = smem_addr(&mbar);

    // ---- MMAs: for each K-step of 8, hi.hi + hi.lo + lo.hi
    if (tid == 0) {
        const uint32_t idesc = tc_idesc_tf32(kTcM, NT);
        const uint32_t a_hi = smem_addr(A_hi), a_lo = smem_addr(A_lo), b_hi = smem_addr(B_hi), b_lo = smem_addr(B_lo);
        uint32_t acc = 0;
        for (int kk = 0; kk < Kp; kk += 8) {
            const uint32_t ko = (uint32_t)(kk / 4) * LBO;
            tc_mma_tf32(tmem, tc_smem_desc(a_hi + ko, LBO, SBO), tc_smem_desc(b_hi + ko, LBO, SBO), idesc, acc);
            acc = 1;
            tc_mma_tf32(tmem, tc_smem_desc(a_hi + ko, LBO, SBO), tc_smem_desc(b_lo + ko, LBO, SBO), idesc, acc);
            tc_mma_tf32(tmem, tc_smem_desc(a_lo + ko, LBO, SBO), tc_smem_desc(b_hi + ko, LBO, SBO), idesc, acc);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
                     : "memory");
    }
    // ---- wait for the accumulator (bounded)
    bool ok = false;
    for (int spin = 0; spin < (1 << 24); ++spin) {
        if (mbar_try_wait(mb, 0)) {
            ok = true;
            break;
        }
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        // epilogue: warp w reads TMEM lanes 32w .. 32w+31 (= elements)
        const int e = e0 + warp * 32 + lane;
        const double tm = (e < ne && theta_mean) ? theta_mean[e] : 0.0;
        for (int c = 0; c < NT; c += 8) {
            uint32_t v[8];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (e < ne) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int s = s0 + c + j;
                    if (s < S) {
                        const float th = (float)(tm + (double)__uint_as_float(v[j]));
                        float sn, cs;
                        sincosf(2.0f * th, &sn, &cs);
                        out[((size_t)s * ne + e) * 2 + 0] = (double)cs;
                        out[((size_t)s * ne + e) * 2 + 1] = (double)sn;
                    }
                }
            }
        }
    } else {
        if (tid == 0) atomicExch(err, 1);
        for (int spin = 0; spin < (1 << 24); ++spin)
            if (mbar_try_wait(mb, 0)) break;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }
}

}  // namespace mlq
