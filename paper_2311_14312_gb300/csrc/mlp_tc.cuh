// The warm-start network's GEMMs on the 5th-generation tensor cores
// (tcgen05, kind::tf32): C[M][N] = sum_k A(m, k) B(n, k) (+ bias[n], GELU),
// with A(m, k) = A[m lda + k] or, with ta, A[k lda + m] (FP32), and B(n, k) =
// B[n ldb + k] or, with tb, B[k ldb + n] (FP32, or BF16 weights).
//
// BF16 values are exact in TF32, so a BF16 operand takes one term; an FP32
// operand is split into x_hi = tf32(x) and x_lo = tf32(x - x_hi), and the
// product A B^T is A_lo B_hi + A_hi B_lo + A_hi B_hi (the lo x lo term is
// below 2^-22 of the result) accumulated in FP32 in TMEM: the GEMM keeps the
// numerics of an FP32 product of the FP32 activations with the BF16 weights.
//
// One CTA (128 threads, thread t = row t of the tile) takes 128 rows and up
// to 256 columns: operands staged 32 values of K at a time in shared memory in
// the canonical K-major layout without swizzling (the M2L's layout: core
// matrices of 8 rows x 16 bytes, LBO 128, SBO 1024), one thread issues the
// MMAs (M 128, N up to 256, K 8), a bounded wait on their commit, then the
// accumulator is read back with tcgen05.ld for the epilogue.  A wait that
// runs out sets *err and ends the CTA's work after the issued MMAs are waited
// for once more (the accumulator is freed only then).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "passes_tc.cuh"

namespace dc {
namespace mlp {

constexpr int kGtM = 128, kGtN = 256, kGtK = 32;
constexpr size_t kGtSmem = (size_t)(2 * kGtM + 2 * kGtN) * kGtK * sizeof(float) + 1024;

template <typename TB>
__device__ __forceinline__ float gt_ldb(const TB *p, size_t i);
template <> __device__ __forceinline__ float gt_ldb<float>(const float *p, size_t i) { return p[i]; }
template <> __device__ __forceinline__ float gt_ldb<__nv_bfloat16>(const __nv_bfloat16 *p, size_t i) {
    return __bfloat162float(p[i]);
}

__device__ __forceinline__ float gt_gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }

// D (+)= A B^T over K = 32 (four MMAs of K = 8), N columns (multiple of 16)
__device__ __forceinline__ void gt_mma(uint32_t tmem, uint32_t sa, uint32_t sb, uint32_t idesc, uint32_t first) {
#pragma unroll
    for (int ks = 0; ks < kGtK / 8; ++ks) {
        const uint64_t da = passes::tc_desc(sa + ks * 2 * passes::kTcCoreLBO);
        const uint64_t db = passes::tc_desc(sb + ks * 2 * passes::kTcCoreLBO);
        const uint32_t acc = (ks > 0 || !first) ? 1u : 0u;
        asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                     " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                     ::"r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
    }
}

template <typename TB>
__global__ void __launch_bounds__(128) gemm_tc_kernel(int M, int N, int K, const float *__restrict__ A, int lda,
                                                      int ta, const TB *__restrict__ B, int ldb, int tb,
                                                      float *__restrict__ C, int ldc,
                                                      const float *__restrict__ bias, int act,
                                                      float *__restrict__ Zpre, int *__restrict__ err) {
    extern __shared__ unsigned char gt_raw[];
    // 1024-byte aligned tiles: A hi / lo [128 x 32], B hi / lo [256 x 32]
    float *base = reinterpret_cast<float *>(((uintptr_t)gt_raw + 1023) & ~(uintptr_t)1023);
    float *sAh = base, *sAl = sAh + kGtM * kGtK, *sBh = sAl + kGtM * kGtK, *sBl = sBh + kGtN * kGtK;
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int m0 = blockIdx.x * kGtM, n0 = blockIdx.y * kGtN;
    const int nn = min(kGtN, N - n0);
    const int nt = (nn + 15) / 16 * 16;   // MMA width: a multiple of 16 for M = 128
    constexpr bool b_exact = sizeof(TB) == 2;   // BF16 weights: exact in TF32, one term
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     ::"r"(passes::tc_smem(&tmem_base)), "r"(kGtN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(passes::tc_smem(&mbar)));
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_base;
    // D F32, A and B TF32, both K-major, N >> 3 at bits 17-22, M >> 4 at 24-28
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(nt >> 3) << 17) |
                           ((uint32_t)(kGtM >> 4) << 24);
    uint32_t phase = 0;
    bool ok = true;
    for (int k0 = 0; k0 < K; k0 += kGtK) {
        // A: 128 x 32, coalesced along the contiguous index of the source
        for (int u = tid; u < kGtM * kGtK; u += 128) {
            const int m = ta ? (u % kGtM) : (u / kGtK), k = ta ? (u / kGtM) : (u % kGtK);
            const int gm = m0 + m, gk = k0 + k;
            float v = 0.f;
            if (gm < M && gk < K) v = ta ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
            const float h = passes::tc_tf32(v);
            const int o = passes::tc_offset(m, k) / 4;
            sAh[o] = h;
            sAl[o] = passes::tc_tf32(v - h);
        }
        // B: nt x 32
        for (int u = tid; u < nt * kGtK; u += 128) {
            const int n = tb ? (u % nt) : (u / kGtK), k = tb ? (u / nt) : (u % kGtK);
            const int gn = n0 + n, gk = k0 + k;
            float v = 0.f;
            if (n < nn && gk < K) v = tb ? gt_ldb(B, (size_t)gk * ldb + gn) : gt_ldb(B, (size_t)gn * ldb + gk);
            const float h = passes::tc_tf32(v);
            const int o = passes::tc_offset(n, k) / 4;
            sBh[o] = h;
            if (!b_exact) sBl[o] = passes::tc_tf32(v - h);
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (tid == 0) {
            const uint32_t a_h = passes::tc_smem(sAh), a_l = passes::tc_smem(sAl);
            const uint32_t b_h = passes::tc_smem(sBh), b_l = passes::tc_smem(sBl);
            // small terms first
            gt_mma(tmem, a_l, b_h, idesc, k0 == 0 ? 1u : 0u);
            if (!b_exact) gt_mma(tmem, a_h, b_l, idesc, 0u);
            gt_mma(tmem, a_h, b_h, idesc, 0u);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                         ::"r"(passes::tc_smem(&mbar)));
        }
        uint32_t done = passes::tc_bounded_wait(passes::tc_smem(&mbar), phase);
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (__syncthreads_or(!done)) {
            if (tid == 0) atomicExch(err, 1);
            if (!done) passes::tc_bounded_wait(passes::tc_smem(&mbar), phase);
            ok = false;
            break;
        }
        phase ^= 1u;
        // the tiles are rewritten by the next chunk
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    }
    if (ok && K > 0) {
        const int gm = m0 + tid;
        for (int c0 = 0; c0 < nt; c0 += 32) {
            uint32_t r[32];
            const uint32_t addr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
                         "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
                           "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
                           "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
                           "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
                           "=r"(r[31])
                         : "r"(addr));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            if (gm < M)
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int gn = n0 + c0 + j;
                    if (c0 + j >= nn) break;
                    const float z = __uint_as_float(r[j]) + (bias ? bias[gn] : 0.f);
                    if (Zpre) Zpre[(size_t)gm * ldc + gn] = z;
                    C[(size_t)gm * ldc + gn] = act ? gt_gelu(z) : z;
                }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kGtN));
}

}  // namespace mlp
}  // namespace dc
