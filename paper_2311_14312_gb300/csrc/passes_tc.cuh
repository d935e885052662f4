// M2L (Eq. 69 over list 2) of the FP32 inner operator on the 5th-generation
// tensor cores (tcgen05, kind::tf32), for inner orders p_i <= 15.
//
// Each list-2 pair applies one of 56 complex (P1 x P1) matrices F_v (7 base
// matrices x 4 rotations x conjugation) to the source cell's moments.  Written
// over the reals (x = [Re m_0, Im m_0, ..., Re m_{P1-1}, Im m_{P1-1}]), a pair
// and channel is a row of a GEMM
//
//     Y[(pair, channel)][n] = sum_k' X[(pair, channel)][k'] G_v[n][k'],
//
// G_v the realified F_v, zero-padded to 32 x 32.  The pairs are grouped by
// variant on the host; one CTA takes up to kTcPairs pairs of one variant
// (3 rows each, 128 rows), stages the gathered moments and G_v in shared
// memory in the canonical K-major layout without swizzling (core matrices of
// 8 rows x 16 bytes; LBO = 128 bytes between core matrices along K, SBO =
// 1024 bytes between core matrices along M or N), and one thread issues the
// MMAs (M = 128, N = 32, K = 8 each) into a 32-column TMEM accumulator.
//
// FP32 accuracy from TF32 inputs by the three-term split: x = x_hi + x_lo
// with x_hi = tf32(x), x_lo = tf32(x - x_hi) (both operands), and
// Y = X_lo G_hi + X_hi G_lo + X_hi G_hi accumulated in FP32 (the X_lo G_lo
// term is below 2^-22 of the result).  m2l_tc_reduce_kernel then adds the
// rows of each target cell's pairs in list order (deterministic) together
// with the -log(w) Mt_0 term of coefficient 0.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "passes.cuh"

namespace dc {
namespace passes {

constexpr int kTcThreads = 128;     // one CTA: 4 warps, one accumulator row each thread
constexpr int kTcPairs = 42;        // pairs per CTA (3 rows each, 126 of 128 rows)
constexpr int kTcK = 32;            // padded 2 P1
constexpr int kTcCoreLBO = 128;     // bytes between core matrices along K
constexpr int kTcCoreSBO = 1024;    // bytes between core matrices along M / N (32 / 4 x 128)
constexpr int kTcMaxP1 = 16;        // 2 P1 <= kTcK

// byte offset of element (row, k) in a 32-column K-major tile (canonical
// layout without swizzling)
__host__ __device__ __forceinline__ int tc_offset(int row, int k) {
    return (row >> 3) * kTcCoreSBO + (k >> 2) * kTcCoreLBO + (row & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ uint32_t tc_smem(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, LBO, SBO (all >> 4), the
// fixed 0b001 at bits 46-48, no swizzling
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(kTcCoreLBO >> 4) << 16;
    d |= (uint64_t)(kTcCoreSBO >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ float tc_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// D (+)= A B^T for the 128 x 32 tile A and the 32 x 32 tile B at the given
// shared addresses, K = 32 in four MMAs; accumulate = 0 overwrites D first.
__device__ __forceinline__ void tc_mma_128x32x32(uint32_t tmem, uint32_t sa, uint32_t sb, uint32_t accumulate) {
    // instruction descriptor: D F32 (bits 4-5 = 1), A and B TF32 (2 at bits
    // 7-9 and 10-12), both K-major, N >> 3 at bits 17-22, M >> 4 at 24-28
    constexpr uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(32 >> 3) << 17) |
                               ((uint32_t)(128 >> 4) << 24);
#pragma unroll
    for (int ks = 0; ks < kTcK / 8; ++ks) {
        const uint64_t da = tc_desc(sa + ks * 2 * kTcCoreLBO), db = tc_desc(sb + ks * 2 * kTcCoreLBO);
        const uint32_t acc = (ks > 0 || accumulate) ? 1u : 0u;
        asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                     " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                     ::"r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
    }
}

// tiles[i] = (variant, first entry in `entries`, pairs, 0); entries: list-2
// entry numbers (into v_idx) grouped by variant; btab[v] = G_v as TF32 hi
// and lo tiles (2 x 1024 floats) already in the canonical layout.  Writes
// Y[(e * 3 + c) * 2 P1 + n] for every listed entry e.  Persistent: CTA b
// takes tiles b, b + gridDim.x, ... with one TMEM allocation.
//
// err[0]: set to 1 when the MMAs of a tile did not complete within the wait
// limit (kTcWaitNs of %globaltimer, and at most kTcWaitIters polls); the CTA
// then stops taking tiles.  err[1]: a test hook, normally -1: the CTA that
// takes tile err[1] issues neither the MMAs nor the commit of that tile, so
// nothing will arrive on the mbarrier and its bounded wait runs out.
//
// The accumulator is freed (tcgen05.dealloc) on every exit.  Freeing TMEM is
// only safe once no MMA that writes it is still in flight: after a wait that
// ran out on a tile whose MMAs were issued, the CTA waits once more, with the
// same bounds, for their commit before it frees the columns; on the test
// hook's tile nothing was issued, so nothing can be in flight.
constexpr int kTcBlocksPerSM = 4;
constexpr unsigned long long kTcWaitNs = 20000000ull;   // 20 ms; a tile's MMAs take about a microsecond
constexpr int kTcWaitIters = 1 << 24;

__device__ __forceinline__ unsigned long long tc_globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}

// Polls the mbarrier phase until it completes or the bounds run out; 1 if it
// completed.
__device__ __forceinline__ uint32_t tc_bounded_wait(uint32_t mbar_addr, uint32_t phase) {
    uint32_t done = 0;
    const unsigned long long t0 = tc_globaltimer();
    for (int it = 0; it < kTcWaitIters && !done; ++it) {
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(mbar_addr), "r"(phase));
        if (!done && (it & 63) == 63 && tc_globaltimer() - t0 > kTcWaitNs) break;
    }
    return done;
}

static __global__ void __launch_bounds__(kTcThreads) m2l_tc_kernel(const int4 *__restrict__ tiles, int n_tiles,
                                                                   const int *__restrict__ entries,
                                                                   const int *__restrict__ v_idx, int P1,
                                                                   const float *__restrict__ btab,
                                                                   const float2 *__restrict__ M,
                                                                   float *__restrict__ Y, int *__restrict__ err) {
    const int skip_tile = err[1];
    __shared__ __align__(1024) float sAh[128 * kTcK];
    __shared__ __align__(1024) float sAl[128 * kTcK];
    __shared__ __align__(1024) float sBh[32 * kTcK];
    __shared__ __align__(1024) float sBl[32 * kTcK];
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     ::"r"(tc_smem(&tmem_base)), "r"(32));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(tc_smem(&mbar)));
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_base;
    const int pi = tid / 3, c = tid - 3 * pi;   // row tid = 3 pair + channel
    uint32_t phase = 0;
    for (int ti = blockIdx.x; ti < n_tiles; ti += gridDim.x) {
        const int4 tl = tiles[ti];
        // G_v (hi, lo): 2 x 4 KB by asynchronous 16-byte copies
        const float *bsrc = btab + (size_t)tl.x * 2 * 32 * kTcK;
        for (int i = tid; i < 32 * kTcK / 4; i += kTcThreads) {
            cp_async16(sBh + 4 * i, bsrc + 4 * i);
            cp_async16(sBl + 4 * i, bsrc + 32 * kTcK + 4 * i);
        }
        cp_async_commit();
        // the row's source moments, split into TF32 hi / lo
        const bool live = pi < tl.z;
        int e = 0;
        float x[kTcK];
#pragma unroll
        for (int k = 0; k < kTcK; ++k) x[k] = 0.f;
        if (live) {
            e = entries[tl.y + pi];
            const float2 *src = M + ((size_t)v_idx[e] * 3 + c) * P1;
#pragma unroll
            for (int k = 0; k < kTcMaxP1; ++k)
                if (k < P1) {
                    const float2 m = src[k];
                    x[2 * k] = m.x;
                    x[2 * k + 1] = m.y;
                }
        }
#pragma unroll
        for (int k4 = 0; k4 < kTcK; k4 += 4) {
            float4 h, l;
            h.x = tc_tf32(x[k4]);
            h.y = tc_tf32(x[k4 + 1]);
            h.z = tc_tf32(x[k4 + 2]);
            h.w = tc_tf32(x[k4 + 3]);
            l.x = tc_tf32(x[k4] - h.x);
            l.y = tc_tf32(x[k4 + 1] - h.y);
            l.z = tc_tf32(x[k4 + 2] - h.z);
            l.w = tc_tf32(x[k4 + 3] - h.w);
            const int o = tc_offset(tid, k4) / 4;
            *reinterpret_cast<float4 *>(sAh + o) = h;
            *reinterpret_cast<float4 *>(sAl + o) = l;
        }
        cp_async_wait<0>();
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");   // generic writes -> tensor core reads
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const bool issue = ti != skip_tile;
        if (tid == 0 && issue) {
            // small terms first: X_lo G_hi, X_hi G_lo, then X_hi G_hi
            tc_mma_128x32x32(tmem, tc_smem(sAl), tc_smem(sBh), 0u);
            tc_mma_128x32x32(tmem, tc_smem(sAh), tc_smem(sBl), 1u);
            tc_mma_128x32x32(tmem, tc_smem(sAh), tc_smem(sBh), 1u);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                         ::"r"(tc_smem(&mbar)));
        }
        // wait for the MMAs, bounded in time and in polls
        uint32_t done = tc_bounded_wait(tc_smem(&mbar), phase);
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (__syncthreads_or(!done)) {
            if (tid == 0) atomicExch(err, 1);
            // MMAs that were issued may still be running: wait for their
            // commit once more before the accumulator is freed below
            if (issue && !done) done = tc_bounded_wait(tc_smem(&mbar), phase);
            break;
        }
        phase ^= 1u;
        uint32_t r[32];
        const uint32_t addr = tmem + ((uint32_t)(warp * 32) << 16);
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
                     "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                       "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                       "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
                       "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
                       "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                     : "r"(addr));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        if (live) {
            float *y = Y + ((size_t)e * 3 + c) * (2 * P1);
#pragma unroll
            for (int n = 0; n < kTcK; ++n)
                if (n < 2 * P1) y[n] = __uint_as_float(r[n]);
        }
        // shared tiles and the accumulator are reused by the next tile
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(32));
}

// Lout[cell][c] += sum over the cell's list-2 entries e, in list order, of
// Y[e][c] + (coefficient 0) -log(w_cell) Re Mt_0 of the source (Lout holds
// zero or the cell's list-4 P2L terms).  One warp
// per cell, lane j holds real component j of the 2 P1.
constexpr int kTcReduceWarps = 8;
static __global__ void __launch_bounds__(32 * kTcReduceWarps) m2l_tc_reduce_kernel(TreeView<float> t,
                                                                                  const int *__restrict__ cells,
                                                                                  int n_cells, int P1,
                                                                                  const float *__restrict__ Y,
                                                                                  const float2 *__restrict__ M,
                                                                                  float2 *__restrict__ Lout) {
    const int ci = blockIdx.x * kTcReduceWarps + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (ci >= n_cells) return;
    const int cell = cells[ci];
    const int n2 = 2 * P1;
    const float mlogw = -t.logw[cell];
    const int e0 = t.v_ptr[cell], e1 = t.v_ptr[cell + 1];
    float acc[3] = {0.f, 0.f, 0.f};
    if (lane < n2)
        for (int eb = e0; eb < e1; eb += 4) {
            // four entries' loads in flight, added in list order
            float yv[4][3], mv[4][3];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = eb + u;
                const bool ok = e < e1;
                const float *y = Y + (size_t)(ok ? e : e0) * 3 * n2 + lane;
                yv[u][0] = ok ? y[0] : 0.f;
                yv[u][1] = ok ? y[n2] : 0.f;
                yv[u][2] = ok ? y[2 * n2] : 0.f;
                mv[u][0] = mv[u][1] = mv[u][2] = 0.f;
                if (lane == 0 && ok) {   // Mt_0 is real
                    const float2 *ms = M + (size_t)t.v_idx[e] * 3 * P1;
                    mv[u][0] = ms[0].x;
                    mv[u][1] = ms[P1].x;
                    mv[u][2] = ms[2 * P1].x;
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                for (int c = 0; c < 3; ++c) acc[c] += yv[u][c] + mlogw * mv[u][c];
        }
    if (lane < n2) {
        float *o = reinterpret_cast<float *>(Lout) + (size_t)cell * 3 * n2 + lane;
        o[0] += acc[0];
        o[n2] += acc[1];
        o[2 * n2] += acc[2];
    }
}

}  // namespace passes
}  // namespace dc
