// Evaluation of the FMM at listed targets (the collocation nodes of the
// matvec, or sorted points): L2P (Eq. 64) + list-3 M2P (Eq. 61) + list-1
// P2P (App. D) per target, templated on the real type.
//
// One block per work item (up to kNodeItem targets of one leaf), 4 warps.
// The list-1 pieces are staged in shared memory in the leaf's frame (FP64
// differences, then rounded to T); each warp owns a subset of the targets
// and its 32 lanes split the staged pieces, so a leaf with few targets still
// keeps every lane busy.  Lane partial sums are combined by a fixed
// butterfly (deterministic).
#pragma once

#include <cuda_runtime.h>

#include "passes.cuh"

namespace dc {
namespace evalnodes {

constexpr int kNodeItem = 16;      // targets per work item
constexpr int kWarps = 4;
constexpr int kStageN = 128;

template <typename T> struct NodeArgs {
    const int *u_ptr, *u_idx, *w_ptr, *w_idx, *pstart, *pcount, *pseg;
    const double *pc64;            // [np][4] absolute
    const double *cc64;            // [cells][2]
    const T *pw;                   // arc weight
    const T *iw, *logw;
    const int4 *items;             // (leaf, first target, count, 0)
    const double *q64;             // [n][2] sorted targets
    const int *own1, *own2, *perm; // own segments (may be null), output order
    int P1;
    const typename passes::V2<T>::type *M, *L;
    const T *sb, *mb;
    int use_s, use_m;
    double *out;                   // [n][3] in the original order
};

__device__ __forceinline__ float elog(float x) { return __logf(x); }
__device__ __forceinline__ double elog(double x) { return log(x); }

template <typename T>
__global__ void __launch_bounds__(32 * kWarps) eval_nodes_kernel(NodeArgs<T> a) {
    using C = typename passes::V2<T>::type;
    __shared__ T sx1[kStageN], sy1[kStageN], sx2[kStageN], sy2[kStageN];
    __shared__ T ssg[3][kStageN], smg[3][kStageN];
    __shared__ int sseg[kStageN];
    const int4 it = a.items[blockIdx.x];
    const int leaf = it.x, t0 = it.y, nt = it.z;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double cx = a.cc64[2 * leaf], cy = a.cc64[2 * leaf + 1];
    constexpr int kPer = kNodeItem / kWarps;   // targets per warp
    T qx[kPer], qy[kPer], acc[kPer][3];
    int o1[kPer], o2[kPer];
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        int ti = t0 + warp + kWarps * j;
        bool ok = (warp + kWarps * j) < nt;
        qx[j] = ok ? (T)(a.q64[2 * ti] - cx) : T(0);
        qy[j] = ok ? (T)(a.q64[2 * ti + 1] - cy) : T(0);
        o1[j] = (ok && a.own1) ? a.own1[ti] : -1;
        o2[j] = (ok && a.own2) ? a.own2[ti] : -1;
        acc[j][0] = acc[j][1] = acc[j][2] = T(0);
    }
    const T k2pi = T(0.15915494309189533577);
    // P2P over list 1
    for (int e = a.u_ptr[leaf]; e < a.u_ptr[leaf + 1]; ++e) {
        const int src = a.u_idx[e];
        const int p0 = a.pstart[src], pn = a.pcount[src];
        for (int base = 0; base < pn; base += kStageN) {
            const int cnt = min(kStageN, pn - base);
            __syncthreads();
            for (int s = threadIdx.x; s < cnt; s += blockDim.x) {
                const int i = p0 + base + s;
                const double *P = a.pc64 + 4 * (size_t)i;
                sx1[s] = (T)(P[0] - cx);
                sy1[s] = (T)(P[1] - cy);
                sx2[s] = (T)(P[2] - cx);
                sy2[s] = (T)(P[3] - cy);
                const int seg = a.pseg[i];
                const T wg = -a.pw[i] * k2pi;
                for (int c = 0; c < 3; ++c) {
                    ssg[c][s] = a.use_s ? wg * a.sb[3 * (size_t)seg + c] : T(0);
                    smg[c][s] = a.use_m ? wg * a.mb[3 * (size_t)seg + c] : T(0);
                }
                sseg[s] = seg;
            }
            __syncthreads();
            for (int s = lane; s < cnt; s += 32) {
                const T x1 = sx1[s], y1 = sy1[s], x2 = sx2[s], y2 = sy2[s];
                const T dx = x2 - x1, dy = y2 - y1;
                const T len = sqrt(dx * dx + dy * dy), ilen = T(1) / len;
                const int seg = sseg[s];
#pragma unroll
                for (int j = 0; j < kPer; ++j) {
                    if (warp + kWarps * j >= nt) break;
                    const T ax = x1 - qx[j], ay = y1 - qy[j], bx = x2 - qx[j], by = y2 - qy[j];
                    const T cr = ax * by - ay * bx, dt = ax * bx + ay * by;
                    const bool own = (seg == o1[j]) || (seg == o2[j]);
                    const T phi = own ? T(0) : passes::tatan2(cr, dt);
                    const T ra2 = ax * ax + ay * ay, rb2 = bx * bx + by * by;
                    const T s1 = (ax * dx + ay * dy) * ilen, s2 = s1 + len;
                    const T la = ra2 > T(0) ? s1 * elog(ra2) : T(0);
                    const T lb = rb2 > T(0) ? s2 * elog(rb2) : T(0);
                    const T il = T(0.5) * (lb - la) - len + cr * ilen * phi;
                    for (int c = 0; c < 3; ++c) acc[j][c] += il * ssg[c][s] + phi * smg[c][s];
                }
            }
        }
    }
    // butterfly over the lanes (fixed order)
#pragma unroll
    for (int j = 0; j < kPer; ++j)
        for (int c = 0; c < 3; ++c)
            for (int off = 16; off > 0; off >>= 1) acc[j][c] += __shfl_xor_sync(0xffffffffu, acc[j][c], off);
    // far field by lane 0 of each warp
    if (lane != 0) return;
    const int P1 = a.P1;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        if (warp + kWarps * j >= nt) break;
        const int ti = t0 + warp + kWarps * j;
        T e0 = 0, e1 = 0, e2 = 0;
        {
            const T iw = a.iw[leaf];
            C z = passes::mk<T>(qx[j] * iw, qy[j] * iw);
            const C *Lc = a.L + (size_t)leaf * 3 * P1;
            C s0 = Lc[P1 - 1], s1 = Lc[2 * P1 - 1], s2 = Lc[3 * P1 - 1];
            for (int k = P1 - 2; k >= 0; --k) {
                s0 = passes::cadd(passes::cmul(s0, z), Lc[k]);
                s1 = passes::cadd(passes::cmul(s1, z), Lc[P1 + k]);
                s2 = passes::cadd(passes::cmul(s2, z), Lc[2 * P1 + k]);
            }
            e0 = s0.x;
            e1 = s1.x;
            e2 = s2.x;
        }
        for (int e = a.w_ptr[leaf]; e < a.w_ptr[leaf + 1]; ++e) {
            const int src = a.w_idx[e];
            const T iws = a.iw[src];
            const T zx = (T)(a.q64[2 * ti] - a.cc64[2 * src]) * iws;
            const T zy = (T)(a.q64[2 * ti + 1] - a.cc64[2 * src + 1]) * iws;
            const C iz = passes::cinv(passes::mk<T>(zx, zy));
            const T lz = T(0.5) * elog(zx * zx + zy * zy) + a.logw[src];
            const C *Ms = a.M + (size_t)src * 3 * P1;
            C m0 = passes::cscl(Ms[P1 - 1], T(1) / (P1 - 1));
            C m1 = passes::cscl(Ms[2 * P1 - 1], T(1) / (P1 - 1));
            C m2 = passes::cscl(Ms[3 * P1 - 1], T(1) / (P1 - 1));
            for (int k = P1 - 2; k >= 1; --k) {
                const T ik = T(1) / k;
                m0 = passes::cadd(passes::cmul(m0, iz), passes::cscl(Ms[k], ik));
                m1 = passes::cadd(passes::cmul(m1, iz), passes::cscl(Ms[P1 + k], ik));
                m2 = passes::cadd(passes::cmul(m2, iz), passes::cscl(Ms[2 * P1 + k], ik));
            }
            m0 = passes::cmul(m0, iz);
            m1 = passes::cmul(m1, iz);
            m2 = passes::cmul(m2, iz);
            e0 += m0.x - lz * Ms[0].x;
            e1 += m1.x - lz * Ms[P1].x;
            e2 += m2.x - lz * Ms[2 * P1].x;
        }
        const int o = a.perm[ti];
        a.out[3 * (size_t)o + 0] = (double)(acc[j][0] + e0 * k2pi);
        a.out[3 * (size_t)o + 1] = (double)(acc[j][1] + e1 * k2pi);
        a.out[3 * (size_t)o + 2] = (double)(acc[j][2] + e2 * k2pi);
    }
}

}  // namespace evalnodes
}  // namespace dc
