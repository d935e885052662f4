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
    const int4 *items;             // (leaf, first target, count, list-1 pieces)
    const double *q64;             // [n][2] sorted targets
    const int *own1, *own2, *perm; // own segments (may be null), output order
    const int *uf_ptr, *uf_seg;    // segments of each leaf's list-1 pieces, flattened
    int P1;
    const typename passes::V2<T>::type *M, *L;
    const T *sb, *mb;
    int use_s, use_m;
    double *out;                   // [n][3] in the original order
};

__device__ __forceinline__ float elog(float x) { return __logf(x); }
__device__ __forceinline__ double elog(double x) { return log(x); }

// Far field into the lane sums: every target's L2P (Eq. 64) on lane 0, its
// list-3 M2P terms (Eq. 61) split over the lanes, so a target's result does
// not depend on its slot in the work item (the order of points within a
// leaf may vary).  qx, qy: targets relative to the leaf centre.
constexpr int kPer = kNodeItem / kWarps;   // targets per warp

template <typename T>
__device__ __forceinline__ void far_into(const NodeArgs<T> &a, int leaf, int t0, int nt, int warp, int lane,
                                         const T (&qx)[kPer], const T (&qy)[kPer], T (&acc)[kPer][3]) {
    using C = typename passes::V2<T>::type;
    const T k2pi = T(0.15915494309189533577);
    const int P1 = a.P1;
    const T iwl = a.iw[leaf];
    const C *Lc = a.L + (size_t)leaf * 3 * P1;
    const int w0 = a.w_ptr[leaf], w1 = a.w_ptr[leaf + 1];
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        if (warp + kWarps * j >= nt) break;
        const int ti = t0 + warp + kWarps * j;
        T e0 = 0, e1 = 0, e2 = 0;
        if (lane == 0) {
            C z = passes::mk<T>(qx[j] * iwl, qy[j] * iwl);
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
        if (w0 + lane < w1) {
            const double tx = a.q64[2 * ti], ty = a.q64[2 * ti + 1];
            for (int e = w0 + lane; e < w1; e += 32) {
                const int src = a.w_idx[e];
                const T iws = a.iw[src];
                const T zx = (T)(tx - a.cc64[2 * src]) * iws;
                const T zy = (T)(ty - a.cc64[2 * src + 1]) * iws;
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
        }
        acc[j][0] += e0 * k2pi;
        acc[j][1] += e1 * k2pi;
        acc[j][2] += e2 * k2pi;
    }
}

// Fixed butterfly over the lanes, then lane 0 writes its targets.
template <typename T>
__device__ __forceinline__ void reduce_write(const NodeArgs<T> &a, int t0, int nt, int warp, int lane,
                                             T (&acc)[kPer][3]) {
#pragma unroll
    for (int j = 0; j < kPer; ++j)
        for (int c = 0; c < 3; ++c)
            for (int off = 16; off > 0; off >>= 1) acc[j][c] += __shfl_xor_sync(0xffffffffu, acc[j][c], off);
    if (lane != 0) return;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        if (warp + kWarps * j >= nt) break;
        const size_t o = 3 * (size_t)a.perm[t0 + warp + kWarps * j];
        a.out[o + 0] = (double)acc[j][0];
        a.out[o + 1] = (double)acc[j][1];
        a.out[o + 2] = (double)acc[j][2];
    }
}

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
    far_into<T>(a, leaf, t0, nt, warp, lane, qx, qy, acc);
    reduce_write<T>(a, t0, nt, warp, lane, acc);
}

// ------------------------------------------------- near-field operator --
// The list-1 (near-field) part of the node operator is the same linear map at
// every GMRES iteration, so its coefficients are formed once per drawing, in
// FP64, and kept resident: for work item it (targets of one leaf), target tl
// of the item and the pl-th piece of the leaf's list 1 (in list order),
//   cg[off[it] + tl nU + pl] = -(w_p / 2 pi) int_piece log|p - q| dS
//   cf[off[it] + tl nU + pl] = -(w_p / 2 pi) phi(q, piece)
// with nU = items[it].w pieces in the list; a node's own segment has phi = 0
// (Eq. 53) and the log integral of the same antiderivative (Eq. 52).  One
// application is then a gather-multiply-add over the coefficients, which
// stream from HBM once per matvec (no transcendental functions).
static __global__ void __launch_bounds__(32 * kWarps) near_coef_kernel(NodeArgs<double> a,
                                                                 const long long *__restrict__ off,
                                                                 double *__restrict__ cg,
                                                                 double *__restrict__ cf) {
    __shared__ double sx1[kStageN], sy1[kStageN], sx2[kStageN], sy2[kStageN], swg[kStageN];
    __shared__ int sseg[kStageN];
    const int4 it = a.items[blockIdx.x];
    const int leaf = it.x, t0 = it.y, nt = it.z, nU = it.w;
    const long long base = off[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double cx = a.cc64[2 * leaf], cy = a.cc64[2 * leaf + 1];
    double qx[kPer], qy[kPer];
    int o1[kPer], o2[kPer];
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        int ti = t0 + warp + kWarps * j;
        bool ok = (warp + kWarps * j) < nt;
        qx[j] = ok ? a.q64[2 * ti] - cx : 0.0;
        qy[j] = ok ? a.q64[2 * ti + 1] - cy : 0.0;
        o1[j] = (ok && a.own1) ? a.own1[ti] : -1;
        o2[j] = (ok && a.own2) ? a.own2[ti] : -1;
    }
    const double k2pi = 0.15915494309189533577;
    int pl0 = 0;
    for (int e = a.u_ptr[leaf]; e < a.u_ptr[leaf + 1]; ++e) {
        const int src = a.u_idx[e];
        const int p0 = a.pstart[src], pn = a.pcount[src];
        for (int b = 0; b < pn; b += kStageN) {
            const int cnt = min(kStageN, pn - b);
            __syncthreads();
            for (int s = threadIdx.x; s < cnt; s += blockDim.x) {
                const int i = p0 + b + s;
                const double *P = a.pc64 + 4 * (size_t)i;
                sx1[s] = P[0] - cx;
                sy1[s] = P[1] - cy;
                sx2[s] = P[2] - cx;
                sy2[s] = P[3] - cy;
                swg[s] = -a.pw[i] * k2pi;
                sseg[s] = a.pseg[i];
            }
            __syncthreads();
            for (int s = lane; s < cnt; s += 32) {
                const double x1 = sx1[s], y1 = sy1[s], x2 = sx2[s], y2 = sy2[s];
                const double dx = x2 - x1, dy = y2 - y1;
                const double len = sqrt(dx * dx + dy * dy), ilen = 1.0 / len;
                const int seg = sseg[s];
                const double wg = swg[s];
#pragma unroll
                for (int j = 0; j < kPer; ++j) {
                    const int tl = warp + kWarps * j;
                    if (tl >= nt) break;
                    const double ax = x1 - qx[j], ay = y1 - qy[j], bx = x2 - qx[j], by = y2 - qy[j];
                    const double cr = ax * by - ay * bx, dt = ax * bx + ay * by;
                    const bool own = (seg == o1[j]) || (seg == o2[j]);
                    const double phi = own ? 0.0 : atan2(cr, dt);
                    const double ra2 = ax * ax + ay * ay, rb2 = bx * bx + by * by;
                    const double s1 = (ax * dx + ay * dy) * ilen, s2 = s1 + len;
                    const double la = ra2 > 0.0 ? s1 * log(ra2) : 0.0;
                    const double lb = rb2 > 0.0 ? s2 * log(rb2) : 0.0;
                    const double il = 0.5 * (lb - la) - len + cr * ilen * phi;
                    const long long idx = base + (long long)tl * nU + pl0 + s;
                    cg[idx] = il * wg;
                    cf[idx] = phi * wg;
                }
            }
            pl0 += cnt;
        }
    }
}

// Far-field coefficients of the node targets, formed once per drawing in FP64:
// the L2P (Eq. 64) and list-3 M2P (Eq. 61) sums are linear in the expansion
// coefficients, u += Re sum_k a_k X_k with
//   block 0 (the leaf's L):      a_k = z^k / 2pi,       z = (q - c_leaf) / w_leaf
//   block b (list-3 source b-1): a_0 = -(log|z| + log w_src) / 2pi (times Re M_0),
//                                a_k = z^-k / (2pi k),  z = (q - c_src) / w_src
// stored per target as (1 + nW) blocks of P1 complex values from block
// off[item] + tl (1 + nW); nW = the leaf's list-3 length.
static __global__ void __launch_bounds__(32 * kWarps) far_coef_kernel(NodeArgs<double> a,
                                                                      const long long *__restrict__ off,
                                                                      double2 *__restrict__ cf) {
    const int4 it = a.items[blockIdx.x];
    const int leaf = it.x, t0 = it.y, nt = it.z;
    const int P1 = a.P1;
    const int w0 = a.w_ptr[leaf], nW = a.w_ptr[leaf + 1] - w0;
    const int nb = 1 + nW;
    const long long base = off[blockIdx.x] * P1;
    const double k2pi = 0.15915494309189533577;
    for (int u = threadIdx.x; u < nt * nb; u += blockDim.x) {
        const int tl = u / nb, b = u - tl * nb;
        const int ti = t0 + tl;
        double2 *row = cf + base + ((long long)tl * nb + b) * P1;
        const double qx = a.q64[2 * ti], qy = a.q64[2 * ti + 1];
        if (b == 0) {
            const double iw = a.iw[leaf];
            const double zx = (qx - a.cc64[2 * leaf]) * iw, zy = (qy - a.cc64[2 * leaf + 1]) * iw;
            double px = k2pi, py = 0.0;
            for (int k = 0; k < P1; ++k) {
                row[k] = make_double2(px, py);
                const double nx = px * zx - py * zy;
                py = px * zy + py * zx;
                px = nx;
            }
        } else {
            const int src = a.w_idx[w0 + b - 1];
            const double iws = a.iw[src];
            const double zx = (qx - a.cc64[2 * src]) * iws, zy = (qy - a.cc64[2 * src + 1]) * iws;
            const double r2 = zx * zx + zy * zy;
            const double ix = zx / r2, iy = -zy / r2;          // 1 / z
            row[0] = make_double2(-k2pi * (0.5 * log(r2) + a.logw[src]), 0.0);
            double px = ix, py = iy;                             // z^-k
            for (int k = 1; k < P1; ++k) {
                row[k] = make_double2(k2pi * px / k, k2pi * py / k);
                const double nx = px * ix - py * iy;
                py = px * iy + py * ix;
                px = nx;
            }
        }
    }
}

// Far field from stored coefficients into the lane sums: lanes split the
// (block, k) terms; in FP32 each term's three expansion coefficients are
// loaded once and applied to all of the warp's targets.
template <typename T>
__device__ __forceinline__ void far_rows_into(const NodeArgs<T> &a, const typename passes::V2<T>::type *__restrict__ cf,
                                              long long base, int leaf, int nt, int warp, int lane,
                                              T (&acc)[kPer][3]) {
    using C = typename passes::V2<T>::type;
    const int P1 = a.P1;
    const int w0 = a.w_ptr[leaf], nb = 1 + a.w_ptr[leaf + 1] - w0;
    const int nterm = nb * P1;
    const C *rows = cf + base;
    if (sizeof(T) == 8) {   // FP64: one target at a time (fewer registers)
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int tl = warp + kWarps * j;
            if (tl >= nt) break;
            const C *row = rows + (long long)tl * nterm;
            for (int u = lane; u < nterm; u += 32) {
                const int b = u / P1, k = u - b * P1;
                const int src = b == 0 ? leaf : a.w_idx[w0 + b - 1];
                const C *X = (b == 0 ? a.L : a.M) + (size_t)src * 3 * P1 + k;
                const C co = row[u];
                const C x0 = X[0], x1 = X[P1], x2 = X[2 * P1];
                acc[j][0] += co.x * x0.x - co.y * x0.y;
                acc[j][1] += co.x * x1.x - co.y * x1.y;
                acc[j][2] += co.x * x2.x - co.y * x2.y;
            }
        }
        return;
    }
#pragma unroll 2
    for (int u = lane; u < nterm; u += 32) {
        const int b = u / P1, k = u - b * P1;
        const int src = b == 0 ? leaf : a.w_idx[w0 + b - 1];
        const C *X = (b == 0 ? a.L : a.M) + (size_t)src * 3 * P1 + k;
        C co[kPer];
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int tl = warp + kWarps * j;
            co[j] = tl < nt ? rows[(long long)tl * nterm + u] : C{T(0), T(0)};
        }
        const C x0 = X[0], x1 = X[P1], x2 = X[2 * P1];
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            acc[j][0] += co[j].x * x0.x - co[j].y * x0.y;
            acc[j][1] += co[j].x * x1.x - co[j].y * x1.y;
            acc[j][2] += co[j].x * x2.x - co[j].y * x2.y;
        }
    }
}

// Node operator with the near field from stored coefficients (near_coef_kernel
// layout): y = sum_pl coef * dens[seg(pl)] + far field (L2P, list-3 M2P),
// the far field from stored coefficients too when far != nullptr.  Lanes
// walk the leaf's list-1 pieces four at a time (FP32; one at a time in
// FP64, whose registers allow no more), issuing every load of a batch
// (segment numbers, coefficients, then densities) before the first
// multiply-add, so that a warp keeps several requests in flight.
template <typename T> struct NearBatch { static constexpr int value = 4; };

template <typename T>
__global__ void __launch_bounds__(32 * kWarps, sizeof(T) == 4 ? 8 : 4) near_apply_kernel(NodeArgs<T> a, const long long *__restrict__ off,
                                                                  const T *__restrict__ coef,
                                                                  const T *__restrict__ dens,
                                                                  const long long *__restrict__ far_off = nullptr,
                                                                  const typename passes::V2<T>::type *__restrict__ far = nullptr) {
    const int4 it = a.items[blockIdx.x];
    const int leaf = it.x, t0 = it.y, nt = it.z, nU = it.w;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T acc[kPer][3];
#pragma unroll
    for (int j = 0; j < kPer; ++j) acc[j][0] = acc[j][1] = acc[j][2] = T(0);
    if (warp < nt && sizeof(T) == 8) {   // FP64: one piece at a time per lane
        const T *rows = coef + off[blockIdx.x];
        const int *segs = a.uf_seg + a.uf_ptr[leaf];
        for (int pl = lane; pl < nU; pl += 32) {
            const size_t o = 3 * (size_t)segs[pl];
            const T d0 = dens[o], d1 = dens[o + 1], d2 = dens[o + 2];
#pragma unroll
            for (int j = 0; j < kPer; ++j) {
                const int tl = warp + kWarps * j;
                if (tl >= nt) break;
                const T cfv = rows[(long long)tl * nU + pl];
                acc[j][0] += cfv * d0;
                acc[j][1] += cfv * d1;
                acc[j][2] += cfv * d2;
            }
        }
    } else if (warp < nt) {
        const T *rows = coef + off[blockIdx.x];
        const int *segs = a.uf_seg + a.uf_ptr[leaf];
        constexpr int kB = NearBatch<T>::value;
        for (int p0 = 0; p0 < nU; p0 += 32 * kB) {
            int sg[kB];
            T cv[kB][kPer];
#pragma unroll
            for (int i = 0; i < kB; ++i) {
                const int pl = p0 + lane + 32 * i;
                sg[i] = pl < nU ? segs[pl] : -1;
#pragma unroll
                for (int j = 0; j < kPer; ++j) {
                    const int tl = warp + kWarps * j;
                    cv[i][j] = (pl < nU && tl < nt) ? rows[(long long)tl * nU + pl] : T(0);
                }
            }
            T d[kB][3];
#pragma unroll
            for (int i = 0; i < kB; ++i) {
                const bool ok = sg[i] >= 0;
                const size_t o = 3 * (size_t)(ok ? sg[i] : 0);
                d[i][0] = ok ? dens[o] : T(0);
                d[i][1] = ok ? dens[o + 1] : T(0);
                d[i][2] = ok ? dens[o + 2] : T(0);
            }
#pragma unroll
            for (int i = 0; i < kB; ++i)
#pragma unroll
                for (int j = 0; j < kPer; ++j) {
                    acc[j][0] += cv[i][j] * d[i][0];
                    acc[j][1] += cv[i][j] * d[i][1];
                    acc[j][2] += cv[i][j] * d[i][2];
                }
        }
    }
    if (far) {
        far_rows_into<T>(a, far, far_off[blockIdx.x] * a.P1, leaf, nt, warp, lane, acc);
    } else {
        const double cx = a.cc64[2 * leaf], cy = a.cc64[2 * leaf + 1];
        T qx[kPer], qy[kPer];
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int tl = warp + kWarps * j;
            const int ti = t0 + (tl < nt ? tl : 0);
            qx[j] = tl < nt ? (T)(a.q64[2 * ti] - cx) : T(0);
            qy[j] = tl < nt ? (T)(a.q64[2 * ti + 1] - cy) : T(0);
        }
        far_into<T>(a, leaf, t0, nt, warp, lane, qx, qy, acc);
    }
    reduce_write<T>(a, t0, nt, warp, lane, acc);
}

// The FP64 node operator from stored coefficients with float-float
// arithmetic on the FP32 pipes: near-field coefficients (hi, lo) per
// (node, piece), segment densities (hi, lo) per channel, far-field
// coefficients and the L / M expansions as float-float complex values
// (float4: re hi, im hi, re lo, im lo).  Same work split as
// near_apply_kernel; lane sums are combined by a fixed butterfly with exact
// two-sums; the result is written in FP64.
static __device__ __forceinline__ void ffa_fma(float2 &acc, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    const float e = fmaf(ah, bh, -p);
    const float sum = __fadd_rn(acc.x, p);
    const float bb = __fsub_rn(sum, acc.x);
    const float q = __fadd_rn(__fsub_rn(acc.x, __fsub_rn(sum, bb)), __fsub_rn(p, bb));
    acc.x = sum;
    acc.y += q + e + fmaf(ah, bl, al * bh);
}

static __global__ void __launch_bounds__(32 * kWarps) near_apply_ff_kernel(NodeArgs<double> a, const long long *__restrict__ off,
                                                                     const float2 *__restrict__ coef,
                                                                     const float2 *__restrict__ dens,
                                                                     const long long *__restrict__ far_off,
                                                                     const float4 *__restrict__ far,
                                                                     const float4 *__restrict__ Lff,
                                                                     const float4 *__restrict__ Mff) {
    const int4 it = a.items[blockIdx.x];
    const int leaf = it.x, t0 = it.y, nt = it.z, nU = it.w;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2 acc[kPer][3];
#pragma unroll
    for (int j = 0; j < kPer; ++j) acc[j][0] = acc[j][1] = acc[j][2] = make_float2(0.f, 0.f);
    if (warp < nt) {
        const float2 *rows = coef + off[blockIdx.x];
        const int *segs = a.uf_seg + a.uf_ptr[leaf];
        for (int pl = lane; pl < nU; pl += 32) {
            const size_t o = 3 * (size_t)segs[pl];
            const float2 d0 = dens[o], d1 = dens[o + 1], d2 = dens[o + 2];
#pragma unroll
            for (int j = 0; j < kPer; ++j) {
                const int tl = warp + kWarps * j;
                if (tl >= nt) break;
                const float2 cf = rows[(long long)tl * nU + pl];
                ffa_fma(acc[j][0], cf.x, cf.y, d0.x, d0.y);
                ffa_fma(acc[j][1], cf.x, cf.y, d1.x, d1.y);
                ffa_fma(acc[j][2], cf.x, cf.y, d2.x, d2.y);
            }
        }
    }
    {   // far field: Re(co x) = co.re x.re - co.im x.im
        const int P1 = a.P1;
        const int w0 = a.w_ptr[leaf], nb = 1 + a.w_ptr[leaf + 1] - w0;
        const int nterm = nb * P1;
        const float4 *rows = far + far_off[blockIdx.x] * P1;
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int tl = warp + kWarps * j;
            if (tl >= nt) break;
            const float4 *row = rows + (long long)tl * nterm;
            for (int u = lane; u < nterm; u += 32) {
                const int b = u / P1, k = u - b * P1;
                const int src = b == 0 ? leaf : a.w_idx[w0 + b - 1];
                const float4 *X = (b == 0 ? Lff : Mff) + (size_t)src * 3 * P1 + k;
                const float4 co = row[u];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float4 x = X[c * P1];
                    ffa_fma(acc[j][c], co.x, co.z, x.x, x.z);
                    ffa_fma(acc[j][c], -co.y, -co.w, x.y, x.w);
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < kPer; ++j)
        for (int c = 0; c < 3; ++c)
            for (int o = 16; o > 0; o >>= 1) {
                const float h2 = __shfl_xor_sync(0xffffffffu, acc[j][c].x, o);
                const float l2 = __shfl_xor_sync(0xffffffffu, acc[j][c].y, o);
                const float sum = __fadd_rn(acc[j][c].x, h2);
                const float bb = __fsub_rn(sum, acc[j][c].x);
                const float q = __fadd_rn(__fsub_rn(acc[j][c].x, __fsub_rn(sum, bb)), __fsub_rn(h2, bb));
                acc[j][c].x = sum;
                acc[j][c].y += l2 + q;
            }
    if (lane != 0) return;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        if (warp + kWarps * j >= nt) break;
        const size_t o = 3 * (size_t)a.perm[t0 + warp + kWarps * j];
        for (int c = 0; c < 3; ++c) a.out[o + c] = (double)acc[j][c].x + (double)acc[j][c].y;
    }
}

}  // namespace evalnodes
}  // namespace dc
