// FP32 ("chosen") form of the FMM of App. E / Alg. 8.
//
// Same passes and scaled expansions as the FP64 form (see fmm.cu), with
// every coordinate held relative to a cell centre so FP32 keeps the local
// relative accuracy: pieces relative to their own leaf, targets relative to
// their leaf, and per-list-entry centre offsets for list 1, 3 and 4.  The
// near field (list 1, closed forms of App. D) stages the pieces of each
// adjacent leaf in shared memory, shifted into the target leaf's frame, with
// the densities pre-multiplied by -w/(2 pi); all targets of a tile sweep the
// staged pieces together.  A pair whose target lies within 1e-4 chord
// lengths of the segment's interior (where the sign of the subtended angle
// decides which side of the curve the pixel is on) is recomputed in FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "evalnodes.cuh"
#include "ffarith.cuh"
#include "passes_tc.cuh"
#include "fmm_impl.h"
#include "segint.cuh"

namespace dc {

namespace {

constexpr float kInv2PiF = 0.15915494309189533577f;
constexpr float kNearFallback = 1e-4f;

__device__ __forceinline__ float2 fmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 fadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 fscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 finv(float2 a) {
    float d = 1.0f / (a.x * a.x + a.y * a.y);
    return make_float2(a.x * d, -a.y * d);
}
__device__ __forceinline__ void ffma2(float2 &acc, float2 m, float2 v) {
    acc.x = fmaf(m.x, v.x, fmaf(-m.y, v.y, acc.x));
    acc.y = fmaf(m.x, v.y, fmaf(m.y, v.x, acc.y));
}
// log(b / a) for a, b away from the origin, with the real part from log1p
// of (|b|^2 - |a|^2) / |a|^2 computed from b - a (no cancellation).
__device__ __forceinline__ float2 flog_ratio(float2 a, float2 b) {
    float2 d = make_float2(b.x - a.x, b.y - a.y), s = make_float2(b.x + a.x, b.y + a.y);
    float num = d.x * s.x + d.y * s.y;            // |b|^2 - |a|^2
    float aa = a.x * a.x + a.y * a.y;
    return make_float2(0.5f * log1pf(num / aa), atan2f(a.x * b.y - a.y * b.x, a.x * b.x + a.y * b.y));
}

// ------------------------------------------------------------ interp --
__global__ void d2f_kernel(const double *__restrict__ a, const double *__restrict__ b,
                           float *__restrict__ fa, float *__restrict__ fb, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        fa[i] = (float)a[i];
        fb[i] = (float)b[i];
    }
}

// sigma_bar = Lambda sigma per panel in float-float (the FP64 node values
// converted once per panel into shared memory; Lambda stored as hi/lo
// floats), rounded to FP32 at the end: one block per panel, one thread per
// segment.  The node values can be large and cancelling (the coarse part of
// the preconditioned vector), so the sums keep more than FP32 accuracy.
__global__ void interp32_kernel(const float2 *__restrict__ lam, const double *__restrict__ nv,
                                float *__restrict__ sv, int s, int g) {
    __shared__ float2 v[3 * kMaxG];
    const int panel = blockIdx.x, kk = threadIdx.x;
    const double *src = nv + (size_t)panel * g * 3;
    for (int i = kk; i < 3 * g; i += blockDim.x) {
        const double x = src[i];
        const float h = (float)x;
        v[i] = make_float2(h, (float)(x - (double)h));
    }
    __syncthreads();
    for (int q = kk; q < s; q += blockDim.x) {
        const float2 *row = lam + (size_t)q * g;
        float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f, h2 = 0.f, l2 = 0.f;
        for (int m = 0; m < g; ++m) {
            const float2 l = row[m];
            dot2ff(h0, l0, l, v[3 * m]);
            dot2ff(h1, l1, l, v[3 * m + 1]);
            dot2ff(h2, l2, l, v[3 * m + 2]);
        }
        const size_t k = (size_t)panel * s + q;
        sv[3 * k + 0] = h0 + l0;
        sv[3 * k + 1] = h1 + l1;
        sv[3 * k + 2] = h2 + l2;
    }
}

// ---------------------------------------------- render preparation --
// Cells whose expansions carry large, cancelling coefficients (next to
// strongly singular densities) are evaluated in FP64: the FP32 rounding of
// a coefficient is ~6e-8 of its size.  hL: sum_l |Lt_l| > kBigCoef; hM:
// 10 |Mt_0| + sum_k |Mt_k| > kBigCoef (max over channels).
#ifndef DC_BIG_COEF
#define DC_BIG_COEF 50.0
#endif
constexpr double kBigCoef = DC_BIG_COEF;
__global__ void big_coef_kernel(const double2 *__restrict__ L, const double2 *__restrict__ M, int n,
                                int P1, unsigned char *__restrict__ hL, unsigned char *__restrict__ hM) {
    // one warp per cell, lanes over the coefficients (coalesced); magnitudes in FP32, since this
    // is a threshold test and FP64 hypot runs at 1/64 of the FP32 rate
    const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (c >= n) return;
    float bl = 0.f, bm = 0.f;
    for (int ch = 0; ch < 3; ++ch) {
        const double2 *l = L + ((size_t)c * 3 + ch) * P1, *m = M + ((size_t)c * 3 + ch) * P1;
        float sl = 0.f, sm = 0.f;
        for (int k = lane; k < P1; k += 32) {
            const double2 lk = l[k], mk = m[k];
            sl += hypotf((float)lk.x, (float)lk.y);
            sm += (k == 0 ? 10.f : 1.f) * hypotf((float)mk.x, (float)mk.y);
        }
        for (int o = 16; o > 0; o >>= 1) {
            sl += __shfl_xor_sync(0xffffffffu, sl, o);
            sm += __shfl_xor_sync(0xffffffffu, sm, o);
        }
        bl = fmaxf(bl, sl);
        bm = fmaxf(bm, sm);
    }
    if (lane == 0) {
        hL[c] = bl > kBigCoef;
        hM[c] = bm > kBigCoef;
    }
}

// The near field of the pixel kernel works in each leaf's frame scaled by
// 1 / rho (rho the leaf width, a power of two); this adds the part
// it leaves out to the leaf's local coefficient L_0 in FP64:
//   L_0 += 2 pi log(rho) sum_i ssg_i rho len'_i,
// i over the leaf's list-1 pieces that are not heavy, with the pixel
// kernel's own FP32 values ssg_i = (-w_i / 2 pi) sigma_bar_c and len'_i =
// len_i / rho, so that the centred sums plus L_0 equal the plain sums.  The
// large log(rho) terms meet the far field's constant here, in FP64, instead
// of in the FP32 near-field sums.  One warp per cell, a fixed order.
__global__ void near_centre_kernel(const int *__restrict__ uf_ptr, const int *__restrict__ uf_idx,
                                   const int *__restrict__ pseg, const float *__restrict__ pw,
                                   const float *__restrict__ plen, const unsigned char *__restrict__ heavy,
                                   const float *__restrict__ sb, const float *__restrict__ iw, int nC, int P1,
                                   double2 *__restrict__ L) {
    const int cell = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (cell >= nC || uf_ptr[cell + 1] == uf_ptr[cell]) return;
    const float iwf = iw[cell];
    double acc[3] = {0.0, 0.0, 0.0};
    for (int f = uf_ptr[cell] + lane; f < uf_ptr[cell + 1]; f += 32) {
        const int i = uf_idx[f];
        if (heavy && heavy[i]) continue;
        const int seg = pseg[i];
        const float wgt = -pw[i] * 0.15915494309189533577f;
        const double lenp = (double)(plen[i] * iwf);
        for (int ch = 0; ch < 3; ++ch) acc[ch] += (double)(wgt * sb[3 * (size_t)seg + ch]) * lenp;
    }
    for (int o = 16; o > 0; o >>= 1)
        for (int ch = 0; ch < 3; ++ch) acc[ch] += __shfl_xor_sync(0xffffffffu, acc[ch], o);
    if (lane == 0) {
        const double iwd = (double)iwf;
        const double k = -6.283185307179586477 * log(iwd) / iwd;   // 2 pi rho log(rho)
        for (int ch = 0; ch < 3; ++ch) L[((size_t)cell * 3 + ch) * P1].x += k * acc[ch];
    }
}

template <typename From, typename To>
__global__ void narrow_kernel(const From *__restrict__ a, To *__restrict__ b, size_t n) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        b[i].x = (float)a[i].x;
        b[i].y = (float)a[i].y;
    }
}

// heavy[i] = 1 when max_c |sigma_bar| w len or |mu_bar| w len of piece i
// exceeds kHeavy: its near-field terms are then summed in FP64.
#ifndef DC_HEAVY
#define DC_HEAVY 1.0
#endif
constexpr double kHeavy = DC_HEAVY;
__global__ void heavy_kernel(const double *__restrict__ sb, const double *__restrict__ mb,
                             const int *__restrict__ pseg, const double *__restrict__ pw,
                             const double *__restrict__ plen, unsigned char *__restrict__ heavy, int np) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    int s = pseg[i];
    double m = 0.0;
    for (int c = 0; c < 3; ++c) m = fmax(m, fmax(fabs(sb[3 * (size_t)s + c]), fabs(mb[3 * (size_t)s + c])));
    heavy[i] = (m * pw[i] * plen[i] > kHeavy) ? 1 : 0;
}

// -------------------------------------------------------------- eval --
// The pixel tile of one block is TW x TH pixels (options.eval_tile picks
// the shape); every shape is compiled for the same resident threads per SM
// (kEvThreadsPerSM), so the register budget does not depend on the shape.
// resident blocks per SM of 64-thread tiles the register budget is set for,
// and pieces staged in shared memory per round
#ifndef DC_EVAL_MINBLOCKS
#define DC_EVAL_MINBLOCKS 12
#endif
#ifndef DC_EVAL_STAGE
#define DC_EVAL_STAGE 128
#endif
constexpr int kEvBlocksPerSM = DC_EVAL_MINBLOCKS;
constexpr int kEvThreadsPerSM = 64 * kEvBlocksPerSM;

constexpr int kStage = DC_EVAL_STAGE;

struct EvalArgs32 {
    DevTree32 t;
    DevTree t64;
    const Tile *items;
    int P1;
    const float2 *M, *L;
    const float *sb, *mb;
    int use_s, use_m;
    // pixel mode
    const VpDev *vps;
    void *rgb;
    int rgb_dtype;
    unsigned char *rgb8;
    // FP64 path for heavy pieces and big-coefficient cells (pixel mode)
    const double *sb64, *mb64;
    const unsigned char *heavy, *hL, *hM;
    const double2 *M64, *L64;

    // persistent launch: the item counter (zero at launch) and the item count
    int *queue;
    int n_items;
    // list mode
    const float2 *q32;
    const double *q64;
    const int *own1, *own2, *perm;
    double *out;
};

__device__ __forceinline__ unsigned char quant8(float v) {
    v = fminf(fmaxf(v, 0.f), 1.f);
    return (unsigned char)floorf(255.f * v + 0.5f);
}

// (hi, lo) of (ah + al) - (bh + bl) from float pairs on the FP32 pipe: the
// difference of the hi parts exactly (two-sum, Knuth), the lo parts added
// to its error; accurate to about 2^-48 of the operands, like split2 of the
// FP64 difference, without FP64 instructions.
__device__ __forceinline__ void diff2(float ah, float al, float bh, float bl, float &hi, float &lo) {
    const float s = __fsub_rn(ah, bh);
    const float bb = __fsub_rn(s, ah);
    const float e = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bb)), __fsub_rn(-bh, bb));
    hi = s;
    lo = __fadd_rn(e, __fsub_rn(al, bl));
}

// float pair (hi, lo) with hi + lo = v to about 2^-48 relative
__device__ __forceinline__ void split2(double v, float &hi, float &lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

template <int MODE, int TW, int TH>
__device__ __forceinline__ void eval32_item(const EvalArgs32 &a, int item) {
    // staged pieces of one list-1 leaf, in the target leaf's frame, each
    // coordinate as a (hi, lo) float pair so differences keep full accuracy
    __shared__ float sx1h[kStage], sx1l[kStage], sy1h[kStage], sy1l[kStage];
    __shared__ float sx2h[kStage], sx2l[kStage], sy2h[kStage], sy2l[kStage];
    __shared__ float slen[kStage];
    __shared__ float ssg[3][kStage], smg[3][kStage];
    __shared__ int sseg[kStage], sidx[kStage];
    __shared__ unsigned char shv[kStage];
    const DevTree32 &t = a.t;
    Tile tl = a.items[item];
    const int leaf = tl.leaf;
    double h0 = 0.0, h1 = 0.0, h2 = 0.0;   // FP64 sums of heavy pieces
    const double cxB = a.t64.cc[2 * leaf], cyB = a.t64.cc[2 * leaf + 1];
    const int j = threadIdx.x;
    bool act;
    double qx64 = 0.0, qy64 = 0.0;
    int own1 = -1, own2 = -1, r = 0, c = 0, ti = 0;
    VpDev vp;
    if (MODE == 0) {
        vp = a.vps[tl.vp];
        act = j < tl.nr * tl.nc;
        if (act) {
            r = tl.r0 + j / tl.nc;
            c = tl.c0 + j % tl.nc;
            qx64 = vp.x0 + (c + 0.5) * vp.dx;
            qy64 = vp.y0 + (r + 0.5) * vp.dy;
        }
    } else {
        act = j < tl.nr;
        if (act) {
            ti = tl.r0 + j;
            qx64 = a.q64[2 * ti];
            qy64 = a.q64[2 * ti + 1];
            if (a.own1) {
                own1 = a.own1[ti];
                own2 = a.own2[ti];
            }
        }
    }
    float qxh, qxl, qyh, qyl;
    split2(qx64 - cxB, qxh, qxl);
    split2(qy64 - cyB, qyh, qyl);
    const float2 q = make_float2(qxh, qyh);
    float u0 = 0.f, u1 = 0.f, u2 = 0.f;
    const int P1 = a.P1;
    if (act) {
        // L2P (Eq. 64)
        float e0 = 0.f, e1 = 0.f, e2 = 0.f;
        if (a.hL && a.hL[leaf]) {
            const double iw = 1.0 / a.t64.cw[leaf];
            const double zx = (qx64 - cxB) * iw, zy = (qy64 - cyB) * iw;
            const double2 *Lc = a.L64 + (size_t)leaf * 3 * P1;
            for (int ch = 0; ch < 3; ++ch) {
                double sx = Lc[ch * P1 + P1 - 1].x, sy = Lc[ch * P1 + P1 - 1].y;
                for (int k = P1 - 2; k >= 0; --k) {
                    double nx = sx * zx - sy * zy + Lc[ch * P1 + k].x;
                    sy = sx * zy + sy * zx + Lc[ch * P1 + k].y;
                    sx = nx;
                }
                (ch == 0 ? h0 : ch == 1 ? h1 : h2) += sx * kInv2Pi;
            }
        } else {
            float iw = t.iw[leaf];
            float2 z = make_float2(q.x * iw, q.y * iw);
            const float2 *Lc = a.L + (size_t)leaf * 3 * P1;
            float2 s0 = Lc[P1 - 1], s1 = Lc[2 * P1 - 1], s2 = Lc[3 * P1 - 1];
            for (int k = P1 - 2; k >= 0; --k) {
                s0 = fadd(fmul(s0, z), Lc[k]);
                s1 = fadd(fmul(s1, z), Lc[P1 + k]);
                s2 = fadd(fmul(s2, z), Lc[2 * P1 + k]);
            }
            e0 = s0.x;
            e1 = s1.x;
            e2 = s2.x;
        }
        // M2P over list 3 (Eq. 61)
        for (int e = t.w_ptr[leaf]; e < t.w_ptr[leaf + 1]; ++e) {
            int src = t.w_idx[e];
            if (a.hM && a.hM[src]) {
                const double iws = 1.0 / a.t64.cw[src];
                const double zx = (qx64 - a.t64.cc[2 * src]) * iws, zy = (qy64 - a.t64.cc[2 * src + 1]) * iws;
                const double d = 1.0 / (zx * zx + zy * zy);
                const double izx = zx * d, izy = -zy * d;
                const double lz = 0.5 * log(zx * zx + zy * zy) + log(a.t64.cw[src]);
                const double2 *Ms = a.M64 + (size_t)src * 3 * P1;
                for (int ch = 0; ch < 3; ++ch) {
                    const double2 *m = Ms + ch * P1;
                    double sx = m[P1 - 1].x / (P1 - 1), sy = m[P1 - 1].y / (P1 - 1);
                    for (int k = P1 - 2; k >= 1; --k) {
                        double nx = sx * izx - sy * izy + m[k].x / k;
                        sy = sx * izy + sy * izx + m[k].y / k;
                        sx = nx;
                    }
                    double rx = sx * izx - sy * izy;
                    (ch == 0 ? h0 : ch == 1 ? h1 : h2) += (rx - lz * m[0].x) * kInv2Pi;
                }
                continue;
            }
            float2 off = t.w_off[e];
            float iws = t.iw[src];
            float2 zz = make_float2((q.x - off.x) * iws, (q.y - off.y) * iws);
            float2 iz = finv(zz);
            float lz = 0.5f * __logf(zz.x * zz.x + zz.y * zz.y) + t.logw[src];
            const float2 *Ms = a.M + (size_t)src * 3 * P1;
            float2 m0 = fscale(Ms[P1 - 1], 1.f / (P1 - 1)), m1 = fscale(Ms[2 * P1 - 1], 1.f / (P1 - 1)),
                   m2 = fscale(Ms[3 * P1 - 1], 1.f / (P1 - 1));
            for (int k = P1 - 2; k >= 1; --k) {
                float ik = 1.f / k;
                m0 = fadd(fmul(m0, iz), fscale(Ms[k], ik));
                m1 = fadd(fmul(m1, iz), fscale(Ms[P1 + k], ik));
                m2 = fadd(fmul(m2, iz), fscale(Ms[2 * P1 + k], ik));
            }
            m0 = fmul(m0, iz);
            m1 = fmul(m1, iz);
            m2 = fmul(m2, iz);
            e0 += m0.x - lz * Ms[0].x;
            e1 += m1.x - lz * Ms[P1].x;
            e2 += m2.x - lz * Ms[2 * P1].x;
        }
        // the far field goes to the FP64 sums: the FP32 near-field sums then
        // start from zero instead of from a value the near field may cancel
        h0 += (double)e0 * kInv2Pi;
        h1 += (double)e1 * kInv2Pi;
        h2 += (double)e2 * kInv2Pi;
    }
    // The near field works in the leaf's frame scaled by 1 / rho, rho the
    // leaf width: its logarithms are then log(r / rho), O(1) for the pieces
    // of list 1, so the single-layer terms (weights times rho) stay O(len)
    // and their FP32 rounding does not pile up where large densities cancel.
    // The constant rest, log(rho) times the weighted lengths, was added to
    // the leaf's local coefficient L_0 in FP64 (near_centre_kernel).
    // Quadtree widths are powers of two, so scaling a (hi, lo) pair by the
    // FP32 1 / width is exact.
    {
        const float iwq = t.iw[leaf];
        qxh *= iwq;
        qxl *= iwq;
        qyh *= iwq;
        qyl *= iwq;
    }
    // P2P over list 1 (App. D): the leaf's list-1 pieces, flattened in list
    // order, staged kStage at a time, relative to the leaf's centre
    float cxh, cxl, cyh, cyl;
    split2(cxB, cxh, cxl);
    split2(cyB, cyh, cyl);
    const int f_end = t.uf_ptr[leaf + 1];
    for (int f0 = t.uf_ptr[leaf]; f0 < f_end; f0 += kStage) {
        {
            int cnt = min(kStage, f_end - f0);
            __syncthreads();
            for (int s = threadIdx.x; s < cnt; s += blockDim.x) {
                int i = t.uf_idx[f0 + s];
                const float iwf = t.iw[leaf], rho = 1.f / iwf;   // exact powers of two
                const float4 ph = t.pch[i], pl = t.pcl[i];
                float h, l;
                diff2(ph.x, pl.x, cxh, cxl, h, l);
                sx1h[s] = h * iwf;
                sx1l[s] = l * iwf;
                diff2(ph.y, pl.y, cyh, cyl, h, l);
                sy1h[s] = h * iwf;
                sy1l[s] = l * iwf;
                diff2(ph.z, pl.z, cxh, cxl, h, l);
                sx2h[s] = h * iwf;
                sx2l[s] = l * iwf;
                diff2(ph.w, pl.w, cyh, cyl, h, l);
                sy2h[s] = h * iwf;
                sy2l[s] = l * iwf;
                slen[s] = t.plen[i] * iwf;
                int seg = t.pseg[i];
                float wgt = -t.pw[i] * kInv2PiF;
                for (int ch = 0; ch < 3; ++ch) {
                    ssg[ch][s] = a.use_s ? (wgt * a.sb[3 * (size_t)seg + ch]) * rho : 0.f;
                    smg[ch][s] = a.use_m ? wgt * a.mb[3 * (size_t)seg + ch] : 0.f;
                }
                sseg[s] = seg;
                sidx[s] = i;
                shv[s] = a.heavy ? a.heavy[i] : 0;
            }
            __syncthreads();
            if (act) {
                for (int s = 0; s < cnt; ++s) {
                    if (shv[s]) {
                        // large density: the whole term in FP64 (App. D forms)
                        const double *P = a.t64.pc + 4 * (size_t)sidx[s];
                        const int seg = sseg[s];
                        const bool own = (seg == own1) || (seg == own2);
                        double il64, ph64;
                        seg_ilog_phi_f64(qx64, qy64, P[0], P[1], P[2], P[3], own, il64, ph64);
                        const double wg = -(double)a.t64.pw[sidx[s]] * kInv2Pi;
                        h0 += wg * (il64 * a.sb64[3 * (size_t)seg + 0] + ph64 * a.mb64[3 * (size_t)seg + 0]);
                        h1 += wg * (il64 * a.sb64[3 * (size_t)seg + 1] + ph64 * a.mb64[3 * (size_t)seg + 1]);
                        h2 += wg * (il64 * a.sb64[3 * (size_t)seg + 2] + ph64 * a.mb64[3 * (size_t)seg + 2]);
                        continue;
                    }
                    float ax = (sx1h[s] - qxh) + (sx1l[s] - qxl), ay = (sy1h[s] - qyh) + (sy1l[s] - qyl);
                    float bx = (sx2h[s] - qxh) + (sx2l[s] - qxl), by = (sy2h[s] - qyh) + (sy2l[s] - qyl);
                    float len = slen[s];
                    float cr = ax * by - ay * bx;
                    float dt = ax * bx + ay * by;
                    bool own = (sseg[s] == own1) || (sseg[s] == own2);
                    float ilog, phi;
                    const float mx = 0.5f * (ax + bx), my = 0.5f * (ay + by);   // midpoint - target
                    const float r2 = mx * mx + my * my;
                    if (!own && 16.f * len * len < r2) {
                        // |eta| = len / (2 |z|) < 1/8: the App. D integrals by their series,
                        // z = midpoint - q, eta = (p2 - p1) / (2 z), zeta = eta^2:
                        //   int log|p-q| dS = len (log|z| - Re sum_k zeta^k / (2k (2k+1)))
                        //   phi = 2 Im atanh(eta)
                        const float dx = bx - ax, dy = by - ay, ir2 = 1.f / r2;
                        const float ex = 0.5f * (dx * mx + dy * my) * ir2;
                        const float ey = 0.5f * (dy * mx - dx * my) * ir2;
                        const float zx = ex * ex - ey * ey, zy = 2.f * ex * ey;
                        // s = zeta (1/6 + zeta (1/20 + zeta / 42))
                        float tx = 1.f / 20.f + zx * (1.f / 42.f), ty = zy * (1.f / 42.f);
                        float ux = 1.f / 6.f + (zx * tx - zy * ty), uy = zx * ty + zy * tx;
                        const float sre = zx * ux - zy * uy;
                        ilog = len * (0.5f * __logf(r2) - sre);
                        // atanh: eta (1 + zeta (1/3 + zeta (1/5 + zeta / 7)))
                        tx = 1.f / 5.f + zx * (1.f / 7.f);
                        ty = zy * (1.f / 7.f);
                        ux = 1.f / 3.f + (zx * tx - zy * ty);
                        uy = zx * ty + zy * tx;
                        const float vx = 1.f + (zx * ux - zy * uy), vy = zx * uy + zy * ux;
                        phi = 2.f * (ex * vy + ey * vx);
                    } else if (!own && dt < 0.f && fabsf(cr) < kNearFallback * len * len) {
                        // near-singular: the side of the curve is decided in FP64
                        const double *P = a.t64.pc + 4 * (size_t)sidx[s];
                        double il64, ph64;
                        seg_ilog_phi_f64(qx64, qy64, P[0], P[1], P[2], P[3], false, il64, ph64);
                        // world units to the scaled frame: il / rho - len' log(rho)
                        // (FP32 from here: these pieces are rare, and nothing
                        // double-precision is kept live across the loop for them)
                        const float iwr = __ldg(t.iw + leaf);
                        ilog = (float)il64 * iwr + len * __logf(iwr);
                        phi = (float)ph64;
                    } else {
                        float ilen = 1.f / len;
                        phi = own ? 0.f : atan2f(cr, dt);
                        float dx = bx - ax, dy = by - ay;
                        float ra2 = ax * ax + ay * ay, rb2 = bx * bx + by * by;
                        float s1 = (ax * dx + ay * dy) * ilen;
                        float s2 = s1 + len;
                        // s2 log rb2 - s1 log ra2, through log1p when rb2 ~ ra2
                        float delta = (dx * (ax + bx) + dy * (ay + by)) / ra2;
                        float lg;
                        if (fabsf(delta) < 0.5f) {
                            lg = s2 * log1pf(delta) + len * __logf(ra2);
                        } else {
                            float la = ra2 > 0.f ? s1 * __logf(ra2) : 0.f;
                            float lb = rb2 > 0.f ? s2 * __logf(rb2) : 0.f;
                            lg = lb - la;
                        }
                        ilog = 0.5f * lg - len + cr * ilen * phi;
                    }
                    u0 = fmaf(ilog, ssg[0][s], fmaf(phi, smg[0][s], u0));
                    u1 = fmaf(ilog, ssg[1][s], fmaf(phi, smg[1][s], u1));
                    u2 = fmaf(ilog, ssg[2][s], fmaf(phi, smg[2][s], u2));
                }
            }
        }
    }
    if (!act) return;
    if (MODE == 0) {
        size_t o = 3 * ((size_t)vp.offset + (size_t)r * vp.width + c);
        float u[3] = {(float)(u0 + h0), (float)(u1 + h1), (float)(u2 + h2)};
        for (int ch = 0; ch < 3; ++ch) {
            if (a.rgb) {
                if (a.rgb_dtype == DC_F64) static_cast<double *>(a.rgb)[o + ch] = (double)u[ch];
                else static_cast<float *>(a.rgb)[o + ch] = u[ch];
            }
            if (a.rgb8) a.rgb8[o + ch] = quant8(u[ch]);
        }
    } else {
        int o = a.perm[ti];
        a.out[3 * (size_t)o + 0] = u0 + h0;
        a.out[3 * (size_t)o + 1] = u1 + h1;
        a.out[3 * (size_t)o + 2] = u2 + h2;
    }
}

// One item per block, or, with a.queue, a persistent grid whose blocks take
// items from the counter *a.queue in list order (the render's tiles are
// listed by decreasing estimated cost, so the longest start first).
template <int MODE, int TW, int TH>
__global__ void __launch_bounds__(TW * TH, kEvThreadsPerSM / (TW * TH)) eval32_kernel(EvalArgs32 a) {
    if (!a.queue) {
        eval32_item<MODE, TW, TH>(a, blockIdx.x);
        return;
    }
    __shared__ int next;
    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) next = atomicAdd(a.queue, 1);
        __syncthreads();
        const int it = next;
        if (it >= a.n_items) break;
        eval32_item<MODE, TW, TH>(a, it);
    }
}

// ----------------------------------------------------- host helpers --
using cd = std::complex<double>;

template <typename T>
cudaError_t up(DevBuf<T> &buf, const std::vector<T> &v, cudaStream_t st) {
    cudaError_t e = buf.alloc(std::max<size_t>(v.size(), 1));
    if (e != cudaSuccess || v.empty()) return e;
    return cudaMemcpyAsync(buf.ptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st);
}

cudaError_t to_f32(DevBuf<float2> &dst, const DevBuf<double2> &src, cudaStream_t st) {
    std::vector<double2> h(src.n);
    cudaError_t e = cudaMemcpyAsync(h.data(), src.ptr, src.bytes(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    std::vector<float2> f(h.size());
    for (size_t i = 0; i < h.size(); ++i) f[i] = make_float2((float)h[i].x, (float)h[i].y);
    return up(dst, f, st);
}

}  // namespace

DevTree32 Fmm::Impl::dt32() const {
    DevTree32 t;
    t.iw = iw32.ptr;
    t.logw = logw32.ptr;
    t.parent = parent.ptr;
    t.child0 = child0.ptr;
    t.quad = quad.ptr;
    t.pstart = pstart.ptr;
    t.pcount = pcount.ptr;
    t.pc = pc32.ptr;
    t.pw = pw32.ptr;
    t.plen = plen32.ptr;
    t.pseg = pseg.ptr;
    t.u_ptr = u_ptr.ptr;
    t.u_idx = u_idx.ptr;
    t.v_ptr = v_ptr.ptr;
    t.v_idx = v_idx.ptr;
    t.v_off = v_off.ptr;
    t.w_ptr = w_ptr.ptr;
    t.w_idx = w_idx.ptr;
    t.x_ptr = x_ptr.ptr;
    t.x_idx = x_idx.ptr;
    t.u_off = uoff32.ptr;
    t.w_off = woff32.ptr;
    t.x_off = xoff32.ptr;
    t.uf_ptr = uf_ptr.ptr;
    t.uf_idx = uf_idx.ptr;
    t.pch = pch32.ptr;
    t.pcl = pcl32.ptr;
    return t;
}

void Fmm::Impl::prep32(const Tree &T, const Geometry &G, Prep32 &o) {
    const int nC = T.n_cells();
    o.iw.resize(nC);
    o.logw.resize(nC);
    o.ccx.resize(nC);
    o.ccy.resize(nC);
    for (int c = 0; c < nC; ++c) {
        double w = T.width(c);
        o.iw[c] = (float)(1.0 / w);
        o.logw[c] = (float)std::log(w);
        o.ccx[c] = T.cx(c);
        o.ccy[c] = T.cy(c);
    }
    const size_t np = T.pc_seg.size();
    o.pcf.resize(np);
    o.pch.resize(np);
    o.pcl.resize(np);
    o.pwf.resize(np);
    o.plf.resize(np);
    std::vector<int> owner(np, -1);
    for (int c = 0; c < nC; ++c)
        for (int i = T.piece_start[c]; i < T.piece_start[c] + T.piece_count[c]; ++i) owner[i] = c;
    for (size_t i = 0; i < np; ++i) {
        const double *q = &T.pc_xy[4 * i];
        int c = owner[i];
        o.pcf[i] = make_float4((float)(q[0] - o.ccx[c]), (float)(q[1] - o.ccy[c]), (float)(q[2] - o.ccx[c]),
                               (float)(q[3] - o.ccy[c]));
        float h[4], l[4];
        for (int k = 0; k < 4; ++k) {
            h[k] = (float)q[k];
            l[k] = (float)(q[k] - (double)h[k]);
        }
        o.pch[i] = make_float4(h[0], h[1], h[2], h[3]);
        o.pcl[i] = make_float4(l[0], l[1], l[2], l[3]);
        o.pwf[i] = (float)G.seg_w[T.pc_seg[i]];
        o.plf[i] = (float)std::hypot(q[2] - q[0], q[3] - q[1]);
    }
    auto offsets = [&](const std::vector<int> &ptr, const std::vector<int> &idx) {
        std::vector<float2> v(idx.size());
        for (int c = 0; c + 1 < (int)ptr.size(); ++c)
            for (int e = ptr[c]; e < ptr[c + 1]; ++e)
                v[e] = make_float2((float)(o.ccx[idx[e]] - o.ccx[c]), (float)(o.ccy[idx[e]] - o.ccy[c]));
        return v;
    };
    o.uo = offsets(T.u_ptr, T.u_idx);
    o.wo = offsets(T.w_ptr, T.w_idx);
    o.xo = offsets(T.x_ptr, T.x_idx);
}

dc_status Fmm::Impl::build32(const Geometry &G, const Prep32 &pr, const std::vector<double> &nxy,
                             const std::vector<int> &start, const std::vector<int> &cnt, cudaStream_t st,
                             std::string &err) {
    const Tree &T = tree;
    const int nC = T.n_cells();
    const size_t np = T.pc_seg.size();
    const std::vector<double> &ccx = pr.ccx, &ccy = pr.ccy;
    // node targets relative to their leaf; work items of <= 64 targets
    const int N = G.n_nodes();
    std::vector<float2> q32(N);
    std::vector<Tile> items;
    for (int c = 0; c < nC; ++c) {
        for (int j = start[c]; j < start[c] + cnt[c]; ++j)
            q32[j] = make_float2((float)(nxy[2 * j] - ccx[c]), (float)(nxy[2 * j + 1] - ccy[c]));
        for (int j = 0; j < cnt[c]; j += 64) items.push_back({c, start[c] + j, 0, std::min(64, cnt[c] - j), 0});
    }
    cudaError_t e;
    n_nt_items = int(items.size());
    if ((e = up(iw32, pr.iw, st)) != cudaSuccess || (e = up(logw32, pr.logw, st)) != cudaSuccess ||
        (e = up(pc32, pr.pcf, st)) != cudaSuccess || (e = up(pch32, pr.pch, st)) != cudaSuccess ||
        (e = up(pcl32, pr.pcl, st)) != cudaSuccess || (e = up(pw32, pr.pwf, st)) != cudaSuccess ||
        (e = up(plen32, pr.plf, st)) != cudaSuccess || (e = up(uoff32, pr.uo, st)) != cudaSuccess ||
        (e = up(woff32, pr.wo, st)) != cudaSuccess || (e = up(xoff32, pr.xo, st)) != cudaSuccess ||
        (e = up(nt_q32, q32, st)) != cudaSuccess || (e = up(nt_items, items, st)) != cudaSuccess ||
        (e = to_f32(m2m32, m2m, st)) != cudaSuccess || (e = to_f32(l2l32, l2l, st)) != cudaSuccess ||
        (e = to_f32(m2l32, m2l, st)) != cudaSuccess || (e = to_f32(base32, base64, st)) != cudaSuccess ||
        (e = Lm2l32.alloc((size_t)nC * 3 * P1)) != cudaSuccess ||
        (e = heavy.alloc(std::max<size_t>(np, 1))) != cudaSuccess ||
        (e = heavyL.alloc((size_t)nC)) != cudaSuccess || (e = heavyM.alloc((size_t)nC)) != cudaSuccess ||
        (e = M32.alloc((size_t)nC * 3 * P1)) != cudaSuccess ||
        (e = L32.alloc((size_t)nC * 3 * P1)) != cudaSuccess ||
        (e = sbar32.alloc((size_t)3 * D->S)) != cudaSuccess ||
        (e = mbar32.alloc((size_t)3 * D->S)) != cudaSuccess) {
        err = std::string("fmm32 allocation: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? DC_ERR_OOM : DC_ERR_CUDA;
    }
    cudaMemsetAsync(sbar32.ptr, 0, sbar32.bytes(), st);
    cudaMemsetAsync(mbar32.ptr, 0, mbar32.bytes(), st);
    cudaMemsetAsync(heavy.ptr, 0, heavy.bytes(), st);
    cudaMemsetAsync(heavyL.ptr, 0, heavyL.bytes(), st);
    cudaMemsetAsync(heavyM.ptr, 0, heavyM.bytes(), st);
    cudaFuncSetAttribute(passes::m2l_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)passes::m2l_smem<float>(P1));
    if (P1i <= passes::kM2LSmallP1)
        cudaFuncSetAttribute(passes::m2l_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)passes::m2l_small_smem(P1i));
    cudaFuncSetAttribute(passes::p2l_kernel<float, passes::PiecesF32>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)passes::p2l_smem<float>(P1));
    cudaFuncSetAttribute(passes::p2m_kernel<float, passes::PiecesF32>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)passes::p2m_smem<float>(P1));
    cudaFuncSetAttribute(passes::p2l_flat_kernel<float, passes::PiecesF32>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)passes::p2l_flat_smem<float>(P1));
    return DC_OK;
}

cudaError_t Fmm::Impl::interp32(const double *node_vals, float *seg_vals, cudaStream_t st) {
    int th = 256;
    (void)th;
    interp32_kernel<<<D->n_panels, std::min(256, (D->s + 31) / 32 * 32), 0, st>>>(lam_ff.ptr, node_vals, seg_vals,
                                                                               D->s, D->g);
    note_launch();
    return cudaGetLastError();
}

cudaError_t Fmm::Impl::to_f32_density(const double *sb, const double *mb, cudaStream_t st) {
    int n = 3 * D->S, th = 256;
    d2f_kernel<<<(n + th - 1) / th, th, 0, st>>>(sb, mb, sbar32.ptr, mbar32.ptr, n); note_launch();
    return cudaGetLastError();
}

passes::TreeView<float> Fmm::Impl::view32() const {
    passes::TreeView<float> v;
    v.iw = iw32.ptr;
    v.logw = logw32.ptr;
    v.parent = parent.ptr;
    v.child0 = child0.ptr;
    v.quad = quad.ptr;
    v.pstart = pstart.ptr;
    v.pcount = pcount.ptr;
    v.pw = pw32.ptr;
    v.plen = plen32.ptr;
    v.pseg = pseg.ptr;
    v.v_ptr = v_ptr.ptr;
    v.v_idx = v_idx.ptr;
    v.v_code = v_code.ptr;
    v.x_ptr = x_ptr.ptr;
    v.x_idx = x_idx.ptr;
    v.x_off = xoff32.ptr;
    return v;
}

// M2L (list 2) of the FP32 passes at order P1i: part 0 is the main kernel
// (tcgen05 tiles for the node schedule when built, else the CUDA-core
// m2l_small_kernel), part 1 the tensor path's per-target reduction (nothing
// on the CUDA cores).
cudaError_t Fmm::Impl::launch_m2l32(const Schedule &sc, int part, cudaStream_t st) {
    const int P1 = P1i;
    passes::TreeView<float> tv = view32();
    if (n_tc_tiles > 0 && &sc == &sched_nodes) {   // tensor cores
        if (part == 0) {
            passes::m2l_tc_kernel<<<std::min(n_tc_tiles, passes::kTcBlocksPerSM * n_sms), passes::kTcThreads, 0, st>>>(
                tc_tiles.ptr, n_tc_tiles, tc_entries.ptr, tv.v_idx, P1, tc_tab.ptr, M32i.ptr, tc_y.ptr, tc_err.ptr);
        } else {
            passes::m2l_tc_reduce_kernel<<<(sc.n_m2l + passes::kTcReduceWarps - 1) / passes::kTcReduceWarps,
                                           32 * passes::kTcReduceWarps, 0, st>>>(tv, sc.m2l.ptr, sc.n_m2l, P1,
                                                                                 tc_y.ptr, M32i.ptr, Lm2l32i.ptr);
        }
        note_launch();
    } else if (part == 0) {
        int grid = std::min((sc.n_m2l + passes::kM2LSmallWarps - 1) / passes::kM2LSmallWarps, 2 * n_sms);
        passes::m2l_small_kernel<<<grid, 32 * passes::kM2LSmallWarps, passes::m2l_small_smem(P1), st>>>(
            tv, sc.m2l.ptr, sc.n_m2l, P1, m2lfull32i.ptr, M32i.ptr, Lm2l32i.ptr);
        note_launch();
    }
    return cudaGetLastError();
}

// Average device time of the inner operator's M2L kernels over `reps`
// launches each (CUDA events on st, one warm-up launch first):
//   out[0] ms of part 0, out[1] ms of part 1 (0 on the CUDA cores),
//   out[2] algorithmic flops per application, 8 P1i^2 per (pair, channel)
//          (one complex multiply-add = 8 real flops),
//   out[3] flops the tensor pipe executes per application (three TF32
//          products of 128 x 32 x 32 per tile; 0 on the CUDA cores),
//   out[4] engine (DC_M2L_TENSOR / DC_M2L_CUDA_CORES), out[5] list-2 pairs.
cudaError_t Fmm::Impl::time_inner_m2l(int reps, cudaStream_t st, double out[6]) {
    const Schedule &sc = sched_nodes;
    for (int i = 0; i < 6; ++i) out[i] = 0.0;
    if (!fp32 || sc.n_m2l == 0) return cudaErrorNotSupported;
    if (!(n_tc_tiles > 0) && !(P1i <= passes::kM2LSmallP1)) return cudaErrorNotSupported;
    cudaError_t e;
    if (!ev0 && (e = cudaEventCreate(&ev0)) != cudaSuccess) return e;
    if (!ev1 && (e = cudaEventCreate(&ev1)) != cudaSuccess) return e;
    const int parts = n_tc_tiles > 0 ? 2 : 1;
    for (int part = 0; part < parts; ++part) {
        if ((e = launch_m2l32(sc, part, st)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(ev0, st)) != cudaSuccess) return e;
        for (int r = 0; r < reps; ++r)
            if ((e = launch_m2l32(sc, part, st)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(ev1, st)) != cudaSuccess) return e;
        if ((e = cudaEventSynchronize(ev1)) != cudaSuccess) return e;
        float ms = 0.f;
        if ((e = cudaEventElapsedTime(&ms, ev0, ev1)) != cudaSuccess) return e;
        out[part] = ms / reps;
    }
    const long long pairs = m2l_pairs_nodes;
    out[2] = 8.0 * P1i * P1i * 3.0 * (double)pairs;
    out[3] = n_tc_tiles > 0 ? 3.0 * 2.0 * 128.0 * 32.0 * 32.0 * n_tc_tiles : 0.0;
    out[4] = n_tc_tiles > 0 ? DC_M2L_TENSOR : DC_M2L_CUDA_CORES;
    out[5] = (double)pairs;
    std::string msg;
    return check_tc_wait(st, msg);
}

cudaError_t Fmm::Impl::passes32(const float *sb, const float *mb, int use_s, int use_m,
                                cudaStream_t st, const Schedule &sc) {
    const int nC = tree.n_cells();
    const int P1 = P1i;
    size_t ebytes = (size_t)nC * 3 * P1 * sizeof(float2);
    cudaError_t e;
    passes::TreeView<float> tv = view32();
    passes::PiecesF32 ps{pc32.ptr};
    if ((e = cudaMemsetAsync(M32i.ptr, 0, ebytes, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(L32i.ptr, 0, ebytes, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(Lm2l32i.ptr, 0, ebytes, st)) != cudaSuccess) return e;
    if (n_p2m > 0) {
        passes::p2m_kernel<float, passes::PiecesF32><<<n_p2m, passes::kChunk, passes::p2m_smem<float>(P1), st>>>(
            tv, ps, p2m_leaves.ptr, sb, mb, use_s, use_m, P1, M32i.ptr, rows_ready && !use_m ? p2m_g32.ptr : nullptr);
        note_launch();
    }
    if (n_mchunks > 0) {   // every inner cell straight from its leaves
        passes::m2m_multi_kernel<float><<<(n_mchunks + passes::kMultiWarps - 1) / passes::kMultiWarps,
                                          32 * passes::kMultiWarps, 0, st>>>(
            pair_geo.ptr, mchunks.ptr, n_mchunks, pair_leaf.ptr, P1, binom32.ptr, M32i.ptr, mpart32.ptr);
        note_launch();
        if (n_mred > 0) {
            passes::m2m_reduce_kernel<float><<<n_mred, passes::kReduceThreads, 0, st>>>(mred.ptr, n_mred, P1, mpart32.ptr,
                                                                                     M32i.ptr);
            note_launch();
        }
    }
    if (sc.n_m2l > 0 && ((n_tc_tiles > 0 && &sc == &sched_nodes) || P1 <= passes::kM2LSmallP1)) {
        if ((e = launch_m2l32(sc, 0, st)) != cudaSuccess) return e;
        if ((e = launch_m2l32(sc, 1, st)) != cudaSuccess) return e;
    } else if (sc.n_m2l > 0) {
        int grid = std::min((sc.n_m2l + passes::kM2LSlots - 1) / passes::kM2LSlots, 4 * n_sms);
        passes::m2l_kernel<float><<<grid, 32 * passes::kM2LSlots, passes::m2l_smem<float>(P1), st>>>(
            tv, sc.m2l.ptr, sc.n_m2l, P1, base32i.ptr, M32i.ptr, Lm2l32i.ptr);
        note_launch();
    }
    if (sc.n_p2l > 0) {
        passes::p2l_flat_kernel<float, passes::PiecesF32><<<sc.n_p2l, passes::kChunk, passes::p2l_flat_smem<float>(P1), st>>>(
            tv, ps, sc.p2l.ptr, p2l_off.ptr, p2l_cnt.ptr, p2l_item.ptr, sb, mb, use_s, use_m, P1, Lm2l32i.ptr);
        note_launch();
    }
    if (sc.n_walk > 0) {
        passes::walk_kernel<float><<<sc.n_walk, std::max(32, (std::max(P1, walk_nmax) + 31) / 32 * 32),
                                     passes::walk_smem<float>(P1, walk_nmax), st>>>(
            tv, sc.walk.ptr, sc.chains.ptr, P1, walk_nmax, l2l32i.ptr, Lm2l32i.ptr, L32i.ptr);
        note_launch();
    }
    return cudaGetLastError();
}

cudaError_t Fmm::Impl::prepare_render32(const double *sb, const double *mb, cudaStream_t st) {
    cudaError_t e = to_f32_density(sb, mb, st);
    if (e != cudaSuccess) return e;
    if ((e = passes(sb, mb, 1, 1, st, sched_all)) != cudaSuccess) return e;
    const int th = 256, np = int(tree.pc_seg.size()), nC = tree.n_cells();
    if (np > 0) {
        heavy_kernel<<<(np + th - 1) / th, th, 0, st>>>(sb, mb, pseg.ptr, pw.ptr, plen64.ptr, heavy.ptr, np);
        note_launch();
    }
    near_centre_kernel<<<(unsigned)(((size_t)nC * 32 + th - 1) / th), th, 0, st>>>(
        uf_ptr.ptr, uf_idx.ptr, pseg.ptr, pw32.ptr, plen32.ptr, np > 0 ? heavy.ptr : nullptr, sbar32.ptr, iw32.ptr, nC,
        P1, L.ptr);
    note_launch();
    big_coef_kernel<<<(unsigned)(((size_t)nC * 32 + th - 1) / th), th, 0, st>>>(L.ptr, M.ptr, nC, P1, heavyL.ptr, heavyM.ptr);
    note_launch();
    const size_t n = (size_t)nC * 3 * P1;
    narrow_kernel<double2, float2><<<(unsigned)((n + th - 1) / th), th, 0, st>>>(M.ptr, M32.ptr, n);
    narrow_kernel<double2, float2><<<(unsigned)((n + th - 1) / th), th, 0, st>>>(L.ptr, L32.ptr, n);
    note_launch(2);
    return cudaGetLastError();
}

cudaError_t Fmm::Impl::apply_nodes32(const double *x, double *y, bool single, cudaStream_t st) {
    cudaError_t e = interp32(x, single ? sbar32.ptr : mbar32.ptr, st);
    if (e != cudaSuccess) return e;
    return nodes32_from_segments(y, single, st);
}

evalnodes::NodeArgs<float> Fmm::Impl::node_args32(double *y, bool single) const {
    evalnodes::NodeArgs<float> a;
    a.u_ptr = u_ptr.ptr;
    a.u_idx = u_idx.ptr;
    a.w_ptr = w_ptr.ptr;
    a.w_idx = w_idx.ptr;
    a.pstart = pstart.ptr;
    a.pcount = pcount.ptr;
    a.pseg = pseg.ptr;
    a.pc64 = pc.ptr;
    a.cc64 = cc.ptr;
    a.pw = pw32.ptr;
    a.iw = iw32.ptr;
    a.logw = logw32.ptr;
    a.items = nt_items4.ptr;
    a.q64 = nt_xy.ptr;
    a.own1 = nt_own1.ptr;
    a.own2 = nt_own2.ptr;
    a.perm = nt_perm.ptr;
    a.sb = sbar32.ptr;
    a.mb = mbar32.ptr;
    a.use_s = single ? 1 : 0;
    a.use_m = single ? 0 : 1;
    a.out = y;
    a.P1 = P1i;
    a.M = M32i.ptr;
    a.L = L32i.ptr;
    a.uf_ptr = uf_ptr.ptr;
    a.uf_seg = uf_seg.ptr;
    return a;
}

cudaError_t Fmm::Impl::nodes32_from_segments(double *y, bool single, cudaStream_t st) {
    if (single && split_ok()) return nodes32_split(y, st, false);
    cudaError_t e;
    int us = single ? 1 : 0, um = single ? 0 : 1;
    if ((e = passes32(sbar32.ptr, mbar32.ptr, us, um, st, sched_nodes)) != cudaSuccess) return e;
    if (n_nt_items4 == 0) return cudaSuccess;
    const evalnodes::NodeArgs<float> a = node_args32(y, single);
    const dim3 grid(n_nt_items4), block(32 * evalnodes::kWarps);
    if (near_ready && single)
        evalnodes::near_apply_kernel<float><<<grid, block, 0, st>>>(
            a, near_off.ptr, near_g32.ptr, sbar32.ptr, far_ready ? far_off.ptr : nullptr,
            far_ready ? far32.ptr : nullptr);
    else
        evalnodes::eval_nodes_kernel<float><<<grid, block, 0, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

// The inner node operator with the list-4 P2L (it needs only the segment
// densities) as a branch of its own on side beside P2M -> M2M (and the
// tensor-core M2L's MMAs) on st; the M2L (its reduction, or the CUDA-core
// kernel) adds onto the P2L terms once the branch is done, then the walk and
// the node evaluation.  (A third branch for the near field measured slower:
// its blocks delay the chain's.)
bool Fmm::Impl::split_ok() const {
    const bool m2l_ok = n_tc_tiles > 0 || P1i <= passes::kM2LSmallP1;   // both engines add onto the P2L terms
    return graph_split && m2l_ok && sched_nodes.n_m2l > 0 && near_ready && n_nt_items4 > 0;
}

cudaError_t Fmm::Impl::nodes32_split(double *y, cudaStream_t st, bool fork) {
    const Schedule &sc = sched_nodes;
    const int nC = tree.n_cells();
    const int P1 = P1i;
    const size_t ebytes = (size_t)nC * 3 * P1 * sizeof(float2);
    cudaError_t e;
    passes::TreeView<float> tv = view32();
    passes::PiecesF32 ps{pc32.ptr};
    if ((e = cudaMemsetAsync(M32i.ptr, 0, ebytes, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(L32i.ptr, 0, ebytes, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(Lm2l32i.ptr, 0, ebytes, st)) != cudaSuccess)
        return e;
    const cudaStream_t s1 = fork ? side : st;
    if (fork && (e = cudaEventRecord(fork_ev[0], st)) != cudaSuccess) return e;
    const evalnodes::NodeArgs<float> a = node_args32(y, true);
    const dim3 grid(n_nt_items4), block(32 * evalnodes::kWarps);
    // branch: list 4
    if (fork && (e = cudaStreamWaitEvent(s1, fork_ev[0], 0)) != cudaSuccess) return e;
    if (sc.n_p2l > 0) {
        passes::p2l_flat_kernel<float, passes::PiecesF32><<<sc.n_p2l, passes::kChunk, passes::p2l_flat_smem<float>(P1),
                                                            s1>>>(tv, ps, sc.p2l.ptr, p2l_off.ptr, p2l_cnt.ptr,
                                                                  p2l_item.ptr, sbar32.ptr, mbar32.ptr, 1, 0, P1,
                                                                  Lm2l32i.ptr);
        note_launch();
    }
    if (fork && (e = cudaEventRecord(fork_ev[1], s1)) != cudaSuccess) return e;
    // main branch
    if (n_p2m > 0) {
        passes::p2m_kernel<float, passes::PiecesF32><<<n_p2m, passes::kChunk, passes::p2m_smem<float>(P1), st>>>(
            tv, ps, p2m_leaves.ptr, sbar32.ptr, mbar32.ptr, 1, 0, P1, M32i.ptr, rows_ready ? p2m_g32.ptr : nullptr);
        note_launch();
    }
    if (n_mchunks > 0) {
        passes::m2m_multi_kernel<float><<<(n_mchunks + passes::kMultiWarps - 1) / passes::kMultiWarps,
                                          32 * passes::kMultiWarps, 0, st>>>(
            pair_geo.ptr, mchunks.ptr, n_mchunks, pair_leaf.ptr, P1, binom32.ptr, M32i.ptr, mpart32.ptr);
        note_launch();
        if (n_mred > 0) {
            passes::m2m_reduce_kernel<float><<<n_mred, passes::kReduceThreads, 0, st>>>(mred.ptr, n_mred, P1,
                                                                                     mpart32.ptr, M32i.ptr);
            note_launch();
        }
    }
    // tensor cores: the MMAs beside the branch, their reduction after it;
    // CUDA cores: the whole M2L after it (both add onto the P2L terms)
    const bool tc = n_tc_tiles > 0;
    if (tc && sc.n_m2l > 0 && (e = launch_m2l32(sc, 0, st)) != cudaSuccess) return e;
    if (fork && (e = cudaStreamWaitEvent(st, fork_ev[1], 0)) != cudaSuccess) return e;
    if (sc.n_m2l > 0 && (e = launch_m2l32(sc, tc ? 1 : 0, st)) != cudaSuccess) return e;
    if (sc.n_walk > 0) {
        passes::walk_kernel<float><<<sc.n_walk, std::max(32, (std::max(P1, walk_nmax) + 31) / 32 * 32),
                                     passes::walk_smem<float>(P1, walk_nmax), st>>>(
            tv, sc.walk.ptr, sc.chains.ptr, P1, walk_nmax, l2l32i.ptr, Lm2l32i.ptr, L32i.ptr);
        note_launch();
    }
    evalnodes::near_apply_kernel<float><<<grid, block, 0, st>>>(a, near_off.ptr, near_g32.ptr, sbar32.ptr,
                                                                far_ready ? far_off.ptr : nullptr,
                                                                far_ready ? far32.ptr : nullptr);
    note_launch();
    return cudaGetLastError();
}

// Captures the FP32 preconditioned matvec (g_in -> g_out) once.
cudaError_t Fmm::Impl::graph_ensure() {
    if (g32_exec) return cudaSuccess;
    cudaError_t e;
    if ((e = g_in.ensure(3 * (size_t)D->N)) != cudaSuccess) return e;
    if ((e = g_out.ensure(3 * (size_t)D->N)) != cudaSuccess) return e;
    // the chain P2M -> M2M -> M2L -> walk is the critical path: its nodes run
    // at the highest priority, the parallel branches at the lowest
    int prio_lo = 0, prio_hi = 0;
    if ((e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi)) != cudaSuccess) return e;
    if (!cap_stream && (e = cudaStreamCreateWithPriority(&cap_stream, cudaStreamNonBlocking, prio_hi)) != cudaSuccess)
        return e;
    if (coarse.aggregated() &&
        ((e = agg_py.ensure(3 * (size_t)D->N)) != cudaSuccess || (e = agg_gpy.ensure(3 * (size_t)D->N)) != cudaSuccess))
        return e;
    // the branches: tensor-core M2L (its reduction adds onto the P2L terms)
    // and the near field from stored coefficients
    const bool split = split_ok();
    if (split) {
        if (!side && (e = cudaStreamCreateWithPriority(&side, cudaStreamNonBlocking, prio_lo)) != cudaSuccess) return e;
        for (auto &ev : fork_ev)
            if (!ev && (e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return e;
    }
    auto node_op = [&](double *y) {
        return split ? nodes32_split(y, cap_stream, true) : nodes32_from_segments(y, true, cap_stream);
    };
    long long before = kernel_launches();
    if ((e = cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
    // M v straight to the segments (sigma_bar = Lambda M v) when the
    // two-level preconditioner is in use, else M v at the nodes first; the
    // aggregated coarse level takes its residual G_H P y from this operator
    cudaError_t e1;
    if (coarse.aggregated()) {
        e1 = coarse.apply_stage1(g_in.ptr, agg_py.ptr, cap_stream);
        if (e1 == cudaSuccess) e1 = interp32(agg_py.ptr, sbar32.ptr, cap_stream);
        if (e1 == cudaSuccess) e1 = node_op(agg_gpy.ptr);
        if (e1 == cudaSuccess)
            e1 = coarse.apply_stage2(pinv.ptr, g_in.ptr, agg_gpy.ptr, nullptr, cap_stream, lam_ff.ptr, D->s, sbar32.ptr);
    } else {
        e1 = coarse.ready() ? coarse.apply(pinv.ptr, g_in.ptr, nullptr, cap_stream, lam_ff.ptr, D->s, sbar32.ptr)
                            : precond(g_in.ptr, ir_t.ptr, cap_stream);
    }
    cudaError_t e2 = e1;
    if (e1 == cudaSuccess)
        e2 = coarse.ready() ? node_op(g_out.ptr) : apply_nodes32(ir_t.ptr, g_out.ptr, true, cap_stream);
    e = cudaStreamEndCapture(cap_stream, &g32);
    g32_kernels = int(kernel_launches() - before);
    note_launch(-g32_kernels);   // counted again at every graph launch
    if (e2 != cudaSuccess) return e2;
    if (e != cudaSuccess) return e;
    return cudaGraphInstantiate(&g32_exec, g32, split ? cudaGraphInstantiateFlagUseNodePriority : 0);
}

// g_out = A32 M g_in (the captured graph)
cudaError_t Fmm::Impl::graph_launch(cudaStream_t st) {
    cudaError_t e = graph_ensure();
    if (e != cudaSuccess) return e;
    if ((e = cudaGraphLaunch(g32_exec, st)) != cudaSuccess) return e;
    note_launch(g32_kernels);
    return cudaSuccess;
}

cudaError_t Fmm::Impl::graph_matvec32(const double *x, double *y, cudaStream_t st) {
    const size_t bytes = sizeof(double) * 3 * (size_t)D->N;
    cudaError_t e = graph_ensure();
    if (e != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(g_in.ptr, x, bytes, cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
    if ((e = graph_launch(st)) != cudaSuccess) return e;
    return cudaMemcpyAsync(y, g_out.ptr, bytes, cudaMemcpyDeviceToDevice, st);
}

cudaError_t Fmm::Impl::render_tiles32(int n_tiles, void *rgb, int rgb_dtype,
                                      unsigned char *rgb8, const double *sb64, const double *mb64,
                                      cudaStream_t st) {
    EvalArgs32 a{};
    a.sb64 = sb64;
    a.mb64 = mb64;
    a.heavy = heavy.ptr;

    a.t = dt32();
    a.t64 = dt();
    a.items = tiles.ptr;
    a.P1 = P1;
    a.M = M32.ptr;
    a.L = L32.ptr;
    a.sb = sbar32.ptr;
    a.mb = mbar32.ptr;
    a.use_s = 1;
    a.use_m = 1;
    a.hL = heavyL.ptr;
    a.hM = heavyM.ptr;
    a.M64 = M.ptr;
    a.L64 = L.ptr;
    a.vps = vps.ptr;
    a.rgb = rgb;
    a.rgb_dtype = rgb_dtype;
    a.rgb8 = rgb8;
    // persistent: as many blocks as are resident (the same register budget
    // for every tile shape), taking tiles from a counter
    cudaError_t e;
    if ((e = render_queue.ensure(1)) != cudaSuccess ||
        (e = cudaMemsetAsync(render_queue.ptr, 0, sizeof(int), st)) != cudaSuccess)
        return e;
    a.queue = render_queue.ptr;
    a.n_items = n_tiles;
    int tw = 8, th = 8;
    tile_shape(opt.eval_tile, tw, th);
    const int grid = std::max(1, std::min(n_tiles, n_sms * (kEvThreadsPerSM / (tw * th))));
    switch (opt.eval_tile) {   // tile shapes of tile_shape()
    case 1: eval32_kernel<0, 16, 8><<<grid, 128, 0, st>>>(a); break;
    case 2: eval32_kernel<0, 16, 16><<<grid, 256, 0, st>>>(a); break;
    case 3: eval32_kernel<0, 32, 8><<<grid, 256, 0, st>>>(a); break;
    default: eval32_kernel<0, 8, 8><<<grid, 64, 0, st>>>(a); break;
    }
    note_launch();
    return cudaGetLastError();
}

cudaError_t Fmm::Impl::eval_points32(int n_items, double *out, const double *sb64,
                                     const double *mb64, cudaStream_t st) {
    return eval_points32_at(pt_items.ptr, n_items, pt_xy.ptr, pt_perm.ptr, out, sb64, mb64, st);
}

cudaError_t Fmm::Impl::eval_points32_at(const Tile *items, int n_items, const double *q64, const int *perm,
                                        double *out, const double *sb64, const double *mb64, cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    EvalArgs32 a{};
    a.sb64 = sb64;
    a.mb64 = mb64;
    a.heavy = heavy.ptr;

    a.hL = heavyL.ptr;
    a.hM = heavyM.ptr;
    a.M64 = M.ptr;
    a.L64 = L.ptr;
    a.t = dt32();
    a.t64 = dt();
    a.items = items;
    a.P1 = P1;
    a.M = M32.ptr;
    a.L = L32.ptr;
    a.sb = sbar32.ptr;
    a.mb = mbar32.ptr;
    a.use_s = 1;
    a.use_m = 1;
    a.q32 = nullptr;
    a.q64 = q64;
    a.perm = perm;
    a.out = out;
    eval32_kernel<1, 8, 8><<<n_items, 64, 0, st>>>(a); note_launch();
    return cudaGetLastError();
}

}  // namespace dc
