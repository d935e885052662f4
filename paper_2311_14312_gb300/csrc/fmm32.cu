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

__global__ void interp32_kernel(const double *__restrict__ lam, const double *__restrict__ nv,
                                float *__restrict__ sv, int S, int s, int g) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= S) return;
    int panel = k / s, kk = k - panel * s;
    const double *row = lam + (size_t)kk * g;
    const double *src = nv + (size_t)panel * g * 3;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int m = 0; m < g; ++m) {
        double l = __ldg(row + m);
        a0 += l * __ldg(src + 3 * m + 0);
        a1 += l * __ldg(src + 3 * m + 1);
        a2 += l * __ldg(src + 3 * m + 2);
    }
    sv[3 * (size_t)k + 0] = (float)a0;
    sv[3 * (size_t)k + 1] = (float)a1;
    sv[3 * (size_t)k + 2] = (float)a2;
}

// --------------------------------------------------------------- P2M --
__global__ void p2m32_kernel(DevTree32 t, const int *__restrict__ leaves, const float *__restrict__ sb,
                             const float *__restrict__ mb, int use_s, int use_m, int P1,
                             float2 *__restrict__ M) {
    int cell = leaves[blockIdx.x];
    int k = threadIdx.x;
    if (k >= P1) return;
    float iw = t.iw[cell];
    float2 acc[3] = {{0, 0}, {0, 0}, {0, 0}};
    int p0 = t.pstart[cell], pn = t.pcount[cell];
    for (int i = p0; i < p0 + pn; ++i) {
        float4 P = t.pc[i];
        float2 a = make_float2(P.x * iw, P.y * iw), b = make_float2(P.z * iw, P.w * iw);
        float len = t.plen[i], om = t.pw[i] * len;
        float2 S = make_float2(1.f, 0.f), Sp = make_float2(0.f, 0.f), ap = make_float2(1.f, 0.f);
        for (int m = 1; m <= k; ++m) {
            ap = fmul(ap, a);
            Sp = S;
            S = fadd(fmul(b, S), ap);
        }
        float2 cg = fscale(S, om / (k + 1));
        float il = iw / len;
        float2 wr = make_float2((P.z - P.x) * il, (P.w - P.y) * il);
        float2 t1 = fmul(wr, Sp);
        float2 cf = make_float2(t1.y * om, -t1.x * om);   // -i (w/r) S_{k-1} om
        int seg = t.pseg[i];
        for (int c = 0; c < 3; ++c) {
            float s = use_s ? sb[3 * (size_t)seg + c] : 0.f;
            float mu = use_m ? mb[3 * (size_t)seg + c] : 0.f;
            acc[c].x += s * cg.x + mu * cf.x;
            acc[c].y += s * cg.y + mu * cf.y;
        }
    }
    for (int c = 0; c < 3; ++c) M[((size_t)cell * 3 + c) * P1 + k] = acc[c];
}

// --------------------------------------------------------------- M2M --
__global__ void m2m32_kernel(DevTree32 t, int c_lo, int P1, const float2 *__restrict__ tab,
                             float2 *__restrict__ M) {
    int cell = c_lo + blockIdx.x;
    int k = threadIdx.x;
    int ch0 = t.child0[cell];
    if (k >= P1 || ch0 < 0) return;
    float2 acc[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int q = 0; q < 4; ++q) {
        const float2 *T = tab + ((size_t)q * P1 + k) * P1;
        const float2 *src = M + (size_t)(ch0 + q) * 3 * P1;
        for (int j = 0; j <= k; ++j) {
            float2 tq = T[j];
            for (int c = 0; c < 3; ++c) ffma2(acc[c], tq, src[c * P1 + j]);
        }
    }
    for (int c = 0; c < 3; ++c) M[((size_t)cell * 3 + c) * P1 + k] = acc[c];
}

// ------------------------------------------------ L2L + M2L + P2L ----
__global__ void down32_kernel(DevTree32 t, int c_lo, int level, int P1, const float2 *__restrict__ l2l,
                              const float2 *__restrict__ m2l, const float2 *__restrict__ M,
                              const float *__restrict__ sb, const float *__restrict__ mb, int use_s,
                              int use_m, float2 *__restrict__ L) {
    int cell = c_lo + blockIdx.x;
    int l = threadIdx.x;
    if (l >= P1) return;
    float2 acc[3] = {{0, 0}, {0, 0}, {0, 0}};
    if (level >= 3) {
        int par = t.parent[cell], q = t.quad[cell];
        const float2 *T = l2l + ((size_t)q * P1 + l) * P1;
        const float2 *src = L + (size_t)par * 3 * P1;
        for (int k = l; k < P1; ++k) {
            float2 tq = T[k];
            for (int c = 0; c < 3; ++c) ffma2(acc[c], tq, src[c * P1 + k]);
        }
    }
    float mlogw = -t.logw[cell];
    for (int e = t.v_ptr[cell]; e < t.v_ptr[cell + 1]; ++e) {
        int src = t.v_idx[e];
        const float2 *T = m2l + ((size_t)t.v_off[e] * P1 + l) * P1;
        const float2 *ms = M + (size_t)src * 3 * P1;
        for (int k = 0; k < P1; ++k) {
            float2 tq = T[k];
            for (int c = 0; c < 3; ++c) ffma2(acc[c], tq, ms[c * P1 + k]);
        }
        if (l == 0)
            for (int c = 0; c < 3; ++c) ffma2(acc[c], make_float2(mlogw, 0.f), ms[c * P1]);
    }
    float iw = t.iw[cell], wcell = 1.0f / iw, logw = t.logw[cell];
    for (int e = t.x_ptr[cell]; e < t.x_ptr[cell + 1]; ++e) {
        int src = t.x_idx[e];
        float2 off = t.x_off[e];
        int p0 = t.pstart[src], pn = t.pcount[src];
        for (int i = p0; i < p0 + pn; ++i) {
            float4 P = t.pc[i];
            float2 a = make_float2((P.x + off.x) * iw, (P.y + off.y) * iw);   // scaled
            float2 b = make_float2((P.z + off.x) * iw, (P.w + off.y) * iw);
            float len = t.plen[i], om = t.pw[i];
            float2 wv = make_float2((P.z - P.x) / len, (P.w - P.y) / len);
            float2 cg, cf;
            if (l <= 1) {
                float2 lba = flog_ratio(a, b);
                if (l == 0) {
                    // omega sigma [ l (1 - log a) - conj(w) b log(b/a) ],  a = ah * width
                    float2 la = make_float2(0.5f * __logf(a.x * a.x + a.y * a.y) + logw, atan2f(a.y, a.x));
                    float2 wb = fmul(make_float2(wv.x, -wv.y), make_float2(b.x * wcell, b.y * wcell));
                    float2 t2 = fmul(wb, lba);
                    cg = make_float2(om * (len * (1.f - la.x) - t2.x), om * (-len * la.y - t2.y));
                    cf = make_float2(-om * lba.y, om * lba.x);
                } else {
                    float2 t2 = fmul(make_float2(wv.x, -wv.y), lba);
                    cg = fscale(t2, om * wcell);
                    float2 ab = fmul(finv(a), finv(b));
                    cf = fscale(fmul(make_float2(-wv.y, wv.x), ab), om * len * iw);
                }
            } else {
                float2 al = finv(a), be = finv(b);
                float2 T = make_float2(1.f, 0.f), Tp = T, bp = make_float2(1.f, 0.f);
                for (int m = 1; m <= l - 1; ++m) {
                    bp = fmul(bp, be);
                    Tp = T;
                    T = fadd(fmul(al, T), bp);
                }
                float2 ab = fmul(al, be);
                cg = fscale(fmul(ab, Tp), om * len / (float(l) * (l - 1)));
                cf = fscale(fmul(fmul(make_float2(-wv.y, wv.x), ab), T), om * len * iw / l);
            }
            int seg = t.pseg[i];
            for (int c = 0; c < 3; ++c) {
                float s = use_s ? sb[3 * (size_t)seg + c] : 0.f;
                float mu = use_m ? mb[3 * (size_t)seg + c] : 0.f;
                acc[c].x += s * cg.x + mu * cf.x;
                acc[c].y += s * cg.y + mu * cf.y;
            }
        }
    }
    for (int c = 0; c < 3; ++c) L[((size_t)cell * 3 + c) * P1 + l] = acc[c];
}

// -------------------------------------------------------------- eval --
constexpr int kEvThreads = 256;
constexpr int kStage = 128;

struct EvalArgs32 {
    DevTree32 t;
    DevTree t64;
    const Tile *items;
    int P1;
    const float2 *M, *L;
    const float *sb, *mb;
    int use_s, use_m;
    // pixel mode
    VpDev vp;
    void *rgb;
    int rgb_dtype;
    unsigned char *rgb8;
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

// float pair (hi, lo) with hi + lo = v to about 2^-48 relative
__device__ __forceinline__ void split2(double v, float &hi, float &lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

template <int MODE>
__global__ void __launch_bounds__(kEvThreads) eval32_kernel(EvalArgs32 a) {
    // staged pieces of one list-1 leaf, in the target leaf's frame, each
    // coordinate as a (hi, lo) float pair so differences keep full accuracy
    __shared__ float sx1h[kStage], sx1l[kStage], sy1h[kStage], sy1l[kStage];
    __shared__ float sx2h[kStage], sx2l[kStage], sy2h[kStage], sy2l[kStage];
    __shared__ float slen[kStage];
    __shared__ float ssg[3][kStage], smg[3][kStage];
    __shared__ int sseg[kStage], sidx[kStage];
    const DevTree32 &t = a.t;
    Tile tl = a.items[blockIdx.x];
    const int leaf = tl.leaf;
    const double cxB = a.t64.cc[2 * leaf], cyB = a.t64.cc[2 * leaf + 1];
    const int j = threadIdx.x;
    bool act;
    double qx64 = 0.0, qy64 = 0.0;
    int own1 = -1, own2 = -1, r = 0, c = 0, ti = 0;
    if (MODE == 0) {
        act = j < tl.nr * tl.nc;
        if (act) {
            r = tl.r0 + j / tl.nc;
            c = tl.c0 + j % tl.nc;
            qx64 = a.vp.x0 + (c + 0.5) * a.vp.dx;
            qy64 = a.vp.y0 + (r + 0.5) * a.vp.dy;
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
        float iw = t.iw[leaf];
        float2 z = make_float2(q.x * iw, q.y * iw);
        const float2 *Lc = a.L + (size_t)leaf * 3 * P1;
        float2 s0 = Lc[P1 - 1], s1 = Lc[2 * P1 - 1], s2 = Lc[3 * P1 - 1];
        for (int k = P1 - 2; k >= 0; --k) {
            s0 = fadd(fmul(s0, z), Lc[k]);
            s1 = fadd(fmul(s1, z), Lc[P1 + k]);
            s2 = fadd(fmul(s2, z), Lc[2 * P1 + k]);
        }
        float e0 = s0.x, e1 = s1.x, e2 = s2.x;
        // M2P over list 3 (Eq. 61)
        for (int e = t.w_ptr[leaf]; e < t.w_ptr[leaf + 1]; ++e) {
            int src = t.w_idx[e];
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
        u0 = e0 * kInv2PiF;
        u1 = e1 * kInv2PiF;
        u2 = e2 * kInv2PiF;
    }
    // P2P over list 1 (App. D)
    for (int e = t.u_ptr[leaf]; e < t.u_ptr[leaf + 1]; ++e) {
        const int src = t.u_idx[e];
        const int p0 = t.pstart[src], pn = t.pcount[src];
        for (int base = 0; base < pn; base += kStage) {
            int cnt = min(kStage, pn - base);
            __syncthreads();
            for (int s = threadIdx.x; s < cnt; s += blockDim.x) {
                int i = p0 + base + s;
                const double *P = a.t64.pc + 4 * (size_t)i;
                split2(P[0] - cxB, sx1h[s], sx1l[s]);
                split2(P[1] - cyB, sy1h[s], sy1l[s]);
                split2(P[2] - cxB, sx2h[s], sx2l[s]);
                split2(P[3] - cyB, sy2h[s], sy2l[s]);
                slen[s] = t.plen[i];
                int seg = t.pseg[i];
                float wgt = -t.pw[i] * kInv2PiF;
                for (int ch = 0; ch < 3; ++ch) {
                    ssg[ch][s] = a.use_s ? wgt * a.sb[3 * (size_t)seg + ch] : 0.f;
                    smg[ch][s] = a.use_m ? wgt * a.mb[3 * (size_t)seg + ch] : 0.f;
                }
                sseg[s] = seg;
                sidx[s] = i;
            }
            __syncthreads();
            if (act) {
                for (int s = 0; s < cnt; ++s) {
                    float ax = (sx1h[s] - qxh) + (sx1l[s] - qxl), ay = (sy1h[s] - qyh) + (sy1l[s] - qyl);
                    float bx = (sx2h[s] - qxh) + (sx2l[s] - qxl), by = (sy2h[s] - qyh) + (sy2l[s] - qyl);
                    float len = slen[s];
                    float cr = ax * by - ay * bx;
                    float dt = ax * bx + ay * by;
                    bool own = (sseg[s] == own1) || (sseg[s] == own2);
                    float ilog, phi;
                    if (!own && dt < 0.f && fabsf(cr) < kNearFallback * len * len) {
                        // near-singular: the side of the curve is decided in FP64
                        const double *P = a.t64.pc + 4 * (size_t)sidx[s];
                        double il64, ph64;
                        seg_ilog_phi_f64(qx64, qy64, P[0], P[1], P[2], P[3], false, il64, ph64);
                        ilog = (float)il64;
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
        size_t o = 3 * ((size_t)r * a.vp.width + c);
        float u[3] = {u0, u1, u2};
        for (int ch = 0; ch < 3; ++ch) {
            if (a.rgb) {
                if (a.rgb_dtype == DC_F64) static_cast<double *>(a.rgb)[o + ch] = (double)u[ch];
                else static_cast<float *>(a.rgb)[o + ch] = u[ch];
            }
            if (a.rgb8) a.rgb8[o + ch] = quant8(u[ch]);
        }
    } else {
        int o = a.perm[ti];
        a.out[3 * (size_t)o + 0] = u0;
        a.out[3 * (size_t)o + 1] = u1;
        a.out[3 * (size_t)o + 2] = u2;
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
    return t;
}

dc_status Fmm::Impl::build32(const Geometry &G, cudaStream_t st, std::string &err) {
    const Tree &T = tree;
    const int nC = T.n_cells();
    std::vector<float> iw(nC), logw(nC);
    std::vector<double> ccx(nC), ccy(nC);
    for (int c = 0; c < nC; ++c) {
        double w = T.width(c);
        iw[c] = (float)(1.0 / w);
        logw[c] = (float)std::log(w);
        ccx[c] = T.cx(c);
        ccy[c] = T.cy(c);
    }
    const size_t np = T.pc_seg.size();
    std::vector<float4> pcf(np);
    std::vector<float> pwf(np), plf(np);
    std::vector<int> owner(np, -1);
    for (int c = 0; c < nC; ++c)
        for (int i = T.piece_start[c]; i < T.piece_start[c] + T.piece_count[c]; ++i) owner[i] = c;
    for (size_t i = 0; i < np; ++i) {
        const double *q = &T.pc_xy[4 * i];
        int c = owner[i];
        pcf[i] = make_float4((float)(q[0] - ccx[c]), (float)(q[1] - ccy[c]), (float)(q[2] - ccx[c]),
                             (float)(q[3] - ccy[c]));
        pwf[i] = (float)G.seg_w[T.pc_seg[i]];
        plf[i] = (float)std::hypot(q[2] - q[0], q[3] - q[1]);
    }
    auto offsets = [&](const std::vector<int> &ptr, const std::vector<int> &idx) {
        std::vector<float2> o(idx.size());
        for (int c = 0; c + 1 < (int)ptr.size(); ++c)
            for (int e = ptr[c]; e < ptr[c + 1]; ++e)
                o[e] = make_float2((float)(ccx[idx[e]] - ccx[c]), (float)(ccy[idx[e]] - ccy[c]));
        return o;
    };
    std::vector<float2> uo = offsets(T.u_ptr, T.u_idx), wo = offsets(T.w_ptr, T.w_idx),
                        xo = offsets(T.x_ptr, T.x_idx);
    // node targets relative to their leaf; work items of <= 64 targets
    const int N = G.n_nodes();
    std::vector<double> nxy(2 * size_t(N));
    std::vector<int> start(nC), cnt(nC);
    cudaError_t e = cudaMemcpyAsync(nxy.data(), nt_xy.ptr, nxy.size() * sizeof(double),
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(start.data(), nt_start.ptr, nC * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cnt.data(), nt_count.ptr, nC * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        err = std::string("fmm32 build: ") + cudaGetErrorString(e);
        return DC_ERR_CUDA;
    }
    std::vector<float2> q32(N);
    std::vector<Tile> items;
    for (int c = 0; c < nC; ++c) {
        for (int j = start[c]; j < start[c] + cnt[c]; ++j)
            q32[j] = make_float2((float)(nxy[2 * j] - ccx[c]), (float)(nxy[2 * j + 1] - ccy[c]));
        for (int j = 0; j < cnt[c]; j += 64) items.push_back({c, start[c] + j, 0, std::min(64, cnt[c] - j), 0});
    }
    n_nt_items = int(items.size());
    if ((e = up(iw32, iw, st)) != cudaSuccess || (e = up(logw32, logw, st)) != cudaSuccess ||
        (e = up(pc32, pcf, st)) != cudaSuccess || (e = up(pw32, pwf, st)) != cudaSuccess ||
        (e = up(plen32, plf, st)) != cudaSuccess || (e = up(uoff32, uo, st)) != cudaSuccess ||
        (e = up(woff32, wo, st)) != cudaSuccess || (e = up(xoff32, xo, st)) != cudaSuccess ||
        (e = up(nt_q32, q32, st)) != cudaSuccess || (e = up(nt_items, items, st)) != cudaSuccess ||
        (e = to_f32(m2m32, m2m, st)) != cudaSuccess || (e = to_f32(l2l32, l2l, st)) != cudaSuccess ||
        (e = to_f32(m2l32, m2l, st)) != cudaSuccess ||
        (e = M32.alloc((size_t)nC * 3 * P1)) != cudaSuccess ||
        (e = L32.alloc((size_t)nC * 3 * P1)) != cudaSuccess ||
        (e = sbar32.alloc((size_t)3 * D->S)) != cudaSuccess ||
        (e = mbar32.alloc((size_t)3 * D->S)) != cudaSuccess) {
        err = std::string("fmm32 allocation: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? DC_ERR_OOM : DC_ERR_CUDA;
    }
    cudaMemsetAsync(sbar32.ptr, 0, sbar32.bytes(), st);
    cudaMemsetAsync(mbar32.ptr, 0, mbar32.bytes(), st);
    return DC_OK;
}

cudaError_t Fmm::Impl::interp32(const double *node_vals, float *seg_vals, cudaStream_t st) {
    int th = 256;
    interp32_kernel<<<(D->S + th - 1) / th, th, 0, st>>>(D->lambda.ptr, node_vals, seg_vals, D->S,
                                                        D->s, D->g); note_launch();
    return cudaGetLastError();
}

cudaError_t Fmm::Impl::to_f32_density(const double *sb, const double *mb, cudaStream_t st) {
    int n = 3 * D->S, th = 256;
    d2f_kernel<<<(n + th - 1) / th, th, 0, st>>>(sb, mb, sbar32.ptr, mbar32.ptr, n); note_launch();
    return cudaGetLastError();
}

cudaError_t Fmm::Impl::passes32(const float *sb, const float *mb, int use_s, int use_m,
                                cudaStream_t st) {
    const int nC = tree.n_cells();
    size_t ebytes = (size_t)nC * 3 * P1 * sizeof(float2);
    cudaError_t e;
    if ((e = cudaMemsetAsync(M32.ptr, 0, ebytes, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(L32.ptr, 0, ebytes, st)) != cudaSuccess) return e;
    DevTree32 t = dt32();
    int th = ((P1 + 31) / 32) * 32;
    if (n_p2m > 0)
        p2m32_kernel<<<n_p2m, th, 0, st>>>(t, p2m_leaves.ptr, sb, mb, use_s, use_m, P1, M32.ptr); note_launch();
    for (int l = tree.depth - 1; l >= 2; --l) {
        int lo = tree.level_start[l], hi = tree.level_start[l + 1];
        if (hi > lo) m2m32_kernel<<<hi - lo, th, 0, st>>>(t, lo, P1, m2m32.ptr, M32.ptr); note_launch();
    }
    for (int l = 2; l <= tree.depth; ++l) {
        int lo = tree.level_start[l], hi = tree.level_start[l + 1];
        if (hi > lo)
            down32_kernel<<<hi - lo, th, 0, st>>>(t, lo, l, P1, l2l32.ptr, m2l32.ptr, M32.ptr, sb, mb,
                                                   use_s, use_m, L32.ptr); note_launch();
    }
    return cudaGetLastError();
}

cudaError_t Fmm::Impl::apply_nodes32(const double *x, double *y, bool single, cudaStream_t st) {
    cudaError_t e = interp32(x, single ? sbar32.ptr : mbar32.ptr, st);
    if (e != cudaSuccess) return e;
    int us = single ? 1 : 0, um = single ? 0 : 1;
    if ((e = passes32(sbar32.ptr, mbar32.ptr, us, um, st)) != cudaSuccess) return e;
    if (n_nt_items == 0) return cudaSuccess;
    EvalArgs32 a{};
    a.t = dt32();
    a.t64 = dt();
    a.items = nt_items.ptr;
    a.P1 = P1;
    a.M = M32.ptr;
    a.L = L32.ptr;
    a.sb = sbar32.ptr;
    a.mb = mbar32.ptr;
    a.use_s = us;
    a.use_m = um;
    a.q32 = nt_q32.ptr;
    a.q64 = nt_xy.ptr;
    a.own1 = nt_own1.ptr;
    a.own2 = nt_own2.ptr;
    a.perm = nt_perm.ptr;
    a.out = y;
    eval32_kernel<1><<<n_nt_items, 64, 0, st>>>(a); note_launch();
    return cudaGetLastError();
}

cudaError_t Fmm::Impl::render_tiles32(const VpDev &vp, int n_tiles, void *rgb, int rgb_dtype,
                                      unsigned char *rgb8, cudaStream_t st) {
    EvalArgs32 a{};
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
    a.vp = vp;
    a.rgb = rgb;
    a.rgb_dtype = rgb_dtype;
    a.rgb8 = rgb8;
    eval32_kernel<0><<<n_tiles, kEvThreads, 0, st>>>(a); note_launch();
    return cudaGetLastError();
}

cudaError_t Fmm::Impl::eval_points32(int n_items, double *out, cudaStream_t st) {
    EvalArgs32 a{};
    a.t = dt32();
    a.t64 = dt();
    a.items = pt_items.ptr;
    a.P1 = P1;
    a.M = M32.ptr;
    a.L = L32.ptr;
    a.sb = sbar32.ptr;
    a.mb = mbar32.ptr;
    a.use_s = 1;
    a.use_m = 1;
    a.q32 = pt_q32.ptr;
    a.q64 = pt_xy.ptr;
    a.perm = pt_perm.ptr;
    a.out = out;
    eval32_kernel<1><<<n_items, 64, 0, st>>>(a); note_launch();
    return cudaGetLastError();
}

}  // namespace dc
