// Up and down passes of the FMM (Alg. 8), templated on the real type, in
// the width-scaled basis described in fmm.cu.  Included by fmm.cu (double)
// and fmm32.cu (float); each includes it once.
//
//  p2m_kernel   leaves: outgoing moments of clipped segments (Eq. 60/76/77),
//               one thread per piece computing S_0..S_p by recurrence into
//               shared memory, then one thread per coefficient summing the
//               chunk in order (deterministic)
//  m2m_kernel   per level, parent from 4 children (Eq. 71)
//  m2l_kernel   all cells at once, persistent blocks: list 2 (Eq. 69) with
//               the 40 offset matrices reduced by the symmetries of the
//               square to 7 base matrices held in shared memory:
//               T(uB) = diag(u^-l) T(B) diag(u^-k), T(u conj B) = its
//               conjugate analogue, u in {1, i, -1, -i}
//  p2l_kernel   cells with a list 4: incoming coefficients of segments
//               (Eq. 62/78/79), chunked like p2m
//  l2l_kernel   per level: L = L_m2l + L2L(parent) (Eq. 73)
#pragma once

#include <cuda_runtime.h>

namespace dc {
namespace passes {

template <typename T> struct V2;
template <> struct V2<float> { using type = float2; };
template <> struct V2<double> { using type = double2; };

template <typename T> __device__ __forceinline__ typename V2<T>::type mk(T x, T y) {
    typename V2<T>::type r;
    r.x = x;
    r.y = y;
    return r;
}
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) {
    C r;
    r.x = a.x + b.x;
    r.y = a.y + b.y;
    return r;
}
template <typename C, typename T> __device__ __forceinline__ C cscl(C a, T s) {
    C r;
    r.x = a.x * s;
    r.y = a.y * s;
    return r;
}
template <typename C> __device__ __forceinline__ C cinv(C a) {
    auto d = 1 / (a.x * a.x + a.y * a.y);
    C r;
    r.x = a.x * d;
    r.y = -a.y * d;
    return r;
}
template <typename C> __device__ __forceinline__ void cfma(C &acc, C m, C v) {
    acc.x += m.x * v.x - m.y * v.y;
    acc.y += m.x * v.y + m.y * v.x;
}
// multiply by u^-n with u = i^r: i^(-r n)
template <typename C> __device__ __forceinline__ C rot_pow(C a, int rn) {
    C r;
    switch (rn & 3) {
        case 0: r = a; break;
        case 1: r.x = a.y; r.y = -a.x; break;       // times -i
        case 2: r.x = -a.x; r.y = -a.y; break;      // times -1
        default: r.x = -a.y; r.y = a.x; break;      // times i
    }
    return r;
}

__device__ __forceinline__ float tlog(float x) { return logf(x); }
__device__ __forceinline__ double tlog(double x) { return log(x); }
__device__ __forceinline__ float tatan2(float y, float x) { return atan2f(y, x); }
__device__ __forceinline__ double tatan2(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ float tlog1p(float x) { return log1pf(x); }
__device__ __forceinline__ double tlog1p(double x) { return log1p(x); }

// Piece endpoints relative to a cell centre, for either precision.
struct PiecesF64 {
    const double *pc;   // [np][4] absolute
    const double *cc;   // [cells][2] centres
    __device__ void rel(int i, int cell, int /*entry*/, const float2 * /*off*/, double &ax,
                        double &ay, double &bx, double &by) const {
        const double *q = pc + 4 * (size_t)i;
        double cx = cc[2 * cell], cy = cc[2 * cell + 1];
        ax = q[0] - cx;
        ay = q[1] - cy;
        bx = q[2] - cx;
        by = q[3] - cy;
    }
};
struct PiecesF32 {
    const float4 *pc;   // [np] relative to the owning leaf's centre
    __device__ void rel(int i, int /*cell*/, int entry, const float2 *off, float &ax, float &ay,
                        float &bx, float &by) const {
        float4 P = pc[i];
        float ox = 0.f, oy = 0.f;
        if (off) {
            ox = off[entry].x;
            oy = off[entry].y;
        }
        ax = P.x + ox;
        ay = P.y + oy;
        bx = P.z + ox;
        by = P.w + oy;
    }
};

template <typename T> struct TreeView {
    const T *iw;              // [cells] 1 / width
    const T *logw;            // [cells] log width
    const int *parent, *child0, *quad;
    const int *pstart, *pcount;
    const T *pw;              // [np] arc weight
    const T *plen;            // [np] chord length
    const int *pseg;
    const int *v_ptr, *v_idx, *v_code;   // list 2 with packed symmetry codes
    const int *x_ptr, *x_idx;            // list 4
    const float2 *x_off;                 // list-4 offsets (FP32 geometry only)
};

constexpr int kChunk = 64;

// ---------------------------------------------------------------- P2M --
template <typename T, typename PS>
__global__ void __launch_bounds__(kChunk) p2m_kernel(TreeView<T> t, PS ps, const int *__restrict__ leaves,
                                                     const T *__restrict__ sb, const T *__restrict__ mb,
                                                     int use_s, int use_m, int P1,
                                                     typename V2<T>::type *__restrict__ M) {
    using C = typename V2<T>::type;
    extern __shared__ unsigned char smem_raw[];
    C *S = reinterpret_cast<C *>(smem_raw);                 // [kChunk][P1 + 1], S_{-1} at 0
    T *om = reinterpret_cast<T *>(S + kChunk * (P1 + 1));   // [kChunk]
    C *wr = reinterpret_cast<C *>(om + kChunk);             // [kChunk]
    int *sg = reinterpret_cast<int *>(wr + kChunk);         // [kChunk]
    const int cell = leaves[blockIdx.x];
    const int tid = threadIdx.x;
    const T iw = t.iw[cell];
    C acc[3];
    for (int c = 0; c < 3; ++c) acc[c] = mk<T>(0, 0);
    const int p0 = t.pstart[cell], pn = t.pcount[cell];
    for (int base = 0; base < pn; base += kChunk) {
        int cnt = min(kChunk, pn - base);
        __syncthreads();
        if (tid < cnt) {
            int i = p0 + base + tid;
            T ax, ay, bx, by;
            ps.rel(i, cell, 0, nullptr, ax, ay, bx, by);
            C a = mk<T>(ax * iw, ay * iw), b = mk<T>(bx * iw, by * iw);
            T len = t.plen[i];
            om[tid] = t.pw[i] * len;
            T il = iw / len;
            wr[tid] = mk<T>((bx - ax) * il, (by - ay) * il);
            sg[tid] = t.pseg[i];
            C *row = S + tid * (P1 + 1);
            row[0] = mk<T>(0, 0);              // S_{-1}
            C s = mk<T>(1, 0), ap = mk<T>(1, 0);
            row[1] = s;                         // S_0
            for (int k = 1; k < P1; ++k) {
                ap = cmul(ap, a);
                s = cadd(cmul(b, s), ap);
                row[k + 1] = s;
            }
        }
        __syncthreads();
        if (tid < P1) {
            const int k = tid;
            for (int j = 0; j < cnt; ++j) {
                const C *row = S + j * (P1 + 1);
                C cg = cscl(row[k + 1], om[j] / (k + 1));
                C t1 = cmul(wr[j], row[k]);
                C cf = mk<T>(t1.y * om[j], -t1.x * om[j]);   // -i (w/r) S_{k-1} om
                int seg = sg[j];
                for (int c = 0; c < 3; ++c) {
                    T s = use_s ? sb[3 * (size_t)seg + c] : T(0);
                    T mu = use_m ? mb[3 * (size_t)seg + c] : T(0);
                    acc[c].x += s * cg.x + mu * cf.x;
                    acc[c].y += s * cg.y + mu * cf.y;
                }
            }
        }
    }
    if (tid < P1)
        for (int c = 0; c < 3; ++c) M[((size_t)cell * 3 + c) * P1 + tid] = acc[c];
}

// ---------------------------------------------------------------- M2M --
template <typename T>
__global__ void m2m_kernel(TreeView<T> t, const int *__restrict__ cells, int P1,
                           const typename V2<T>::type *__restrict__ tab,
                           typename V2<T>::type *__restrict__ M) {
    using C = typename V2<T>::type;
    const int cell = cells[blockIdx.x];
    const int k = threadIdx.x;
    const int ch0 = t.child0[cell];
    if (k >= P1) return;
    C acc[3];
    for (int c = 0; c < 3; ++c) acc[c] = mk<T>(0, 0);
    for (int q = 0; q < 4; ++q) {
        const C *Tq = tab + ((size_t)q * P1 + k) * P1;
        const C *src = M + (size_t)(ch0 + q) * 3 * P1;
        for (int j = 0; j <= k; ++j) {
            C tq = Tq[j];
            for (int c = 0; c < 3; ++c) cfma(acc[c], tq, src[c * P1 + j]);
        }
    }
    for (int c = 0; c < 3; ++c) M[((size_t)cell * 3 + c) * P1 + k] = acc[c];
}

// ---------------------------------------------------------------- M2L --
// v_code of a list-2 entry: base matrix b (0..6) | rotation r << 3 |
// conjugation << 5.  The 7 base tables are transposed: base[b][k][l].
constexpr int kM2LSlots = 4;   // target cells per block (one warp each)

template <typename T>
__global__ void __launch_bounds__(32 * kM2LSlots) m2l_kernel(TreeView<T> t, const int *__restrict__ cells,
                                                             int n_cells, int P1,
                                                             const typename V2<T>::type *__restrict__ base,
                                                             const typename V2<T>::type *__restrict__ M,
                                                             typename V2<T>::type *__restrict__ Lout) {
    using C = typename V2<T>::type;
    extern __shared__ unsigned char smem_raw[];
    C *B = reinterpret_cast<C *>(smem_raw);   // [7][P1][P1]
    for (int i = threadIdx.x; i < 7 * P1 * P1; i += blockDim.x) B[i] = base[i];
    __syncthreads();
    const int slot = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int ci = blockIdx.x * kM2LSlots + slot; ci < n_cells; ci += gridDim.x * kM2LSlots) {
        const int cell = cells[ci];
        if (l >= P1) continue;
        C acc[3];
        for (int c = 0; c < 3; ++c) acc[c] = mk<T>(0, 0);
        const T mlogw = -t.logw[cell];
        for (int e = t.v_ptr[cell]; e < t.v_ptr[cell + 1]; ++e) {
            const int src = t.v_idx[e], code = t.v_code[e];
            const int b = code & 7, r = (code >> 3) & 3, cj = code >> 5;
            const C *Tb = B + (size_t)b * P1 * P1;
            const C *ms = M + (size_t)src * 3 * P1;
            C part[3];
            for (int c = 0; c < 3; ++c) part[c] = mk<T>(0, 0);
            for (int k = 0; k < P1; ++k) {
                C tk = Tb[k * P1 + l];
                for (int c = 0; c < 3; ++c) {
                    C m = rot_pow(ms[c * P1 + k], r * k);
                    if (cj) m.y = -m.y;
                    cfma(part[c], tk, m);
                }
            }
            for (int c = 0; c < 3; ++c) {
                C v = part[c];
                if (cj) v.y = -v.y;
                v = rot_pow(v, r * l);
                acc[c].x += v.x;
                acc[c].y += v.y;
                if (l == 0) acc[c].x += mlogw * ms[c * P1].x;   // Mt_0 is real
            }
        }
        for (int c = 0; c < 3; ++c) Lout[((size_t)cell * 3 + c) * P1 + l] = acc[c];
    }
}

// ---------------------------------------------------------------- P2L --
template <typename T, typename PS>
__global__ void __launch_bounds__(kChunk) p2l_kernel(TreeView<T> t, PS ps, const int *__restrict__ cells,
                                                     const T *__restrict__ sb, const T *__restrict__ mb,
                                                     int use_s, int use_m, int P1,
                                                     typename V2<T>::type *__restrict__ Lout) {
    using C = typename V2<T>::type;
    extern __shared__ unsigned char smem_raw[];
    C *G = reinterpret_cast<C *>(smem_raw);          // [kChunk][P1] sigma coefficients
    C *F = G + kChunk * P1;                          // [kChunk][P1] mu coefficients
    int *sg = reinterpret_cast<int *>(F + kChunk * P1);
    const int cell = cells[blockIdx.x];
    const int tid = threadIdx.x;
    const T iw = t.iw[cell], w = 1 / iw, logw = t.logw[cell];
    C acc[3];
    for (int c = 0; c < 3; ++c) acc[c] = mk<T>(0, 0);
    for (int e = t.x_ptr[cell]; e < t.x_ptr[cell + 1]; ++e) {
        const int src = t.x_idx[e];
        const int p0 = t.pstart[src], pn = t.pcount[src];
        for (int base = 0; base < pn; base += kChunk) {
            int cnt = min(kChunk, pn - base);
            __syncthreads();
            if (tid < cnt) {
                int i = p0 + base + tid;
                T ax, ay, bx, by;
                ps.rel(i, cell, e, t.x_off, ax, ay, bx, by);
                C a = mk<T>(ax * iw, ay * iw), b = mk<T>(bx * iw, by * iw);   // scaled
                T len = t.plen[i], om = t.pw[i];
                C wv = mk<T>((bx - ax) / len, (by - ay) / len);
                // log(b/a) on the continuous branch (|arg| < pi: separated)
                C d = mk<T>(b.x - a.x, b.y - a.y), s = mk<T>(b.x + a.x, b.y + a.y);
                T aa = a.x * a.x + a.y * a.y;
                C lba = mk<T>(T(0.5) * tlog1p((d.x * s.x + d.y * s.y) / aa),
                              tatan2(a.x * b.y - a.y * b.x, a.x * b.x + a.y * b.y));
                C *g = G + tid * P1, *f = F + tid * P1;
                // l = 0: omega [ l (1 - log a) - conj(w) b w_cell log(b/a) ] and i log(b/a)
                {
                    C la = mk<T>(T(0.5) * tlog(aa) + logw, tatan2(a.y, a.x));
                    C wb = cmul(mk<T>(wv.x, -wv.y), mk<T>(b.x * w, b.y * w));
                    C t2 = cmul(wb, lba);
                    g[0] = mk<T>(om * (len * (1 - la.x) - t2.x), om * (-len * la.y - t2.y));
                    f[0] = mk<T>(-om * lba.y, om * lba.x);
                }
                if (P1 > 1) {
                    C t2 = cmul(mk<T>(wv.x, -wv.y), lba);
                    g[1] = cscl(t2, om * w);
                }
                C al = cinv(a), be = cinv(b), ab = cmul(al, be);
                C iwv = mk<T>(-wv.y, wv.x);                 // i w
                C fb = cscl(cmul(iwv, ab), om * len * iw);  // F factor, times T_{l-1} / l
                C gb = cscl(ab, om * len);                  // G factor, times T_{l-2} / (l (l-1))
                // T_m = sum_j al^j be^(m-j): T_0 = 1, T_m = al T_{m-1} + be^m
                C Tm = mk<T>(1, 0), bp = mk<T>(1, 0);       // T_0
                if (P1 > 1) f[1] = fb;                       // l = 1: T_0 / 1
                for (int l = 2; l < P1; ++l) {
                    // here Tm = T_{l-2}
                    g[l] = cscl(cmul(gb, Tm), T(1) / (T(l) * (l - 1)));
                    bp = cmul(bp, be);
                    Tm = cadd(cmul(al, Tm), bp);             // T_{l-1}
                    f[l] = cscl(cmul(fb, Tm), T(1) / T(l));
                }
                sg[tid] = t.pseg[i];
            }
            __syncthreads();
            if (tid < P1) {
                for (int j = 0; j < cnt; ++j) {
                    C cg = G[j * P1 + tid], cf = F[j * P1 + tid];
                    int seg = sg[j];
                    for (int c = 0; c < 3; ++c) {
                        T s = use_s ? sb[3 * (size_t)seg + c] : T(0);
                        T mu = use_m ? mb[3 * (size_t)seg + c] : T(0);
                        acc[c].x += s * cg.x + mu * cf.x;
                        acc[c].y += s * cg.y + mu * cf.y;
                    }
                }
            }
        }
    }
    if (tid < P1)
        for (int c = 0; c < 3; ++c) {
            C *o = Lout + ((size_t)cell * 3 + c) * P1 + tid;
            o->x += acc[c].x;
            o->y += acc[c].y;
        }
}

// ---------------------------------------------------------------- L2L --
template <typename T>
__global__ void l2l_kernel(TreeView<T> t, const int *__restrict__ cells, int n, int level, int P1,
                           const typename V2<T>::type *__restrict__ tab,
                           const typename V2<T>::type *__restrict__ Lm2l,
                           typename V2<T>::type *__restrict__ L) {
    using C = typename V2<T>::type;
    const int idx = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int l = threadIdx.x & 31;
    if (idx >= n || l >= P1) return;
    const int cell = cells[idx];
    C acc[3];
    for (int c = 0; c < 3; ++c) acc[c] = Lm2l[((size_t)cell * 3 + c) * P1 + l];
    if (level >= 3) {
        const int par = t.parent[cell], q = t.quad[cell];
        const C *Tq = tab + ((size_t)q * P1 + l) * P1;
        const C *src = L + (size_t)par * 3 * P1;
        for (int k = l; k < P1; ++k) {
            C tq = Tq[k];
            for (int c = 0; c < 3; ++c) cfma(acc[c], tq, src[c * P1 + k]);
        }
    }
    for (int c = 0; c < 3; ++c) L[((size_t)cell * 3 + c) * P1 + l] = acc[c];
}

template <typename T> inline size_t p2m_smem(int P1) {
    using C = typename V2<T>::type;
    return kChunk * (P1 + 1) * sizeof(C) + kChunk * sizeof(T) + kChunk * sizeof(C) + kChunk * sizeof(int);
}
template <typename T> inline size_t p2l_smem(int P1) {
    using C = typename V2<T>::type;
    return 2 * kChunk * P1 * sizeof(C) + kChunk * sizeof(int);
}
template <typename T> inline size_t m2l_smem(int P1) {
    using C = typename V2<T>::type;
    return 7 * (size_t)P1 * P1 * sizeof(C);
}

}  // namespace passes
}  // namespace dc
