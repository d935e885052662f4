// Up and down passes of the FMM (Alg. 8), templated on the real type, in
// the width-scaled basis described in fmm.cu.  Included by fmm.cu (double)
// and fmm32.cu (float); each includes it once.
//
//  p2m_kernel   leaves: outgoing moments of clipped segments (Eq. 60/76/77),
//               one thread per piece computing S_0..S_p by recurrence into
//               shared memory, then one thread per coefficient summing the
//               chunk in order (deterministic)
//               (or from stored per-piece coefficient rows)
//  m2m_kernel   per level, parent from its 4 children (Eq. 71)
//  m2m_multi_kernel  every inner cell straight from its leaves (all levels
//               in one launch, no chain of dependent levels)
//  m2l_kernel   all cells at once, persistent blocks: list 2 (Eq. 69) with
//               the 40 offset matrices reduced by the symmetries of the
//               square to 7 base matrices held in shared memory:
//               T(uB) = diag(u^-l) T(B) diag(u^-k), T(u conj B) = its
//               conjugate analogue, u in {1, i, -1, -i}
//  p2l_kernel   cells with a list 4: incoming coefficients of segments
//               (Eq. 62/78/79), chunked like p2m
//  l2l_kernel   per level: L = L_m2l + L2L(parent) (Eq. 73)
//  walk_kernel  the same recursion for listed leaves only, walking down from
//               each leaf's level-2 ancestor (one launch for all levels)
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
// P2M of listed leaves, one block per leaf.
template <typename T, typename PS>
__global__ void __launch_bounds__(kChunk) p2m_kernel(TreeView<T> t, PS ps, const int *__restrict__ leaves,
                                                     const T *__restrict__ sb, const T *__restrict__ mb,
                                                     int use_s, int use_m, int P1,
                                                     typename V2<T>::type *__restrict__ M,
                                                     const typename V2<T>::type *__restrict__ rows_g = nullptr,
                                                     const typename V2<T>::type *__restrict__ rows_f = nullptr,
                                                     typename V2<T>::type *__restrict__ out_g = nullptr,
                                                     typename V2<T>::type *__restrict__ out_f = nullptr) {
    // rows_g / rows_f: stored per-piece coefficients [pieces][P1] (then no
    // recurrence runs); out_g / out_f: write those coefficients instead of
    // forming expansions.
    using C = typename V2<T>::type;
    extern __shared__ unsigned char smem_raw[];
    C *S = reinterpret_cast<C *>(smem_raw);                 // [kChunk][P1 + 1], S_{-1} at 0
    T *om = reinterpret_cast<T *>(S + kChunk * (P1 + 1));   // [kChunk]
    C *wr = reinterpret_cast<C *>(om + kChunk);             // [kChunk]
    int *sg = reinterpret_cast<int *>(wr + kChunk);         // [kChunk]
    const int cell = leaves[blockIdx.x];
    const int tid = threadIdx.x;
    // phase 2: thread tid sums coefficient k = tid % P1 over the pieces
    // j = grp, grp + ngrp, ... of each chunk (grp = tid / P1)
    const int ngrp = kChunk / P1, grp = tid / P1, k = tid - grp * P1;
    const T iw = t.iw[cell];
    C acc[3];
    for (int c = 0; c < 3; ++c) acc[c] = mk<T>(0, 0);
    const int p0 = t.pstart[cell], pn = t.pcount[cell];
    for (int base = 0; base < pn; base += kChunk) {
        int cnt = min(kChunk, pn - base);
        __syncthreads();
        if (tid < cnt && rows_g) sg[tid] = t.pseg[p0 + base + tid];
        if (tid < cnt && !rows_g) {
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
            for (int q = 1; q < P1; ++q) {
                ap = cmul(ap, a);
                s = cadd(cmul(b, s), ap);
                row[q + 1] = s;
            }
        }
        __syncthreads();
        if (grp < ngrp) {
            for (int j = grp; j < cnt; j += ngrp) {
                const size_t ri = (size_t)(p0 + base + j) * P1 + k;
                C cg, cf;
                if (rows_g) {
                    cg = rows_g[ri];
                    cf = rows_f ? rows_f[ri] : mk<T>(0, 0);
                } else {
                    const C *row = S + j * (P1 + 1);
                    cg = cscl(row[k + 1], om[j] / (k + 1));
                    C t1 = cmul(wr[j], row[k]);
                    cf = mk<T>(t1.y * om[j], -t1.x * om[j]);   // -i (w/r) S_{k-1} om
                }
                if (out_g) {
                    out_g[ri] = cg;
                    out_f[ri] = cf;
                    continue;
                }
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
    if (out_g) return;
    // the groups' partial sums, added in group order
    __syncthreads();
    if (grp < ngrp)
        for (int c = 0; c < 3; ++c) S[(grp * 3 + c) * P1 + k] = acc[c];
    __syncthreads();
    if (tid < P1)
        for (int c = 0; c < 3; ++c) {
            C a = S[c * P1 + tid];
            for (int q = 1; q < ngrp; ++q) a = cadd(a, S[(q * 3 + c) * P1 + tid]);
            M[((size_t)cell * 3 + c) * P1 + tid] = a;
        }
}

// ---------------------------------------------------------------- M2M --
// One level: each listed cell's expansion from its four children (Eq. 71),
// one warp per cell, lane k holds coefficient k (P1 <= 32).
constexpr int kLevelWarps = 4;

template <typename T>
__global__ void __launch_bounds__(32 * kLevelWarps) m2m_kernel(const int *__restrict__ child0,
                                                               const int *__restrict__ cells, int n, int P1,
                                                               const typename V2<T>::type *__restrict__ tab,
                                                               typename V2<T>::type *__restrict__ M) {
    using C = typename V2<T>::type;
    const int idx = blockIdx.x * kLevelWarps + (threadIdx.x >> 5);
    const int k = threadIdx.x & 31;
    if (idx >= n || k >= P1) return;
    const int cell = cells[idx];
    const int ch0 = child0[cell];
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

// M2M from each leaf straight to every listed ancestor, all levels in one
// launch: Eq. 71 with the shift d = (c_leaf - c_anc) / w_anc and the scale
// rho = w_leaf / w_anc of the width-scaled basis (pair_geo = (d, rho, 0)),
//   Mt_anc[k] += sum_{j <= k} C(k, j) d^(k - j) rho^j Mt_leaf[j].
// No level waits for another (each leaf moment is translated once per
// ancestor instead of through the chain of parents).  One warp per chunk of
// up to kMultiLeaves (ancestor, leaf) pairs; a chunk writes the ancestor's
// expansion when it is the cell's only chunk, else a partial sum that
// m2m_reduce_kernel adds up in chunk order.  For P1 <= 16 the half-warps
// take alternate pairs (lane k + 16 h holds coefficient k of pair 2 i + h)
// and are added at the end; above 16 lane k holds coefficient k of every
// pair.  The binomial table is staged in shared memory.
constexpr int kMultiLeaves = 16;
constexpr int kMultiWarps = 4;

template <typename T>
__global__ void __launch_bounds__(32 * kMultiWarps) m2m_multi_kernel(const float4 *__restrict__ pair_geo,
                                                                     const int4 *__restrict__ chunks, int n_chunks,
                                                                     const int *__restrict__ pair_leaf, int P1,
                                                                     const T *__restrict__ binom,
                                                                     typename V2<T>::type *__restrict__ M,
                                                                     typename V2<T>::type *__restrict__ partial) {
    using C = typename V2<T>::type;
    __shared__ C zp[kMultiWarps][32];
    __shared__ T rp[kMultiWarps][32];
    __shared__ C ms[kMultiWarps][2][96];
    __shared__ T sbin[32 * 32];
    for (int i = threadIdx.x; i < P1 * 32; i += blockDim.x) sbin[i] = binom[i];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ci = blockIdx.x * kMultiWarps + warp;
    if (ci >= n_chunks) return;
    const int4 ch = chunks[ci];          // (ancestor, first pair, pairs, partial slot or -1)
    const int anc = ch.x;
    const int halves = P1 <= 16 ? 2 : 1;
    const int span = 32 / halves;                       // lanes per pair
    const int h = halves == 2 ? lane >> 4 : 0, k = lane - h * span;
    C acc[3];
    for (int c = 0; c < 3; ++c) acc[c] = mk<T>(0, 0);
    const int nM = 3 * P1;
    for (int e0 = ch.y; e0 < ch.y + ch.z; e0 += halves) {
        const int e = e0 + h;
        const bool has = e < ch.y + ch.z;
        // d^k and rho^k by binary powering (the pair's shift d and scale rho
        // were formed once per drawing)
        const float4 geo = has ? pair_geo[e] : make_float4(0.f, 0.f, 0.f, 0.f);
        const C d = mk<T>((T)geo.x, (T)geo.y);
        const T rho = (T)geo.z;
        C pz = mk<T>(1, 0), bz = d;
        T pr = 1, br = rho;
        for (int bit = 1; bit < 32; bit <<= 1) {
            if (k & bit) {
                pz = cmul(pz, bz);
                pr *= br;
            }
            bz = cmul(bz, bz);
            br *= br;
        }
        __syncwarp();
        zp[warp][lane] = pz;                         // [h][k] = lane
        rp[warp][lane] = pr;
        if (has) {
            const C *src = M + (size_t)pair_leaf[e] * nM;
            for (int i = k; i < nM; i += span) ms[warp][h][i] = src[i];
        }
        __syncwarp();
        if (has && k < P1) {
            const T *bk = sbin + k * 32;
            const C *z = zp[warp] + h * span;
            const T *r = rp[warp] + h * span;
            const C *m = ms[warp][h];
            for (int j = 0; j <= k; ++j) {
                const C co = cscl(z[k - j], bk[j] * r[j]);
                for (int c = 0; c < 3; ++c) cfma(acc[c], co, m[c * P1 + j]);
            }
        }
    }
    if (halves == 2)
        for (int c = 0; c < 3; ++c) {
            acc[c].x += __shfl_xor_sync(0xffffffffu, acc[c].x, 16);
            acc[c].y += __shfl_xor_sync(0xffffffffu, acc[c].y, 16);
        }
    if (h == 0 && k < P1) {
        C *dst = ch.w < 0 ? M + (size_t)anc * nM : partial + (size_t)ch.w * nM;
        for (int c = 0; c < 3; ++c) dst[c * P1 + k] = acc[c];
    }
}

// Cells whose leaves span several chunks: M = sum of the chunk partials in
// chunk order (deterministic).  red = (cell, first slot, slots).  One block
// per cell: slice s of the kReduceThreads / (3 P1) slices sums the slots
// s, s + S, ... of every coefficient, and the slices are added in order.
constexpr int kReduceThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kReduceThreads) m2m_reduce_kernel(const int4 *__restrict__ red, int n, int P1,
                                                                    const typename V2<T>::type *__restrict__ partial,
                                                                    typename V2<T>::type *__restrict__ M) {
    using C = typename V2<T>::type;
    __shared__ C part[kReduceThreads];
    const int4 r = red[blockIdx.x];
    const int nM = 3 * P1;
    const int S = kReduceThreads / nM;
    const int s = threadIdx.x / nM, i = threadIdx.x - s * nM;
    if (s < S) {
        C a = mk<T>(0, 0);
        const C *p = partial + (size_t)r.y * nM + i;
#pragma unroll 4
        for (int q = s; q < r.z; q += S) a = cadd(a, p[(size_t)q * nM]);
        part[s * nM + i] = a;
    }
    __syncthreads();
    if (threadIdx.x < nM) {
        C a = part[threadIdx.x];
        for (int q = 1; q < S; ++q) a = cadd(a, part[q * nM + threadIdx.x]);
        M[(size_t)r.x * nM + threadIdx.x] = a;
    }
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

// M2L for low orders in FP32 (P1 <= 21, the inner operator of the
// iterative refinement).  The 56 (base, rotation, conjugation) variants are
// expanded into full tables in shared memory,
//   F[b + 7 r + 28 cj][l][k] = (cj ? conj(B_b[k][l]) : B_b[k][l]) i^(-r (k + l)),
// which is the same linear map as the symmetric form of m2l_kernel, so a pair
// costs P1 x P1 complex multiply-adds per channel and no bookkeeping.  One
// warp per target cell: for P1 <= 16 lane l + 16 h sums the terms k = h,
// h + 2, ... of coefficient l and the halves are added at the end; above 16
// lane l sums all k.  The source moments of the pairs are copied into a
// per-warp ring of kM2LDepth shared-memory slots by asynchronous copies
// (cp.async), kM2LDepth - 1 pairs ahead of the products.
constexpr int kM2LSmallP1 = 21;
constexpr int kM2LSmallWarps = 16;
constexpr int kM2LDepth = 4;

inline size_t m2l_small_smem(int P1) {
    return (56 * (size_t)P1 * P1 + kM2LSmallWarps * kM2LDepth * 64) * sizeof(float2);
}

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

template <typename V> __device__ __forceinline__ void cp_async_any(V *smem, const V *gmem) {
    if (sizeof(V) == 16) cp_async16(smem, gmem);
    else cp_async8(smem, gmem);
}

// dst[i] = src[i] for i < n (shared <- global), thread t of a block of
// `stride` threads, by asynchronous copies so that every element is in
// flight at once; the caller then runs cp_async_commit(), cp_async_wait<0>()
// and __syncthreads().  Elements of 8 or 16 bytes, both arrays aligned.
template <typename V>
__device__ __forceinline__ void stage_async(V *dst, const V *src, int n, int t, int stride) {
    static_assert(sizeof(V) == 8 || sizeof(V) == 16, "8- or 16-byte elements");
    for (int i = t; i < n; i += stride) {
        if (sizeof(V) == 16) cp_async16(dst + i, src + i);
        else cp_async8(dst + i, src + i);
    }
}

static __global__ void __launch_bounds__(32 * kM2LSmallWarps) m2l_small_kernel(TreeView<float> t, const int *__restrict__ cells,
                                                                               int n_cells, int P1,
                                                                               const float2 *__restrict__ full,
                                                                               const float2 *__restrict__ M,
                                                                               float2 *__restrict__ Lout) {
    extern __shared__ unsigned char smem_raw[];
    float2 *Tf = reinterpret_cast<float2 *>(smem_raw);            // [56][P1][P1]
    float2 *stage = Tf + 56 * P1 * P1;                            // [warps][kM2LDepth][64]
    stage_async(Tf, full, 56 * P1 * P1, threadIdx.x, blockDim.x);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int halves = P1 <= 16 ? 2 : 1;
    const int l = halves == 2 ? (lane & 15) : lane, h = halves == 2 ? (lane >> 4) : 0;
    const int lr = min(l, P1 - 1);
    const int nM = 3 * P1;
    float2 *buf = stage + warp * kM2LDepth * 64;
    const float2 zero = make_float2(0.f, 0.f);
    // the first 32 entries of the list (source, symmetry code) are loaded
    // up front, one per lane, and passed around by shuffles
    int my_src = 0, my_code = 0;
    auto entry_src = [&](int e, int e0) {
        const int r = e - e0;
        const int v = __shfl_sync(0xffffffffu, my_src, r & 31);
        return r < 32 ? v : t.v_idx[e];
    };
    // copy the moments of list-2 entry e into ring slot (e - e0) mod depth
    auto issue = [&](int e, int e0, int src) {
        float2 *dst = buf + ((e - e0) % kM2LDepth) * 64;
        const float2 *ms = M + (size_t)src * nM;
        if (lane < nM) cp_async8(dst + lane, ms + lane);
        if (lane + 32 < nM) cp_async8(dst + lane + 32, ms + lane + 32);
    };
    for (int ci = blockIdx.x * kM2LSmallWarps + warp; ci < n_cells; ci += gridDim.x * kM2LSmallWarps) {
        const int cell = cells[ci];
        const float mlogw = -t.logw[cell];
        float2 acc[3] = {zero, zero, zero};
        const int e0 = t.v_ptr[cell], e1 = t.v_ptr[cell + 1];
        if (e0 + lane < e1) {
            my_src = t.v_idx[e0 + lane];
            my_code = t.v_code[e0 + lane];
        }
#pragma unroll
        for (int d = 0; d < kM2LDepth - 1; ++d) {
            if (e0 + d < e1) issue(e0 + d, e0, entry_src(e0 + d, e0));   // warp-uniform branch
            cp_async_commit();
        }
        for (int e = e0; e < e1; ++e) {
            // the slot refilled here was read in the previous iteration,
            // which ended with __syncwarp
            const int en = e + kM2LDepth - 1;
            if (en < e1) issue(en, e0, entry_src(en, e0));             // warp-uniform branch
            cp_async_commit();
            const int re = e - e0;
            const int cv = __shfl_sync(0xffffffffu, my_code, re & 31);
            const int code = re < 32 ? cv : t.v_code[e];
            cp_async_wait<kM2LDepth - 1>();        // entry e has landed (own copies)
            __syncwarp();                           // and every lane's copies are visible
            const float2 *cur = buf + ((e - e0) % kM2LDepth) * 64;
            const int b = code & 7, r = (code >> 3) & 3, cj = code >> 5;
            const float2 *Tl = Tf + ((size_t)(b + 7 * r + 28 * cj) * P1 + lr) * P1;
            for (int k = h; k < P1; k += halves) {
                const float2 tk = Tl[k];
#pragma unroll
                for (int c = 0; c < 3; ++c) cfma(acc[c], tk, cur[c * P1 + k]);
            }
            if (lane == 0)
#pragma unroll
                for (int c = 0; c < 3; ++c) acc[c].x += mlogw * cur[c * P1].x;   // Mt_0 is real
            __syncwarp();
        }
        if (halves == 2)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                acc[c].x += __shfl_xor_sync(0xffffffffu, acc[c].x, 16);
                acc[c].y += __shfl_xor_sync(0xffffffffu, acc[c].y, 16);
            }
        if (h == 0 && l < P1)   // onto zero, or the cell's list-4 P2L terms
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float2 &o = Lout[((size_t)cell * 3 + c) * P1 + l];
                o.x += acc[c].x;
                o.y += acc[c].y;
            }
    }
    cp_async_wait<0>();
}

// ------------------------------------------------ M2L in float-float --
// The FP64 passes spend most of their time in M2L, and FP64 arithmetic runs
// at 1/64 of the FP32 rate on this GPU.  This kernel computes the same sums
// (the symmetric form of m2l_kernel) in float-float arithmetic: every value
// is an unevaluated sum hi + lo of two floats, products are split exactly
// with an FMA (TwoProduct) and the leading parts are accumulated with
// Knuth's TwoSum, the error terms in a second float (the compensated dot
// product of Ogita, Rump and Oishi, "Accurate sum and dot product", SIAM J.
// Sci. Comput. 26, 2005).  The result carries about 48 significant bits,
// ample for the 1e-10 relative residual the FP64 passes serve.
// A float-float complex value is a float4 (hi.re, hi.im, lo.re, lo.im).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// acc (re, im as hi/lo pairs) += t * m, all float-float complex
__device__ __forceinline__ void ff_cfma(float4 &acc, const float4 t, const float4 m) {
    // real part: t.re m.re - t.im m.im
    float p1 = __fmul_rn(t.x, m.x), e1 = fmaf(t.x, m.x, -p1);
    float p2 = __fmul_rn(-t.y, m.y), e2 = fmaf(-t.y, m.y, -p2);
    float s, q1, q2;
    two_sum(acc.x, p1, s, q1);
    two_sum(s, p2, acc.x, q2);
    float lo = fmaf(t.x, m.z, fmaf(t.z, m.x, fmaf(-t.y, m.w, -t.w * m.y)));
    acc.z += ((q1 + q2) + (e1 + e2)) + lo;
    // imaginary part: t.re m.im + t.im m.re
    p1 = __fmul_rn(t.x, m.y);
    e1 = fmaf(t.x, m.y, -p1);
    p2 = __fmul_rn(t.y, m.x);
    e2 = fmaf(t.y, m.x, -p2);
    two_sum(acc.y, p1, s, q1);
    two_sum(s, p2, acc.y, q2);
    lo = fmaf(t.x, m.w, fmaf(t.z, m.y, fmaf(t.y, m.z, t.w * m.x)));
    acc.w += ((q1 + q2) + (e1 + e2)) + lo;
}

// acc += v (float-float complex)
__device__ __forceinline__ void ff_cadd(float4 &acc, const float4 v) {
    float s, q;
    two_sum(acc.x, v.x, s, q);
    acc.x = s;
    acc.z += q + v.z;
    two_sum(acc.y, v.y, s, q);
    acc.y = s;
    acc.w += q + v.w;
}

__device__ __forceinline__ float4 ff_from(double2 v) {
    const float hx = (float)v.x, hy = (float)v.y;
    return make_float4(hx, hy, (float)(v.x - (double)hx), (float)(v.y - (double)hy));
}

// v times i^(-n) (exact: a permutation with signs), optionally conjugated first
__device__ __forceinline__ float4 ff_rot(float4 v, int n) {
    switch (n & 3) {
        case 0: return v;
        case 1: return make_float4(v.y, -v.x, v.w, -v.z);      // times -i
        case 2: return make_float4(-v.x, -v.y, -v.z, -v.w);    // times -1
        default: return make_float4(-v.y, v.x, -v.w, v.z);     // times i
    }
}
__device__ __forceinline__ float4 ff_conj(float4 v) { return make_float4(v.x, -v.y, v.z, -v.w); }

// Per-level M2M (Eq. 71) and L2L (Eq. 73) of the FP64 passes in float-float
// (the tables of m2m_kernel / l2l_kernel stored as float-float): one warp per
// cell, lane k holds coefficient k; the FP64 inputs (children's moments, the
// parent's local expansion) are converted once per cell into shared memory,
// so the inner loops run on the FP32 pipes only.
// M2M lanes: coefficient k and P1 - 1 - k share a lane (k + 1 and P1 - k
// terms, P1 + 1 together), and the two half-warps take children 0, 1 and
// 2, 3, so 2 ceil(P1 / 2) lanes carry equal loads; the halves' sums are
// added at the end.  The four quadrant tables are staged in shared memory.
__device__ __forceinline__ float4 ff_shfl_xor(float4 v, int m) {
    return make_float4(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m),
                       __shfl_xor_sync(0xffffffffu, v.z, m), __shfl_xor_sync(0xffffffffu, v.w, m));
}

__device__ __forceinline__ double2 ff_to_double(float4 a) {
    return make_double2((double)a.x + (double)a.z, (double)a.y + (double)a.w);
}

// shared memory of m2m_ff_kernel: the four quadrant tables and each warp's
// staged children
inline size_t mlff_smem(int P1) { return (4 * (size_t)P1 * P1 + 4 * 4 * 3 * (size_t)P1) * sizeof(float4); }

static __global__ void __launch_bounds__(128) m2m_ff_kernel(const int *__restrict__ child0,
                                                            const int *__restrict__ cells, int n, int P1,
                                                            const float4 *__restrict__ tab,
                                                            double2 *__restrict__ M) {
    extern __shared__ unsigned char smem_raw[];
    float4 *tabs = reinterpret_cast<float4 *>(smem_raw);   // [4][P1][P1]
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nM = 3 * P1;
    float4 *smw = tabs + 4 * P1 * P1 + w * 4 * nM;          // this warp's 4 children
    stage_async(tabs, tab, 4 * P1 * P1, threadIdx.x, blockDim.x);
    cp_async_commit();
    const int idx = blockIdx.x * 4 + w;
    const bool live = idx < n;
    const int cell = live ? cells[idx] : 0;
    if (live) {
        const double2 *src = M + (size_t)child0[cell] * nM;   // the 4 children are contiguous
        // four loads in flight per lane, then the conversions
        for (int i0 = lane; i0 < 4 * nM; i0 += 4 * 32) {
            double2 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = i0 + 32 * u;
                v[u] = i < 4 * nM ? src[i] : make_double2(0.0, 0.0);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = i0 + 32 * u;
                if (i < 4 * nM) smw[i] = ff_from(v[u]);
            }
        }
    }
    cp_async_wait<0>();
    __syncthreads();
    if (!live) return;
    tab = tabs;
    const int kk = lane & 15, h = lane >> 4;
    const int k1 = kk, k2 = P1 - 1 - kk;
    const bool on = k1 <= k2, two = k1 < k2;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 a1[3] = {z, z, z}, a2[3] = {z, z, z};
    if (on)
        for (int q = 2 * h; q < 2 * h + 2; ++q) {
            const float4 *mq = smw + q * nM;
            const float4 *T1 = tab + ((size_t)q * P1 + k1) * P1;
            for (int j = 0; j <= k1; ++j) {
                const float4 tq = T1[j];
                for (int c = 0; c < 3; ++c) ff_cfma(a1[c], tq, mq[c * P1 + j]);
            }
            if (two) {
                const float4 *T2 = tab + ((size_t)q * P1 + k2) * P1;
                for (int j = 0; j <= k2; ++j) {
                    const float4 tq = T2[j];
                    for (int c = 0; c < 3; ++c) ff_cfma(a2[c], tq, mq[c * P1 + j]);
                }
            }
        }
    for (int c = 0; c < 3; ++c) {
        ff_cadd(a1[c], ff_shfl_xor(a1[c], 16));
        ff_cadd(a2[c], ff_shfl_xor(a2[c], 16));
    }
    if (h != 0 || !on) return;
    for (int c = 0; c < 3; ++c) {
        M[((size_t)cell * 3 + c) * P1 + k1] = ff_to_double(a1[c]);
        if (two) M[((size_t)cell * 3 + c) * P1 + k2] = ff_to_double(a2[c]);
    }
}

static __global__ void __launch_bounds__(128) l2l_ff_kernel(TreeView<double> t, const int *__restrict__ cells, int n,
                                                            int level, int P1, const float4 *__restrict__ tab,
                                                            const double2 *__restrict__ Lm2l,
                                                            double2 *__restrict__ L) {
    __shared__ float4 sp[4][3 * 32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int idx = blockIdx.x * 4 + w;
    if (idx >= n) return;
    const int cell = cells[idx];
    const int nM = 3 * P1;
    const bool up = level >= 3;
    if (up) {
        const double2 *src = L + (size_t)t.parent[cell] * nM;
        for (int i = l; i < nM; i += 32) sp[w][i] = ff_from(src[i]);
    }
    __syncwarp();
    if (l >= P1) return;
    float4 acc[3];
    for (int c = 0; c < 3; ++c) acc[c] = ff_from(Lm2l[((size_t)cell * 3 + c) * P1 + l]);
    if (up) {
        const float4 *Tq = tab + ((size_t)t.quad[cell] * P1 + l) * P1;
        int k = l;
        for (; k + 4 <= P1; k += 4) {   // four table loads in flight
            float4 tq[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) tq[u] = Tq[k + u];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                for (int c = 0; c < 3; ++c) ff_cfma(acc[c], tq[u], sp[w][c * P1 + k + u]);
        }
        for (; k < P1; ++k) {
            const float4 tq = Tq[k];
            for (int c = 0; c < 3; ++c) ff_cfma(acc[c], tq, sp[w][c * P1 + k]);
        }
    }
    for (int c = 0; c < 3; ++c)
        L[((size_t)cell * 3 + c) * P1 + l] =
            make_double2((double)acc[c].x + (double)acc[c].z, (double)acc[c].y + (double)acc[c].w);
}

// ------------------------------------- stored rows in float-float --
// P2M and list-4 P2L of the FP64 passes from stored per-piece coefficient
// rows kept as float-float complex values (float4: re hi, im hi, re lo,
// im lo) and densities converted to float-float once per piece: the sums run
// on the FP32 pipes (FP64 arithmetic is 1/64 of the FP32 rate here) with
// about 2^-44 relative error per term, and the results are written as FP64.

// hi + lo += (ah + al) (bh + bl)
__device__ __forceinline__ void ff_fma(float &hi, float &lo, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    const float e = fmaf(ah, bh, -p);
    float sum, q;
    two_sum(hi, p, sum, q);
    hi = sum;
    lo += q + e + fmaf(ah, bl, al * bh);
}

__device__ __forceinline__ float2 ff_of(double v) {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
}

// acc (complex float-float) += row (complex float-float) * d (real float-float)
__device__ __forceinline__ void ff_row_fma(float4 &acc, float4 row, float2 d) {
    ff_fma(acc.x, acc.z, row.x, row.z, d.x, d.y);
    ff_fma(acc.y, acc.w, row.y, row.w, d.x, d.y);
}

// M[leaf] = sum over the leaf's pieces of rows_g sigma_bar + rows_f mu_bar
// (rows_f only when use_m); block per leaf as p2m_kernel.
static __global__ void __launch_bounds__(kChunk) p2m_rows_ff_kernel(TreeView<double> t, const int *__restrict__ leaves,
                                                                    const double *__restrict__ sb,
                                                                    const double *__restrict__ mb, int use_s,
                                                                    int use_m, int P1, double2 *__restrict__ M,
                                                                    const float4 *__restrict__ rows_g,
                                                                    const float4 *__restrict__ rows_f) {
    __shared__ float2 D[kChunk * 6];
    __shared__ float4 part[3 * kChunk];
    const int cell = leaves[blockIdx.x];
    const int tid = threadIdx.x;
    const int ngrp = kChunk / P1, grp = tid / P1, k = tid - grp * P1;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 acc[3] = {z, z, z};
    const int p0 = t.pstart[cell], pn = t.pcount[cell];
    for (int base = 0; base < pn; base += kChunk) {
        const int cnt = min(kChunk, pn - base);
        __syncthreads();
        if (tid < cnt) {
            const size_t seg = (size_t)t.pseg[p0 + base + tid];
            for (int c = 0; c < 3; ++c) {
                D[tid * 6 + c] = ff_of(use_s ? sb[3 * seg + c] : 0.0);
                D[tid * 6 + 3 + c] = ff_of(use_m ? mb[3 * seg + c] : 0.0);
            }
        }
        __syncthreads();
        if (grp < ngrp)
#pragma unroll 2
            for (int j = grp; j < cnt; j += ngrp) {
                const size_t ri = (size_t)(p0 + base + j) * P1 + k;
                const float4 cg = rows_g[ri];
                const float4 cf = use_m ? rows_f[ri] : z;
                for (int c = 0; c < 3; ++c) {
                    ff_row_fma(acc[c], cg, D[j * 6 + c]);
                    if (use_m) ff_row_fma(acc[c], cf, D[j * 6 + 3 + c]);
                }
            }
    }
    __syncthreads();
    if (grp < ngrp)
        for (int c = 0; c < 3; ++c) part[(grp * 3 + c) * P1 + k] = acc[c];
    __syncthreads();
    if (tid < P1)
        for (int c = 0; c < 3; ++c) {
            float4 a = part[c * P1 + tid];
            for (int q = 1; q < ngrp; ++q) ff_cadd(a, part[(q * 3 + c) * P1 + tid]);
            M[((size_t)cell * 3 + c) * P1 + tid] =
                make_double2((double)a.x + (double)a.z, (double)a.y + (double)a.w);
        }
}

// Lout[cell] += sum over the cell's list-4 rows (row_off, row_cnt, item as
// in p2l_flat_kernel) of rows_g sigma_bar + rows_f mu_bar.
static __global__ void __launch_bounds__(kChunk) p2l_rows_ff_kernel(TreeView<double> t, const int *__restrict__ cells,
                                                                    const long long *__restrict__ row_off,
                                                                    const int *__restrict__ row_cnt,
                                                                    const int2 *__restrict__ item,
                                                                    const double *__restrict__ sb,
                                                                    const double *__restrict__ mb, int use_s,
                                                                    int use_m, int P1, double2 *__restrict__ Lout,
                                                                    const float4 *__restrict__ rows_g,
                                                                    const float4 *__restrict__ rows_f) {
    __shared__ float2 D[kChunk * 6];
    __shared__ float4 part[3 * kChunk];
    const int cell = cells[blockIdx.x];
    const int tid = threadIdx.x;
    const int ngrp = kChunk / P1, grp = tid / P1, l = tid - grp * P1;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 acc[3] = {z, z, z};
    const long long r0 = row_off[cell];
    const int n = row_cnt[cell];
    for (int base = 0; base < n; base += kChunk) {
        const int cnt = min(kChunk, n - base);
        __syncthreads();
        if (tid < cnt) {
            const size_t seg = (size_t)t.pseg[item[r0 + base + tid].x];
            for (int c = 0; c < 3; ++c) {
                D[tid * 6 + c] = ff_of(use_s ? sb[3 * seg + c] : 0.0);
                D[tid * 6 + 3 + c] = ff_of(use_m ? mb[3 * seg + c] : 0.0);
            }
        }
        __syncthreads();
        if (grp < ngrp)
#pragma unroll 2
            for (int j = grp; j < cnt; j += ngrp) {
                const size_t ri = (size_t)(r0 + base + j) * P1 + l;
                const float4 cg = rows_g[ri];
                const float4 cf = use_m ? rows_f[ri] : z;
                for (int c = 0; c < 3; ++c) {
                    ff_row_fma(acc[c], cg, D[j * 6 + c]);
                    if (use_m) ff_row_fma(acc[c], cf, D[j * 6 + 3 + c]);
                }
            }
    }
    __syncthreads();
    if (grp < ngrp)
        for (int c = 0; c < 3; ++c) part[(grp * 3 + c) * P1 + l] = acc[c];
    __syncthreads();
    if (tid < P1)
        for (int c = 0; c < 3; ++c) {
            float4 a = part[c * P1 + tid];
            for (int q = 1; q < ngrp; ++q) ff_cadd(a, part[(q * 3 + c) * P1 + tid]);
            double2 *o = Lout + ((size_t)cell * 3 + c) * P1 + tid;
            o->x += (double)a.x + (double)a.z;
            o->y += (double)a.y + (double)a.w;
        }
}

// float-float copies of FP64 complex rows
static __global__ void rows_to_ff_kernel(const double2 *__restrict__ in, float4 *__restrict__ out, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double2 v = in[i];
        const float hx = (float)v.x, hy = (float)v.y;
        out[i] = make_float4(hx, hy, (float)(v.x - (double)hx), (float)(v.y - (double)hy));
    }
}

constexpr int kM2LffWarps = 8;
#ifndef DC_M2LFF_FULL
#define DC_M2LFF_FULL 12
#endif
constexpr int kM2LffFull = DC_M2LFF_FULL;   // source moments summed in float-float; the rest in FP32

inline size_t m2l_ff_smem(int P1) {
    return (7 * (size_t)P1 * P1 + kM2LffWarps * 2 * 3 * 32) * sizeof(float4);
}

// One warp per target cell, lane l holds coefficient l (P1 <= 32).  base:
// the 7 base matrices in float-float, transposed like m2l_kernel's
// ([b][k][l]).  The source moments of a pair are staged rotated and
// conjugated (m'_k = conj^cj(M_k i^(-r k))), double buffered.
static __global__ void __launch_bounds__(32 * kM2LffWarps) m2l_ff_kernel(TreeView<double> t, const int *__restrict__ cells,
                                                                         int n_cells, int P1,
                                                                         const float4 *__restrict__ base,
                                                                         const double2 *__restrict__ M,
                                                                         double2 *__restrict__ Lout) {
    extern __shared__ unsigned char smem_raw[];
    float4 *B = reinterpret_cast<float4 *>(smem_raw);                 // [7][P1][P1]
    float4 *stage = B + 7 * P1 * P1;                                  // [warps][2][3 * 32]
    stage_async(B, base, 7 * P1 * P1, threadIdx.x, blockDim.x);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nM = 3 * P1;
    const int lr = min(lane, P1 - 1);
    float4 *buf = stage + warp * 2 * 96;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int ci = blockIdx.x * kM2LffWarps + warp; ci < n_cells; ci += gridDim.x * kM2LffWarps) {
        const int cell = cells[ci];
        const double mlogw = -t.logw[cell];
        float4 acc[3] = {zero, zero, zero};
        double acc0[3] = {0.0, 0.0, 0.0};    // the -log(w) Mt_0 term of l = 0, in FP64
        const int e0 = t.v_ptr[cell], e1 = t.v_ptr[cell + 1];
        double2 pf[3];
        int code = 0;
        auto fetch = [&](int e) {
            const double2 *ms = M + (size_t)t.v_idx[e] * nM;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const int idx = lane + 32 * j;
                pf[j] = idx < nM ? ms[idx] : make_double2(0.0, 0.0);
            }
            code = t.v_code[e];
        };
        if (e0 < e1) fetch(e0);
        int slot = 0;
        for (int e = e0; e < e1; ++e) {
            const int b = code & 7, r = (code >> 3) & 3, cj = code >> 5;
            float4 *cur = buf + slot * 96;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const int idx = lane + 32 * j;
                if (idx < nM) {
                    float4 v = ff_rot(ff_from(pf[j]), r * (idx % P1));
                    cur[idx] = cj ? ff_conj(v) : v;
                }
            }
            const double2 *ms0 = M + (size_t)t.v_idx[e] * nM;
            if (lane == 0)
#pragma unroll
                for (int c = 0; c < 3; ++c) acc0[c] += mlogw * ms0[c * P1].x;    // Mt_0 is real
            __syncwarp();
            if (e + 1 < e1) fetch(e + 1);
            float4 part[3] = {zero, zero, zero};
            float2 tail[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
            const float4 *Tb = B + (size_t)b * P1 * P1;
            const int kff = min(P1, kM2LffFull);
            for (int k = 0; k < kff; ++k) {
                const float4 tk = Tb[k * P1 + lr];
#pragma unroll
                for (int c = 0; c < 3; ++c) ff_cfma(part[c], tk, cur[c * P1 + k]);
            }
            // moments k >= kM2LffFull in FP32: their terms carry at most a few
            // 1e-6 of the sum (the source moments of a well-separated cell
            // fall off like (sqrt(2) / 4)^k against the first), so FP32
            // rounding of them stays near 1e-14 of the result
            for (int k = kff; k < P1; ++k) {
                const float4 tk = Tb[k * P1 + lr];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float4 m = cur[c * P1 + k];
                    tail[c].x = fmaf(tk.x, m.x, fmaf(-tk.y, m.y, tail[c].x));
                    tail[c].y = fmaf(tk.x, m.y, fmaf(tk.y, m.x, tail[c].y));
                }
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                ff_cadd(part[c], make_float4(tail[c].x, tail[c].y, 0.f, 0.f));
                float4 v = cj ? ff_conj(part[c]) : part[c];
                ff_cadd(acc[c], ff_rot(v, r * lane));
            }
            slot ^= 1;
        }
        if (lane < P1)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                double2 o;
                o.x = ((double)acc[c].x + (double)acc[c].z) + (lane == 0 ? acc0[c] : 0.0);
                o.y = (double)acc[c].y + (double)acc[c].w;
                Lout[((size_t)cell * 3 + c) * P1 + lane] = o;
            }
    }
}

// ---------------------------------------------------------------- P2L --
// Incoming (local) coefficients of one segment piece for a list-4 cell
// (Eq. 62 for the single layer, Eq. 78/79 for the double layer): a, b the
// piece's end points relative to the cell centre (unscaled), len its chord
// length, om its arc weight, iw = 1/w and logw = log w of the cell.  Writes
// g[0..P1) and, when want_f, f[0..P1).
template <typename T>
__device__ __forceinline__ void p2l_piece_coefs(T ax, T ay, T bx, T by, T len, T om, T iw, T w, T logw, int P1,
                                                bool want_f, typename V2<T>::type *g, typename V2<T>::type *f) {
    using C = typename V2<T>::type;
    C a = mk<T>(ax * iw, ay * iw), b = mk<T>(bx * iw, by * iw);   // scaled
    C wv = mk<T>((bx - ax) / len, (by - ay) / len);
    // log(b/a) on the continuous branch (|arg| < pi: separated)
    C d = mk<T>(b.x - a.x, b.y - a.y), s = mk<T>(b.x + a.x, b.y + a.y);
    T aa = a.x * a.x + a.y * a.y;
    C lba = mk<T>(T(0.5) * tlog1p((d.x * s.x + d.y * s.y) / aa),
                  tatan2(a.x * b.y - a.y * b.x, a.x * b.x + a.y * b.y));
    // l = 0: omega [ l (1 - log a) - conj(w) b w_cell log(b/a) ] and i log(b/a)
    {
        C la = mk<T>(T(0.5) * tlog(aa) + logw, tatan2(a.y, a.x));
        C wb = cmul(mk<T>(wv.x, -wv.y), mk<T>(b.x * w, b.y * w));
        C t2 = cmul(wb, lba);
        g[0] = mk<T>(om * (len * (1 - la.x) - t2.x), om * (-len * la.y - t2.y));
        if (want_f) f[0] = mk<T>(-om * lba.y, om * lba.x);
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
    if (P1 > 1 && want_f) f[1] = fb;             // l = 1: T_0 / 1
    for (int q = 2; q < P1; ++q) {
        // here Tm = T_{q-2}
        g[q] = cscl(cmul(gb, Tm), T(1) / (T(q) * (q - 1)));
        bp = cmul(bp, be);
        Tm = cadd(cmul(al, Tm), bp);             // T_{q-1}
        if (want_f) f[q] = cscl(cmul(fb, Tm), T(1) / T(q));
    }
}

template <typename T, typename PS>
__global__ void __launch_bounds__(kChunk) p2l_kernel(TreeView<T> t, PS ps, const int *__restrict__ cells,
                                                     const T *__restrict__ sb, const T *__restrict__ mb,
                                                     int use_s, int use_m, int P1,
                                                     typename V2<T>::type *__restrict__ Lout,
                                                     const long long *__restrict__ row_off = nullptr,
                                                     const typename V2<T>::type *__restrict__ rows_g = nullptr,
                                                     const typename V2<T>::type *__restrict__ rows_f = nullptr,
                                                     typename V2<T>::type *__restrict__ out_g = nullptr,
                                                     typename V2<T>::type *__restrict__ out_f = nullptr) {
    // Stored coefficients: row row_off[cell] + r, r counting the pieces of the
    // cell's list 4 in order, P1 entries each.  rows_g / rows_f: use them (no
    // geometry); out_g / out_f: write them instead of accumulating.
    using C = typename V2<T>::type;
    extern __shared__ unsigned char smem_raw[];
    C *G = reinterpret_cast<C *>(smem_raw);          // [kChunk][P1] sigma coefficients
    C *F = G + kChunk * P1;                          // [kChunk][P1] mu coefficients
    int *sg = reinterpret_cast<int *>(F + kChunk * P1);
    const int cell = cells[blockIdx.x];
    const int tid = threadIdx.x;
    const int ngrp = kChunk / P1, grp = tid / P1, l = tid - grp * P1;   // as in p2m_kernel
    const bool want_f = use_m || out_g;
    const T iw = t.iw[cell], w = 1 / iw, logw = t.logw[cell];
    C acc[3];
    for (int c = 0; c < 3; ++c) acc[c] = mk<T>(0, 0);
    const long long r0 = row_off ? row_off[cell] : 0;
    int rr = 0;
    for (int e = t.x_ptr[cell]; e < t.x_ptr[cell + 1]; ++e) {
        const int src = t.x_idx[e];
        const int p0 = t.pstart[src], pn = t.pcount[src];
        for (int base = 0; base < pn; base += kChunk) {
            int cnt = min(kChunk, pn - base);
            __syncthreads();
            if (tid < cnt && rows_g) sg[tid] = t.pseg[p0 + base + tid];
            if (tid < cnt && !rows_g) {
                int i = p0 + base + tid;
                T ax, ay, bx, by;
                ps.rel(i, cell, e, t.x_off, ax, ay, bx, by);
                p2l_piece_coefs<T>(ax, ay, bx, by, t.plen[i], t.pw[i], iw, w, logw, P1, want_f, G + tid * P1,
                                   F + tid * P1);
                sg[tid] = t.pseg[i];
            }
            __syncthreads();
            if (grp < ngrp) {
                for (int j = grp; j < cnt; j += ngrp) {
                    const size_t ri = (size_t)(r0 + rr + j) * P1 + l;
                    C cg, cf;
                    if (rows_g) {
                        cg = rows_g[ri];
                        cf = rows_f ? rows_f[ri] : mk<T>(0, 0);
                    } else {
                        cg = G[j * P1 + l];
                        cf = use_m || out_g ? F[j * P1 + l] : mk<T>(0, 0);
                    }
                    if (out_g) {
                        out_g[ri] = cg;
                        out_f[ri] = cf;
                        continue;
                    }
                    int seg = sg[j];
                    for (int c = 0; c < 3; ++c) {
                        T s = use_s ? sb[3 * (size_t)seg + c] : T(0);
                        T mu = use_m ? mb[3 * (size_t)seg + c] : T(0);
                        acc[c].x += s * cg.x + mu * cf.x;
                        acc[c].y += s * cg.y + mu * cf.y;
                    }
                }
            }
            rr += cnt;
        }
    }
    if (out_g) return;
    // the groups' partial sums, added in group order
    __syncthreads();
    if (grp < ngrp)
        for (int c = 0; c < 3; ++c) G[(grp * 3 + c) * P1 + l] = acc[c];
    __syncthreads();
    if (tid < P1)
        for (int c = 0; c < 3; ++c) {
            C a = G[c * P1 + tid];
            for (int q = 1; q < ngrp; ++q) a = cadd(a, G[(q * 3 + c) * P1 + tid]);
            C *o = Lout + ((size_t)cell * 3 + c) * P1 + tid;
            o->x += a.x;
            o->y += a.y;
        }
}

// ---------------------------------------------------------------- L2L --
// One level: L = L_m2l + L2L(parent) (Eq. 73) for the listed cells (the
// parent term from level 3 on), one warp per cell, lane l holds coefficient l.
template <typename T>
__global__ void __launch_bounds__(32 * kLevelWarps) l2l_kernel(TreeView<T> t, const int *__restrict__ cells, int n,
                                                               int level, int P1,
                                                               const typename V2<T>::type *__restrict__ tab,
                                                               const typename V2<T>::type *__restrict__ Lm2l,
                                                               typename V2<T>::type *__restrict__ L) {
    using C = typename V2<T>::type;
    const int idx = blockIdx.x * kLevelWarps + (threadIdx.x >> 5);
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

// Incoming expansion of each listed leaf by the recursion of Eq. 73 along its
// ancestors: L = Lm2l(a_2) at the level-2 ancestor, then L = Lm2l(a) +
// L2L(L) for each ancestor a below it and the leaf itself (the level-invariant
// table of the child's quadrant).  Inner cells get no expansion: only leaves
// hold targets.  One block per leaf (blockDim >= P1, a multiple of 32); the
// chain's Lm2l is staged in shared memory up front.  For P1 <= 16 lane l + 16 h sums the terms k = l + h, l + h + 2, ...
// of coefficient l and the halves are added by a shuffle; above 16 thread l
// sums all k >= l.
constexpr int kWalkMax = 48;    // ancestors kept (tree depth <= 40)

template <typename T>
__global__ void walk_kernel(TreeView<T> t, const int *__restrict__ leaves, const int *__restrict__ chains,
                            int P1, int n_max, const typename V2<T>::type *__restrict__ tab,
                            const typename V2<T>::type *__restrict__ Lm2l,
                            typename V2<T>::type *__restrict__ L) {
    using C = typename V2<T>::type;
    extern __shared__ unsigned char smem_raw[];
    C *cur = reinterpret_cast<C *>(smem_raw);   // [3][P1]
    C *pre = cur + 3 * P1;                       // [n][3][P1]: the chain's Lm2l
    __shared__ int chain[kWalkMax], quad[kWalkMax];
    __shared__ int n_chain;
    const int leaf = leaves[blockIdx.x];
    const int tid = threadIdx.x;
    // chains[blockIdx.x * (n_max + 1)]: length, then the leaf and its
    // ancestors down to level 2 (formed once per drawing)
    const int *ch = chains + (size_t)blockIdx.x * (n_max + 1);
    if (tid == 0) n_chain = ch[0];
    if (tid < n_max) {
        const int c = ch[1 + tid];
        chain[tid] = c;
        quad[tid] = c >= 0 ? t.quad[c] : 0;
    }
    __syncthreads();
    const int n = n_chain;
    const int nM = 3 * P1;
    for (int i = tid; i < n * nM; i += blockDim.x) {
        const int a = i / nM;
        if (sizeof(C) == 8 || sizeof(C) == 16) cp_async_any(pre + i, Lm2l + (size_t)chain[a] * nM + (i - a * nM));
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    const int halves = P1 <= 16 ? 2 : 1;
    const int l = halves == 2 ? (tid & 31 & 15) + (tid >> 5) * 32 : tid;
    const int h = halves == 2 ? ((tid & 31) >> 4) : 0;
    const bool on = l < P1;
    C acc[3];
    for (int c = 0; c < 3; ++c) acc[c] = mk<T>(0, 0);
    if (n > 0 && on && h == 0)
        for (int c = 0; c < 3; ++c) acc[c] = pre[((n - 1) * 3 + c) * P1 + l];
    for (int i = n - 2; i >= 0; --i) {
        __syncthreads();
        if (on && h == 0)
            for (int c = 0; c < 3; ++c) cur[c * P1 + l] = acc[c];
        __syncthreads();
        for (int c = 0; c < 3; ++c) acc[c] = (on && h == 0) ? pre[(i * 3 + c) * P1 + l] : mk<T>(0, 0);
        if (on) {
            const C *Tq = tab + ((size_t)quad[i] * P1 + l) * P1;
            for (int k = l + h; k < P1; k += halves) {
                const C tk = Tq[k];
                for (int c = 0; c < 3; ++c) cfma(acc[c], tk, cur[c * P1 + k]);
            }
        }
        if (halves == 2)
            for (int c = 0; c < 3; ++c) {
                acc[c].x += __shfl_xor_sync(0xffffffffu, acc[c].x, 16);
                acc[c].y += __shfl_xor_sync(0xffffffffu, acc[c].y, 16);
            }
    }
    if (on && h == 0)
        for (int c = 0; c < 3; ++c) L[((size_t)leaf * 3 + c) * P1 + l] = acc[c];
}

// n_max: the longest chain (levels 2 .. deepest), at most kWalkMax
template <typename T> inline size_t walk_smem(int P1, int n_max) {
    return 3 * (size_t)P1 * (1 + n_max) * sizeof(typename V2<T>::type);
}

template <typename T> inline size_t p2m_smem(int P1) {
    using C = typename V2<T>::type;
    return kChunk * (P1 + 1) * sizeof(C) + kChunk * sizeof(T) + kChunk * sizeof(C) + kChunk * sizeof(int);
}
// P2L over a flat list of each cell's list-4 pieces: item[r] = (piece,
// list-4 entry) for rows r = row_off[cell] .. row_off[cell] + row_cnt[cell],
// in the row order of the stored coefficients.  Chunks of kChunk pieces span
// the cell's source leaves, and each piece's densities are staged in shared
// memory next to its coefficients (recomputed, or read from rows_g / rows_f),
// so the accumulation reads no global memory.
template <typename T, typename PS>
__global__ void __launch_bounds__(kChunk) p2l_flat_kernel(TreeView<T> t, PS ps, const int *__restrict__ cells,
                                                          const long long *__restrict__ row_off,
                                                          const int *__restrict__ row_cnt,
                                                          const int2 *__restrict__ item,
                                                          const T *__restrict__ sb, const T *__restrict__ mb,
                                                          int use_s, int use_m, int P1,
                                                          typename V2<T>::type *__restrict__ Lout,
                                                          const typename V2<T>::type *__restrict__ rows_g = nullptr,
                                                          const typename V2<T>::type *__restrict__ rows_f = nullptr) {
    using C = typename V2<T>::type;
    extern __shared__ unsigned char smem_raw[];
    C *G = reinterpret_cast<C *>(smem_raw);          // [kChunk][P1] sigma coefficients
    C *F = G + kChunk * P1;                          // [kChunk][P1] mu coefficients
    T *D = reinterpret_cast<T *>(F + kChunk * P1);   // [kChunk][6] sigma, mu of the piece's segment
    const int cell = cells[blockIdx.x];
    const int tid = threadIdx.x;
    const int ngrp = kChunk / P1, grp = tid / P1, l = tid - grp * P1;
    const bool want_f = use_m != 0;
    const T iw = t.iw[cell], w = 1 / iw, logw = t.logw[cell];
    C acc[3];
    for (int c = 0; c < 3; ++c) acc[c] = mk<T>(0, 0);
    const long long r0 = row_off[cell];
    const int n = row_cnt[cell];
    for (int base = 0; base < n; base += kChunk) {
        const int cnt = min(kChunk, n - base);
        __syncthreads();
        if (tid < cnt) {
            const int2 it = item[r0 + base + tid];
            const int i = it.x;
            const size_t seg = (size_t)t.pseg[i];
            T *dd = D + 6 * tid;
            for (int c = 0; c < 3; ++c) {
                dd[c] = use_s ? sb[3 * seg + c] : T(0);
                dd[3 + c] = use_m ? mb[3 * seg + c] : T(0);
            }
            if (!rows_g) {
                T ax, ay, bx, by;
                ps.rel(i, cell, it.y, t.x_off, ax, ay, bx, by);
                p2l_piece_coefs<T>(ax, ay, bx, by, t.plen[i], t.pw[i], iw, w, logw, P1, want_f, G + tid * P1,
                                   F + tid * P1);
            }
        }
        __syncthreads();
        if (grp < ngrp) {
            for (int j = grp; j < cnt; j += ngrp) {
                C cg, cf = mk<T>(0, 0);
                if (rows_g) {
                    const size_t ri = (size_t)(r0 + base + j) * P1 + l;
                    cg = rows_g[ri];
                    if (use_m && rows_f) cf = rows_f[ri];
                } else {
                    cg = G[j * P1 + l];
                    if (use_m) cf = F[j * P1 + l];
                }
                const T *dd = D + 6 * j;
                for (int c = 0; c < 3; ++c) {
                    acc[c].x += dd[c] * cg.x + dd[3 + c] * cf.x;
                    acc[c].y += dd[c] * cg.y + dd[3 + c] * cf.y;
                }
            }
        }
    }
    // the groups' partial sums, added in group order
    __syncthreads();
    if (grp < ngrp)
        for (int c = 0; c < 3; ++c) G[(grp * 3 + c) * P1 + l] = acc[c];
    __syncthreads();
    if (tid < P1)
        for (int c = 0; c < 3; ++c) {
            C a = G[c * P1 + tid];
            for (int q = 1; q < ngrp; ++q) a = cadd(a, G[(q * 3 + c) * P1 + tid]);
            C *o = Lout + ((size_t)cell * 3 + c) * P1 + tid;
            o->x += a.x;
            o->y += a.y;
        }
}

template <typename T> inline size_t p2l_flat_smem(int P1) {
    using C = typename V2<T>::type;
    return 2 * kChunk * P1 * sizeof(C) + 6 * kChunk * sizeof(T);
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
