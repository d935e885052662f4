// Two-level preconditioner for the single-layer system G_H sigma = b (Eq. 27):
// the panel block-Jacobi smoother B (inverse self-interaction blocks) and a
// coarse space of panel-wise constants, applied multiplicatively:
//
//   y = Ac^-1 R v            (R: sum over a panel's nodes, Ac ~ R G_H P)
//   M v = P y + B (v - A~ P y)
//
// where P spreads y_j to the nodes of panel j and A~ P approximates G_H P:
// exact for near panel pairs (closed forms, App. D) and the panel's
// monopole, l_j G(q_a, c_j), for the others.  M is a fixed linear map, so
// GMRES on G_H M still converges to the solution of Eq. 27; only the
// iteration count changes.  Not in the paper (plain GMRES there).
//
// The coarse matrix Ac = R A~ P (panels x panels, FP32) is inverted once per
// drawing by blocked Gauss-Jordan elimination without pivoting (it is
// strongly diagonal: a panel's self term dominates its row), one launch per
// 32-wide pivot block.
//
// Drawings with more panels than the dense coarse inverse can hold group
// the panels into aggregates of K panels consecutive in the Morton order of
// their centroids, K = ceil(P / (limit - 32)); the coarse space is then one
// constant per aggregate and Ac = R_agg A~ P_agg comes from the same
// panel-level monopoles and near-pair corrections.  The coarse residual
// takes the FMM itself, M v = P y + B (v - G_H P y): a monopole sum would
// cost (nodes x panels) logarithms per application at these sizes, while
// G_H P y is one more operator application (the caller supplies it between
// apply_stage1 and apply_stage2).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "dc_internal.h"
#include "ffarith.cuh"
#include "segint.cuh"

namespace dc {

namespace {

constexpr int kGJ = 32;                 // block size of the Gauss-Jordan inversion
constexpr int kMaxCoarse = 12288;       // default largest coarse system inverted (padded)
// -log|q - c| / 2pi = kMonoLog2 * log2(|q - c|^2)
constexpr float kMonoLog2 = -0.0551589000381629f;   // -ln 2 / 4pi

// log2 |q - c|^2 in FP32 from FP32 positions; the 1e-30 keeps a node that
// sits on a centroid finite and changes no other value.
__device__ __forceinline__ float mono_lg2(float2 q, float2 c) {
    const float dx = q.x - c.x, dy = q.y - c.y;
    return __log2f(fmaf(dx, dx, fmaf(dy, dy, 1e-30f)));
}

// Monopole kernel of panel j at a node: -log|q - c| / 2pi (the near pairs
// subtract exactly this value).
__device__ __forceinline__ float mono32(float2 q, float2 c) { return kMonoLog2 * mono_lg2(q, c); }

// corr[e][m] = (G_H 1_j)(q_{i,m}) - l_j mono32(q_{i,m}, c_j) for the near pair
// e = (i, j): the single layer of panel j with unit density (Lambda
// reproduces constants) at the nodes of panel i, minus its monopole.  One
// warp per pair; with g <= 16 each node takes two lanes, which split the
// segments between them.  A segment within kNearSeg chord lengths of the
// node (and the node's own segment, singular) needs the FP64 closed form;
// the others, whose terms are smooth, take the FP32 one on coordinates
// taken relative to the node in FP64 (the same closed form, App. D).  The
// FP64 logarithms and arctangents are this GPU's slowest path, and a warp
// pays for an FP64 instruction whatever lanes it runs for: the first sweep
// does the FP32 terms and lists the near (node, segment) entries in shared
// memory (in sweep order), the warp then computes the listed entries with
// all lanes busy, and each node adds its entries in list order (entries
// beyond the list's room are computed in place).
constexpr double kNearSeg = 8.0;
constexpr int kNearCap = 512;
__global__ void __launch_bounds__(32) near_pairs_kernel(const int2 *__restrict__ pairs, const double *__restrict__ seg,
                                                        const double *__restrict__ segw,
                                                        const double *__restrict__ nxy, const int *__restrict__ nseg,
                                                        const int *__restrict__ nseg2,
                                                        const float2 *__restrict__ q32,
                                                        const float2 *__restrict__ c32,
                                                        const double *__restrict__ plen, int s, int g,
                                                        double *__restrict__ corr) {
    __shared__ int nl_tag[kNearCap];      // node m << 16 | segment kk
    __shared__ double nl_g[kNearCap];
    const int e = blockIdx.x, lane = threadIdx.x;
    const int halves = g <= 16 ? 2 : 1;
    const int m = halves == 2 ? (lane & 15) : lane, part = halves == 2 ? (lane >> 4) : 0;
    const bool valid = m < g;
    const int2 pr = pairs[e];
    const int a = pr.x * g + (valid ? m : 0), j = pr.y;
    const double qx = nxy[2 * a], qy = nxy[2 * a + 1];
    const int own1 = nseg[a], own2 = nseg2[a];
    double acc64 = 0.0;   // entries beyond the list's room
    float acc = 0.f;
    int listed = 0;       // entries listed so far (the same in every lane)
    const int sweeps = (s + halves - 1) / halves;
    for (int it = 0; it < sweeps; ++it) {
        const int kk = part + it * halves;
        const bool act = valid && kk < s;
        const int k = j * s + (act ? kk : 0);
        const double *q = seg + 4 * (size_t)k;
        const double ax = q[0] - qx, ay = q[1] - qy, bx = q[2] - qx, by = q[3] - qy;
        const double dx = q[2] - q[0], dy = q[3] - q[1];
        const bool own = k == own1 || k == own2;
        const bool near = act && (own || seg_is_near(ax, ay, bx, by, dx, dy, kNearSeg));
        const unsigned bal = __ballot_sync(0xffffffffu, near);
        if (near) {
            const int pos = listed + __popc(bal & ((1u << lane) - 1u));
            if (pos < kNearCap) {
                nl_tag[pos] = (m << 16) | kk;
            } else {
                double G, F;
                seg_gf_f64(qx, qy, q[0], q[1], q[2], q[3], segw[k], own, G, F);
                acc64 += G;
            }
        } else if (act) {
            acc += (float)segw[k] * seg_g_far_f32(ax, ay, bx, by, dx, dy);
        }
        listed += __popc(bal);
    }
    __syncwarp();
    const int n_list = min(listed, kNearCap);
    for (int i = lane; i < n_list; i += 32) {
        const int mi = nl_tag[i] >> 16, k = j * s + (nl_tag[i] & 0xffff);
        const int ai = pr.x * g + mi;
        const double *q = seg + 4 * (size_t)k;
        double G, F;
        seg_gf_f64(nxy[2 * ai], nxy[2 * ai + 1], q[0], q[1], q[2], q[3], segw[k], k == nseg[ai] || k == nseg2[ai],
                   G, F);
        nl_g[i] = G;
    }
    __syncwarp();
    if (halves == 2) {
        acc64 += __shfl_down_sync(0xffffffffu, acc64, 16);
        acc += __shfl_down_sync(0xffffffffu, acc, 16);
    }
    if (valid && part == 0) {
        double near_sum = 0.0;
        for (int i = 0; i < n_list; ++i)
            if ((nl_tag[i] >> 16) == m) near_sum += nl_g[i];
        corr[(size_t)e * g + m] = near_sum + acc64 + (double)acc - plen[j] * (double)mono32(q32[a], c32[j]);
    }
}

// Ac[i][j] = sum_m (l_j mono32(q_{i,m}, c_j) + corr), padded with the identity
// to n_pad; one block per row.
__global__ void coarse_matrix_kernel(const float2 *__restrict__ q32, const float2 *__restrict__ c32,
                                     const float *__restrict__ plen32, const int *__restrict__ nptr,
                                     const int2 *__restrict__ pairs, const double *__restrict__ corr,
                                     int P, int g, int n_pad, float *__restrict__ Ac) {
    const int i = blockIdx.x;
    float *row = Ac + (size_t)i * n_pad;
    if (i >= P) {
        for (int j = threadIdx.x; j < n_pad; j += blockDim.x) row[j] = (i == j) ? 1.f : 0.f;
        return;
    }
    for (int j = threadIdx.x; j < n_pad; j += blockDim.x) {
        float v = 0.f;
        if (j < P) {
            const float2 c = c32[j];
            for (int m = 0; m < g; ++m) v += mono32(q32[i * g + m], c);
            v *= plen32[j];
        }
        row[j] = v;
    }
    __syncthreads();
    for (int e = nptr[i]; e < nptr[i + 1]; ++e) {
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int m = 0; m < g; ++m) s += corr[(size_t)e * g + m];
            row[pairs[e].y] += (float)s;
        }
        __syncthreads();
    }
}

// Aggregated form: Ac[I][J] = sum over the nodes q of aggregate I and the
// panels j of aggregate J of l_j mono32(q, c_j) (one block per row I; the
// panels of aggregate a are pagg[a] .. pagg[a + 1] - 1), padded with the
// identity to n_pad.  The near-pair corrections are added by
// coarse_agg_corr_kernel.
__global__ void coarse_agg_matrix_kernel(const float2 *__restrict__ q32, const float2 *__restrict__ c32,
                                         const float *__restrict__ plen32, const int *__restrict__ pagg,
                                         const int *__restrict__ perm, int nA, int g, int n_pad,
                                         float *__restrict__ Ac) {
    const int I = blockIdx.x;
    float *row = Ac + (size_t)I * n_pad;
    if (I >= nA) {
        for (int j = threadIdx.x; j < n_pad; j += blockDim.x) row[j] = (I == j) ? 1.f : 0.f;
        return;
    }
    for (int J = threadIdx.x; J < n_pad; J += blockDim.x) {
        float v = 0.f;
        if (J < nA)
            for (int u = pagg[J]; u < pagg[J + 1]; ++u) {
                const int j = perm[u];
                const float2 c = c32[j];
                float t = 0.f;
                for (int w = pagg[I]; w < pagg[I + 1]; ++w) {
                    const int i = perm[w];
                    for (int m = 0; m < g; ++m) t += mono32(q32[i * g + m], c);
                }
                v += plen32[j] * t;
            }
        row[J] = v;
    }
}

// Ac[agg(i)][agg(j)] += sum_m corr[e][m] over the near panel pairs e = (i, j)
// of the panels i of aggregate I (one thread per row, pairs in order).
__global__ void coarse_agg_corr_kernel(const int *__restrict__ pagg, const int *__restrict__ perm,
                                       const int *__restrict__ agg_of, int nA, const int *__restrict__ nptr,
                                       const int2 *__restrict__ pairs, const double *__restrict__ corr, int g,
                                       int n_pad, float *__restrict__ Ac) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nA) return;
    float *row = Ac + (size_t)I * n_pad;
    for (int w = pagg[I]; w < pagg[I + 1]; ++w) {
        const int i = perm[w];
        for (int e = nptr[i]; e < nptr[i + 1]; ++e) {
            double t = 0.0;
            for (int m = 0; m < g; ++m) t += corr[(size_t)e * g + m];
            row[agg_of[pairs[e].y]] += (float)t;
        }
    }
}

// s[I][c] = sum over aggregate I's nodes of v, as a float-float pair
__global__ void restrict_agg_kernel(const double *__restrict__ v, const int *__restrict__ pagg,
                                    const int *__restrict__ perm, int nA, int g, float2 *__restrict__ s) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * nA) return;
    const int I = t / 3, c = t % 3;
    double a = 0.0;
    for (int w = pagg[I]; w < pagg[I + 1]; ++w)
        for (int n = perm[w] * g; n < (perm[w] + 1) * g; ++n) a += v[3 * (size_t)n + c];
    const float hi = (float)a;
    s[t] = make_float2(hi, (float)(a - (double)hi));
}

// py[node][c] = y[agg(panel(node))][c]: the coarse correction spread to the nodes
__global__ void spread_agg_kernel(const double *__restrict__ y, const int *__restrict__ agg_of, int N, int g,
                                  double *__restrict__ py) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * N) return;
    const int c = t % 3, n = t / 3;
    py[t] = y[3 * agg_of[n / g] + c];
}

// One step k of the blocked Gauss-Jordan inversion (no pivoting), the whole
// matrix read from A and written to B (every entry of the step's result reads
// entries that other blocks rewrite, hence two buffers).  With D = A_kk the
// pivot block and the rows / columns of block k called pivot rows / columns:
//   B_kk = D^-1,  B_kj = D^-1 A_kj,  B_ik = -A_ik D^-1,  B_ij = A_ij - A_ik D^-1 A_kj.
// A block of 256 threads writes a 64 x 64 tile.  Warp 0 inverts D in
// registers (lane t holds column t; one pivot per step, the pivot column
// passed by shuffles) while the others stage the tile's pivot-column rows
// A_ik and pivot-row columns A_kj in shared memory.  Then Y = D^-1 A_kj
// (D^-1 itself for pivot columns), and every entry is Y for pivot rows,
// else (A_ij or 0 for pivot columns) - A_ik Y.
constexpr int kGjTile = 64;
__global__ void __launch_bounds__(256) gj_step_kernel(const float *__restrict__ A, float *__restrict__ B, int n,
                                                      int k) {
    static_assert(kGJ == 32, "one warp inverts the pivot block");
    __shared__ float Di[kGJ][kGJ + 1];
    __shared__ float Aik[kGjTile][kGJ + 1];
    __shared__ float Akj[kGJ][kGjTile + 1];
    __shared__ float Y[kGJ][kGjTile + 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int i0 = blockIdx.y * kGjTile, j0 = blockIdx.x * kGjTile, kc = k * kGJ;
    if (warp == 0) {
        float a[kGJ];   // a[r] = D[r][lane]
#pragma unroll
        for (int r = 0; r < kGJ; ++r) a[r] = A[(size_t)(kc + r) * n + kc + lane];
#pragma unroll
        for (int c = 0; c < kGJ; ++c) {
            const float rp = 1.f / __shfl_sync(0xffffffffu, a[c], c);
            const float rowc = (lane == c) ? rp : a[c] * rp;
#pragma unroll
            for (int r = 0; r < kGJ; ++r) {
                if (r == c) continue;
                const float f = __shfl_sync(0xffffffffu, a[r], c);   // D[r][c] before this pivot
                a[r] = (lane == c) ? -f * rp : fmaf(-f, rowc, a[r]);
            }
            a[c] = rowc;
        }
#pragma unroll
        for (int r = 0; r < kGJ; ++r) Di[r][lane] = a[r];
    } else {
        for (int u = tid - 32; u < kGjTile * kGJ; u += 224) {
            const int r = u / kGJ, c = u % kGJ;
            Aik[r][c] = (i0 + r < n) ? A[(size_t)(i0 + r) * n + kc + c] : 0.f;
            const int r2 = u / kGjTile, c2 = u % kGjTile;
            Akj[r2][c2] = (j0 + c2 < n) ? A[(size_t)(kc + r2) * n + j0 + c2] : 0.f;
        }
    }
    __syncthreads();
    for (int u = tid; u < kGJ * kGjTile; u += 256) {
        const int t = u / kGjTile, jj = u % kGjTile, j = j0 + jj;
        float v;
        if (j >= kc && j < kc + kGJ) {
            v = Di[t][j - kc];
        } else {
            v = 0.f;
#pragma unroll 8
            for (int q = 0; q < kGJ; ++q) v = fmaf(Di[t][q], Akj[q][jj], v);
        }
        Y[t][jj] = v;
    }
    __syncthreads();
    // thread (ty, tx): rows ty + 16 a, columns tx + 16 b
    const int tx = tid & 15, ty = tid >> 4;
#pragma unroll
    for (int aa = 0; aa < 4; ++aa) {
        const int ii = ty + 16 * aa, i = i0 + ii;
        if (i >= n) continue;
        const bool prow = (i >= kc && i < kc + kGJ);
        float acc[4];
#pragma unroll
        for (int bb = 0; bb < 4; ++bb) acc[bb] = 0.f;
        if (!prow) {
#pragma unroll 8
            for (int q = 0; q < kGJ; ++q) {
                const float w = Aik[ii][q];
#pragma unroll
                for (int bb = 0; bb < 4; ++bb) acc[bb] = fmaf(w, Y[q][tx + 16 * bb], acc[bb]);
            }
        }
#pragma unroll
        for (int bb = 0; bb < 4; ++bb) {
            const int jj = tx + 16 * bb, j = j0 + jj;
            if (j >= n) continue;
            const bool pcol = (j >= kc && j < kc + kGJ);
            float v;
            if (prow) v = Y[i - kc][jj];
            else v = (pcol ? 0.f : A[(size_t)i * n + j]) - acc[bb];
            B[(size_t)i * n + j] = v;
        }
    }
}

// ------------------------------------------------------------------ apply --
// s[j][c] = sum over panel j's nodes of v, as a float-float pair (hi, lo)
__global__ void restrict_kernel(const double *__restrict__ v, int P, int g, float2 *__restrict__ s) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * P) return;
    const int j = t / 3, c = t % 3;
    double a = 0.0;
    for (int m = 0; m < g; ++m) a += v[3 * ((size_t)j * g + m) + c];
    const float hi = (float)a;
    s[t] = make_float2(hi, (float)(a - (double)hi));
}

// acc (hi, lo) += w * (x.hi + x.lo): the product's leading part split exactly
// (FMA TwoProduct), summed by TwoSum; the small terms go to lo (the
// compensated dot product of Ogita, Rump and Oishi)
__device__ __forceinline__ void dot2_step(float &hi, float &lo, float w, float2 x) {
    const float p = __fmul_rn(w, x.x);
    const float pe = fmaf(w, x.x, -p);
    const float sum = __fadd_rn(hi, p);
    const float bb = __fsub_rn(sum, hi);
    const float se = __fadd_rn(__fsub_rn(hi, __fsub_rn(sum, bb)), __fsub_rn(p, bb));
    hi = sum;
    lo += se + pe + w * x.y;
}

// y = Ac^-1 s (fixed-order reduction); pan[j] = (c_j, k l_j y_j for
// channels 0, 1), pan2[j] = k l_j y_j for channel 2, k = kMonoLog2 (FP32).
// One warp per row, kSolveRows rows per block: the vector s is staged in
// shared memory kSolveCols columns at a time and serves all of the block's
// rows.  Compensated (float-float) sums: M amplifies by ~1e4-1e5, and its
// rounding must stay well below the FP32 operator's own error.
constexpr int kSolveRows = 8, kSolveCols = 2048, kSolveLoads = 8;
__global__ void __launch_bounds__(32 * kSolveRows) coarse_solve_kernel(const float *__restrict__ Ainv, int n_pad, int P,
                                                                       const float2 *__restrict__ s,
                                                                       const float *__restrict__ plen32,
                                                                       const float2 *__restrict__ c32,
                                                                       double *__restrict__ y,
                                                                       float4 *__restrict__ pan,
                                                                       float *__restrict__ pan2) {
    __shared__ float2 ss[3 * kSolveCols];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = blockIdx.x * kSolveRows + w;
    const float *row = Ainv + (size_t)min(i, P - 1) * n_pad;
    float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f, h2 = 0.f, l2 = 0.f;
    for (int c0 = 0; c0 < P; c0 += kSolveCols) {
        const int cn = min(kSolveCols, P - c0);
        __syncthreads();
        for (int u = threadIdx.x; u < 3 * cn; u += 32 * kSolveRows) ss[u] = s[3 * (size_t)c0 + u];
        __syncthreads();
        for (int jj = lane; jj < cn; jj += kSolveLoads * 32) {
            // kSolveLoads columns' loads in flight per lane (the warp waits on
            // load latency: one warp per row leaves most warp slots empty)
            float wv[kSolveLoads];
#pragma unroll
            for (int u = 0; u < kSolveLoads; ++u) {
                const int j = jj + 32 * u;
                wv[u] = j < cn ? row[c0 + j] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < kSolveLoads; ++u) {
                const int j = jj + 32 * u;
                if (j >= cn) break;
                dot2_step(h0, l0, wv[u], ss[3 * j]);
                dot2_step(h1, l1, wv[u], ss[3 * j + 1]);
                dot2_step(h2, l2, wv[u], ss[3 * j + 2]);
            }
        }
    }
    double a0 = (double)h0 + (double)l0, a1 = (double)h1 + (double)l1, a2 = (double)h2 + (double)l2;
    for (int off = 16; off > 0; off >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, off);
        a1 += __shfl_xor_sync(0xffffffffu, a1, off);
        a2 += __shfl_xor_sync(0xffffffffu, a2, off);
    }
    if (lane == 0 && i < P) {
        y[3 * i + 0] = a0;
        y[3 * i + 1] = a1;
        y[3 * i + 2] = a2;
        const float k = kMonoLog2 * plen32[i];
        const float2 c = c32[i];
        pan[i] = make_float4(c.x, c.y, k * (float)a0, k * (float)a1);
        pan2[i] = k * (float)a2;
    }
}

// The monopoles of all panels at every node, t_q[a] = sum over the panels
// of part q of l_j y_j mono32(q_a, c_j): kSplit parts in parallel (tiles of
// panels staged in shared memory), added in order by residual_kernel.  Each
// thread takes kMonoNodes nodes, so one pair of shared-memory loads serves
// kMonoNodes logarithms.
#ifndef DC_MONO_SPLIT
#define DC_MONO_SPLIT 8
#endif
#ifndef DC_MONO_NODES
#define DC_MONO_NODES 2
#endif
constexpr int kTile = 256;
constexpr int kSplit = DC_MONO_SPLIT;
constexpr int kMonoNodes = DC_MONO_NODES;
constexpr int kMonoThreads = 128;
__global__ void __launch_bounds__(kMonoThreads) monopole_kernel(const float2 *__restrict__ q32,
                                                                const float4 *__restrict__ pan,
                                                                const float *__restrict__ pan2, int P, int N,
                                                                float *__restrict__ part) {
    __shared__ float4 sp[kTile];
    __shared__ float sp2[kTile];
    const int a0 = blockIdx.x * (kMonoThreads * kMonoNodes) + threadIdx.x;
    const int per = (P + kSplit - 1) / kSplit;
    const int lo = blockIdx.y * per, hi = min(P, lo + per);
    float2 q[kMonoNodes];
    float t[kMonoNodes][3];
#pragma unroll
    for (int n = 0; n < kMonoNodes; ++n) {
        const int a = a0 + n * kMonoThreads;
        q[n] = a < N ? q32[a] : make_float2(0.f, 0.f);
        t[n][0] = t[n][1] = t[n][2] = 0.f;
    }
    for (int base = lo; base < hi; base += kTile) {
        const int cnt = min(kTile, hi - base);
        __syncthreads();
        for (int u = threadIdx.x; u < cnt; u += kMonoThreads) {
            sp[u] = pan[base + u];
            sp2[u] = pan2[base + u];
        }
        __syncthreads();
        for (int u = 0; u < cnt; ++u) {
            const float4 p = sp[u];
            const float p2 = sp2[u];
            const float2 c = make_float2(p.x, p.y);
#pragma unroll
            for (int n = 0; n < kMonoNodes; ++n) {
                const float k = mono_lg2(q[n], c);
                t[n][0] += k * p.z;
                t[n][1] += k * p.w;
                t[n][2] += k * p2;
            }
        }
    }
#pragma unroll
    for (int n = 0; n < kMonoNodes; ++n) {
        const int a = a0 + n * kMonoThreads;
        if (a >= N) continue;
        float *o = part + ((size_t)blockIdx.y * N + a) * 3;
        o[0] = t[n][0];
        o[1] = t[n][1];
        o[2] = t[n][2];
    }
}

// Per panel i (one block): r = v - A~ P y at its nodes (the monopole parts,
// added in part order, plus the near-pair corrections), w = P y + B r with
// B_i the panel's inverse self-interaction block, written when w is given,
// and, when lam is given, sigma_bar = Lambda w for the panel's s segments in
// float-float (w converted to hi/lo pairs once, Lambda stored as hi/lo
// floats), rounded to FP32.
// With agg given (the aggregated form): r = v - gpy with gpy = G_H P y
// from the caller, and the coarse value is y[agg[i]].
constexpr int kPanelThreads = 128;
__global__ void __launch_bounds__(kPanelThreads) panel_apply_kernel(
    const float *__restrict__ part, int N, int g, int s, const int *__restrict__ nptr,
    const int2 *__restrict__ pairs, const double *__restrict__ corr, const double *__restrict__ y,
    const double *__restrict__ v, const double *__restrict__ inv, double *__restrict__ w,
    const float2 *__restrict__ lam, float *__restrict__ sv, const int *__restrict__ agg,
    const double *__restrict__ gpy) {
    __shared__ double rs[3 * kMaxG];
    __shared__ float2 ws[3 * kMaxG];
    const int i = blockIdx.x, t = threadIdx.x;
    if (agg) {   // aggregated form: r = v - G_H P y, supplied by the caller's FMM
        if (t < 3 * g) rs[t] = v[3 * (size_t)i * g + t] - gpy[3 * (size_t)i * g + t];
    } else if (t < 3 * g) {
        const int m = t / 3, c = t - 3 * m;
        const size_t a = (size_t)i * g + m;
        double acc = 0.0;
        for (int q = 0; q < kSplit; ++q) acc += part[((size_t)q * N + a) * 3 + c];
        for (int e0 = nptr[i]; e0 < nptr[i + 1]; e0 += 4) {   // four pairs' loads in flight
            double cv[4], yv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + u;
                const bool ok = e < nptr[i + 1];
                cv[u] = ok ? corr[(size_t)e * g + m] : 0.0;
                yv[u] = ok ? y[3 * pairs[e].y + c] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) acc += cv[u] * yv[u];
        }
        rs[t] = v[3 * a + c] - acc;
    }
    __syncthreads();
    if (t < 3 * g) {
        const int m = t / 3, c = t - 3 * m;
        const double *row = inv + ((size_t)i * g + m) * g;
        double acc = y[3 * (agg ? agg[i] : i) + c];
        for (int n = 0; n < g; ++n) acc += row[n] * rs[3 * n + c];
        if (w) w[3 * ((size_t)i * g + m) + c] = acc;
        const float h = (float)acc;
        ws[t] = make_float2(h, (float)(acc - (double)h));
    }
    if (!lam) return;
    __syncthreads();
    for (int q = t; q < s; q += kPanelThreads) {
        const float2 *lr = lam + (size_t)q * g;
        float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f, h2 = 0.f, l2 = 0.f;
        for (int m = 0; m < g; ++m) {
            const float2 l = lr[m];
            dot2ff(h0, l0, l, ws[3 * m]);
            dot2ff(h1, l1, l, ws[3 * m + 1]);
            dot2ff(h2, l2, l, ws[3 * m + 2]);
        }
        const size_t k = (size_t)i * s + q;
        sv[3 * k + 0] = h0 + l0;
        sv[3 * k + 1] = h1 + l1;
        sv[3 * k + 2] = h2 + l2;
    }
}

// |(Ai Ac)[r][c] - delta_rc| for the sampled rows r = rows[blockIdx.y] and
// columns c = blockIdx.y + 7 blockIdx.x (FP64 sums), and bad[0] set when an
// entry of Ai is not finite (checked by the first row's blocks).
__global__ void inverse_check_kernel(const float *__restrict__ Ai, const float *__restrict__ Ac, int n,
                                     int4 rows4, int row5, double *__restrict__ err, int *__restrict__ bad) {
    const int rows[5] = {rows4.x, rows4.y, rows4.z, rows4.w, row5};
    const int ci = blockIdx.y, c = ci + 7 * blockIdx.x, r = rows[ci];
    const int ncol = gridDim.x;
    double acc = 0.0;
    if (c < n)
        for (int k = threadIdx.x; k < n; k += blockDim.x) acc += (double)Ai[(size_t)r * n + k] * Ac[(size_t)k * n + c];
    if (ci == 0)   // every entry of Ai once across the first row's blocks
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (size_t)n * n; i += (size_t)ncol * blockDim.x)
            if (!isfinite(Ai[i])) atomicOr(bad, 1);
    __shared__ double red[4];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        const double v = red[0] + red[1] + red[2] + red[3];
        err[(size_t)ci * ncol + blockIdx.x] = c < n ? fabs(v - (r == c ? 1.0 : 0.0)) : 0.0;
    }
}

}  // namespace

void TwoLevel::plan(const Geometry &G, int max_coarse) {
    ready_ = false;
    planned_ = false;
    const int P = G.n_panels, g = G.g, s = G.s, N = G.n_nodes();
    if (P < 2) return;
    P_ = P;
    g_ = g;
    s_seg_ = s;
    N_ = N;
    const int maxc = max_coarse > 0 ? max_coarse : kMaxCoarse;
    // panel centroids (node average) and arc lengths
    std::vector<double> cen(2 * P);
    std::vector<double> &pl = h_pl_;
    pl.assign(P, 0.0);
    h_c32_.resize(P);
    h_q32_.resize(N);
    h_pl32_.resize(P);
    for (int j = 0; j < P; ++j) {
        double sx = 0, sy = 0;
        for (int m = 0; m < g; ++m) {
            sx += G.node_xy[2 * (j * g + m)];
            sy += G.node_xy[2 * (j * g + m) + 1];
        }
        cen[2 * j] = sx / g;
        cen[2 * j + 1] = sy / g;
        double L = 0.0;
        for (int k = 0; k < s; ++k) {
            const double *q = &G.seg_xy[4 * (size_t)(j * s + k)];
            L += G.seg_w[j * s + k] * std::hypot(q[2] - q[0], q[3] - q[1]);
        }
        pl[j] = L;
        h_c32_[j] = make_float2((float)cen[2 * j], (float)cen[2 * j + 1]);
        h_pl32_[j] = (float)L;
    }
    for (int a = 0; a < N; ++a) h_q32_[a] = make_float2((float)G.node_xy[2 * a], (float)G.node_xy[2 * a + 1]);
    // coarse unknowns: one per panel (K = 1) while the padded count fits the
    // dense inverse, else aggregates of K panels consecutive in the Morton
    // order of the centroids (16 bits per axis over the centroids' box, ties
    // by panel index), K = ceil(P / (limit - 32))
    std::vector<int> &pagg = h_pagg_, &perm = h_perm_, &agg_of = h_agg_of_;
    pagg.clear();
    perm.resize(P);
    agg_of.resize(P);
    if ((P + kGJ - 1) / kGJ * kGJ <= maxc) {
        K_ = 1;
        for (int j = 0; j < P; ++j) perm[j] = agg_of[j] = j;
    } else {
        K_ = (P + (maxc - kGJ) - 1) / (maxc - kGJ);
        double lo[2] = {cen[0], cen[1]}, hi[2] = {cen[0], cen[1]};
        for (int j = 0; j < P; ++j)
            for (int d = 0; d < 2; ++d) {
                lo[d] = std::min(lo[d], cen[2 * j + d]);
                hi[d] = std::max(hi[d], cen[2 * j + d]);
            }
        std::vector<unsigned long long> key(P);
        for (int j = 0; j < P; ++j) {
            unsigned q[2];
            for (int d = 0; d < 2; ++d) {
                const double ext = hi[d] - lo[d];
                const double f = ext > 0.0 ? (cen[2 * j + d] - lo[d]) / ext : 0.0;
                q[d] = (unsigned)std::min(65535.0, std::floor(f * 65536.0));
            }
            unsigned long long k = 0;
            for (int b = 15; b >= 0; --b) k = (k << 2) | (((q[1] >> b) & 1u) << 1) | ((q[0] >> b) & 1u);
            key[j] = (k << 32) | (unsigned long long)j;
        }
        for (int j = 0; j < P; ++j) perm[j] = j;
        std::sort(perm.begin(), perm.end(), [&](int a, int b) { return key[a] < key[b]; });
    }
    for (int u = 0; u < P; ++u) {
        if (u % K_ == 0) pagg.push_back(u);
        agg_of[perm[u]] = int(pagg.size()) - 1;
    }
    pagg.push_back(P);
    nA_ = int(pagg.size()) - 1;
    n_pad_ = (nA_ + kGJ - 1) / kGJ * kGJ;
    // near panel pairs (i, j), i's list in j order: |c_i - c_j| < 1.5 (l_i + l_j);
    // candidates from a sweep over the centroids sorted by x
    std::vector<int> &nptr = h_nptr_;
    std::vector<int2> &pairs = h_pairs_;
    nptr.assign(P + 1, 0);
    pairs.clear();
    {
        std::vector<int> ord(P);
        for (int j = 0; j < P; ++j) ord[j] = j;
        std::sort(ord.begin(), ord.end(), [&](int a, int b) { return cen[2 * a] < cen[2 * b]; });
        double lmax = 0.0;
        for (int j = 0; j < P; ++j) lmax = std::max(lmax, pl[j]);
        std::vector<std::vector<int>> nb(P);
        for (int u = 0; u < P; ++u) {
            const int i = ord[u];
            for (int w = u; w < P; ++w) {
                const int j = ord[w];
                if (cen[2 * j] - cen[2 * i] >= 1.5 * (pl[i] + lmax)) break;
                const double dx = cen[2 * i] - cen[2 * j], dy = cen[2 * i + 1] - cen[2 * j + 1];
                const double lim = 1.5 * (pl[i] + pl[j]);
                if (dx * dx + dy * dy < lim * lim) {
                    nb[i].push_back(j);
                    if (j != i) nb[j].push_back(i);
                }
            }
        }
        for (int i = 0; i < P; ++i) {
            std::sort(nb[i].begin(), nb[i].end());
            nptr[i] = int(pairs.size());
            for (int j : nb[i]) pairs.push_back(make_int2(i, j));
        }
        nptr[P] = int(pairs.size());
    }
    planned_ = true;
}

cudaError_t TwoLevel::launch(const DevGeom &D, cudaStream_t st) {
    launched_ = false;
    if (!planned_) return cudaSuccess;
    const int P = P_, g = g_, s = s_seg_, N = N_;
    cudaError_t e;
    // pageable sources: each copy has left the host vector when the call
    // returns, so the vectors are released below.  A copy from pageable
    // memory first waits for the stream's earlier work: all uploads come
    // before the first kernel.
    auto up = [&](auto &buf, const auto &v) -> cudaError_t {
        cudaError_t r = buf.alloc(std::max<size_t>(v.size(), 1));
        if (r != cudaSuccess || v.empty()) return r;
        return cudaMemcpyAsync(buf.ptr, v.data(), v.size() * sizeof(v[0]), cudaMemcpyHostToDevice, st);
    };
    const size_t n_pairs = h_pairs_.size();
    if ((e = up(c32_, h_c32_)) != cudaSuccess || (e = up(q32_, h_q32_)) != cudaSuccess ||
        (e = up(plen_, h_pl_)) != cudaSuccess || (e = up(plen32_, h_pl32_)) != cudaSuccess ||
        (e = up(nptr_, h_nptr_)) != cudaSuccess || (e = up(pairs_, h_pairs_)) != cudaSuccess)
        return e;
    if (K_ > 1 && ((e = up(pagg_, h_pagg_)) != cudaSuccess || (e = up(agg_of_, h_agg_of_)) != cudaSuccess ||
                   (e = up(perm_, h_perm_)) != cudaSuccess))
        return e;
    if ((e = corr_.alloc(n_pairs * (size_t)g)) != cudaSuccess ||
        (e = Ainv_.alloc((size_t)n_pad_ * n_pad_)) != cudaSuccess || (e = s_.alloc(3 * (size_t)P)) != cudaSuccess ||
        (e = y_.alloc(3 * (size_t)P)) != cudaSuccess || (e = pan_.alloc((size_t)P)) != cudaSuccess || (e = pan2_.alloc((size_t)P)) != cudaSuccess ||
        (K_ == 1 && (e = part_.alloc((size_t)kSplit * 3 * N)) != cudaSuccess))
        return e;
    const int ncol = (n_pad_ + 6) / 7;   // columns per checked row and block
    if ((e = Ac_.alloc((size_t)n_pad_ * n_pad_)) != cudaSuccess ||
        (e = gj_tmp_.alloc((size_t)n_pad_ * n_pad_)) != cudaSuccess || (e = errs_.alloc((size_t)5 * ncol)) != cudaSuccess ||
        (e = bad_.alloc(1)) != cudaSuccess)
        return e;
    near_pairs_kernel<<<(unsigned)n_pairs, 32, 0, st>>>(pairs_.ptr, D.seg.ptr, D.segw.ptr, D.node_xy.ptr,
                                                        D.node_seg.ptr, D.node_seg2.ptr, q32_.ptr, c32_.ptr,
                                                        plen_.ptr, s, g, corr_.ptr);
    note_launch();
    // the coarse matrix into Ac_ (kept for the check below)
    if (K_ == 1) {
        coarse_matrix_kernel<<<n_pad_, 256, 0, st>>>(q32_.ptr, c32_.ptr, plen32_.ptr, nptr_.ptr, pairs_.ptr,
                                                    corr_.ptr, P, g, n_pad_, Ac_.ptr);
        note_launch();
    } else {
        coarse_agg_matrix_kernel<<<n_pad_, 256, 0, st>>>(q32_.ptr, c32_.ptr, plen32_.ptr, pagg_.ptr, perm_.ptr, nA_,
                                                        g, n_pad_, Ac_.ptr);
        coarse_agg_corr_kernel<<<(nA_ + 127) / 128, 128, 0, st>>>(pagg_.ptr, perm_.ptr, agg_of_.ptr, nA_, nptr_.ptr,
                                                                 pairs_.ptr, corr_.ptr, g, n_pad_, Ac_.ptr);
        note_launch(2);
    }
    // Gauss-Jordan steps between Ainv_ and gj_tmp_, the first reading Ac_
    // and the last writing Ainv_
    const int nb = n_pad_ / kGJ;
    const dim3 ug((n_pad_ + kGjTile - 1) / kGjTile, (n_pad_ + kGjTile - 1) / kGjTile);
    const float *src = Ac_.ptr;
    for (int k = 0; k < nb; ++k) {
        float *dst = ((nb - 1 - k) % 2 == 0) ? Ainv_.ptr : gj_tmp_.ptr;
        gj_step_kernel<<<ug, 256, 0, st>>>(src, dst, n_pad_, k);
        note_launch();
        src = dst;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // check the inverse on a few rows, on the device (a vanished or tiny
    // pivot shows up as non-finite entries or a large error)
    if ((e = cudaMemsetAsync(bad_.ptr, 0, sizeof(int), st)) != cudaSuccess) return e;
    inverse_check_kernel<<<dim3(ncol, 5), 128, 0, st>>>(Ainv_.ptr, Ac_.ptr, n_pad_,
                                                       make_int4(0, nA_ / 4, nA_ / 2, (3 * nA_) / 4), nA_ - 1,
                                                       errs_.ptr, bad_.ptr);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    n_pairs_ = int(n_pairs);
    std::vector<double>().swap(h_pl_);
    std::vector<float2>().swap(h_c32_);
    std::vector<float2>().swap(h_q32_);
    std::vector<float>().swap(h_pl32_);
    std::vector<int2>().swap(h_pairs_);
    std::vector<int>().swap(h_nptr_);
    std::vector<int>().swap(h_pagg_);
    std::vector<int>().swap(h_perm_);
    std::vector<int>().swap(h_agg_of_);
    launched_ = true;
    return cudaSuccess;
}

cudaError_t TwoLevel::finish(cudaStream_t st) {
    if (!launched_) return cudaSuccess;
    launched_ = false;
    cudaError_t e;
    std::vector<double> errs_h(errs_.n);
    int bad_h = 0;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess ||
        (e = cudaMemcpy(errs_h.data(), errs_.ptr, errs_.bytes(), cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemcpy(&bad_h, bad_.ptr, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return e;
    Ac_.release();
    gj_tmp_.release();
    errs_.release();
    bad_.release();
    // keep the one-level preconditioner unless the inverse is accurate
    if (bad_h) return cudaSuccess;
    double worst = 0.0;
    for (double v : errs_h) worst = std::max(worst, v);
    check_ = worst;
    if (!(worst < 1e-2)) return cudaSuccess;
    ready_ = true;
    return cudaSuccess;
}

cudaError_t TwoLevel::apply(const double *inv, const double *v, double *w, cudaStream_t st, const float2 *lam, int s,
                            float *sv) {
    const int P = P_, g = g_, N = P * g;
    if (K_ > 1) return cudaErrorNotSupported;   // aggregated: apply_stage1 / apply_stage2
    restrict_kernel<<<(3 * P + 255) / 256, 256, 0, st>>>(v, P, g, s_.ptr);
    coarse_solve_kernel<<<(P + kSolveRows - 1) / kSolveRows, 32 * kSolveRows, 0, st>>>(
        Ainv_.ptr, n_pad_, P, s_.ptr, plen32_.ptr, c32_.ptr, y_.ptr, pan_.ptr, pan2_.ptr);
    const int per_block = kMonoThreads * kMonoNodes;
    monopole_kernel<<<dim3((N + per_block - 1) / per_block, kSplit), kMonoThreads, 0, st>>>(q32_.ptr, pan_.ptr,
                                                                                         pan2_.ptr, P, N, part_.ptr);
    panel_apply_kernel<<<P, kPanelThreads, 0, st>>>(part_.ptr, N, g, s, nptr_.ptr, pairs_.ptr, corr_.ptr, y_.ptr, v,
                                                    inv, w, lam, sv, nullptr, nullptr);
    note_launch(4);
    return cudaGetLastError();
}

cudaError_t TwoLevel::apply_stage1(const double *v, double *py, cudaStream_t st) {
    const int N = P_ * g_;
    restrict_agg_kernel<<<(3 * nA_ + 255) / 256, 256, 0, st>>>(v, pagg_.ptr, perm_.ptr, nA_, g_, s_.ptr);
    coarse_solve_kernel<<<(nA_ + kSolveRows - 1) / kSolveRows, 32 * kSolveRows, 0, st>>>(
        Ainv_.ptr, n_pad_, nA_, s_.ptr, plen32_.ptr, c32_.ptr, y_.ptr, pan_.ptr, pan2_.ptr);
    spread_agg_kernel<<<(3 * N + 255) / 256, 256, 0, st>>>(y_.ptr, agg_of_.ptr, N, g_, py);
    note_launch(3);
    return cudaGetLastError();
}

cudaError_t TwoLevel::apply_stage2(const double *inv, const double *v, const double *gpy, double *w, cudaStream_t st,
                                   const float2 *lam, int s, float *sv) {
    panel_apply_kernel<<<P_, kPanelThreads, 0, st>>>(nullptr, P_ * g_, g_, s, nptr_.ptr, pairs_.ptr, corr_.ptr, y_.ptr,
                                                     v, inv, w, lam, sv, agg_of_.ptr, gpy);
    note_launch();
    return cudaGetLastError();
}

}  // namespace dc
