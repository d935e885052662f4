// K8: restarted GMRES on the device for the three colour channels at once
// (Sec. 5.5: x = GMRES(f, x0, y, eps) with the FMM or dense operator as f).
//
// Each channel has its own Krylov space; vectors are [N][3] with the channel
// fastest, FP64 except the basis of inner solves of a refinement, which is
// kept in FP32 (their tolerance is far above FP32 rounding).  Arnoldi uses classical Gram-Schmidt with a second
// (re-orthogonalisation) pass when the first one cancelled more than 90% of
// the vector's norm in some channel (a looser form of the criterion of
// Daniel, Gragg, Kaufman and Stewart; the flag is set and read on the
// device, so a skipped pass costs two empty launches); Givens rotations
// (run by the last block of the orthogonalisation), the residual estimate
// and the triangular solve run on the device.  Reductions are two-stage with a fixed order, so results are
// bit-reproducible.  The host learns of convergence from per-channel flags
// copied back after every iteration, read kPollLag iterations late so that
// the device queue never drains; iterations enqueued after the last channel
// converged leave the solution unchanged (the Givens step ignores finished
// channels).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>

#include "dc_internal.h"

namespace dc {

namespace {

constexpr int kChunk = 1024;     // rows per partial dot-product block
constexpr int kDotThreads = 256;
constexpr int kPollRing = 4;     // pinned flag slots / events
constexpr int kPollLag = 1;      // iterations between enqueue and flag read
constexpr double kPredictMargin = 4.0;   // see the convergence look-ahead in gmres_solve
constexpr size_t kGivensSmem = 40 * 1024;   // Givens step staged in shared memory up to this
// second Gram-Schmidt pass when ||w after||^2 < kReorthEta2 ||w before||^2
// (0.01: more than 90% of the norm cancelled; on the bench drawing the
// solve took 23.1 ms with the classical 1/2, 22.5 ms with 0.01 and 22.7 ms
// with no second pass at all, at the same iteration counts)
#ifndef DC_REORTH_ETA2
#define DC_REORTH_ETA2 0.01
#endif
constexpr double kReorthEta2 = DC_REORTH_ETA2;
#ifndef DC_BASIS32_MIN_TOL
#define DC_BASIS32_MIN_TOL 1e-6
#endif
constexpr double kBasis32MinTol = DC_BASIS32_MIN_TOL;   // FP32 Krylov basis from this tolerance up

// partial[(j * nchunk + chunk) * 3 + c] = sum over rows of the chunk of
// V_j[i][c] * w[i][c]
__global__ void dots_partial_kernel(const double *__restrict__ V, size_t vstride,
                                    const double *__restrict__ w, int N, int nchunk,
                                    double *__restrict__ partial) {
    int chunk = blockIdx.x, j = blockIdx.y;
    const double *v = V + (size_t)j * vstride;
    int lo = chunk * kChunk, hi = min(N, lo + kChunk);
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int i = lo + threadIdx.x; i < hi; i += kDotThreads) {
        a0 += v[3 * (size_t)i + 0] * w[3 * (size_t)i + 0];
        a1 += v[3 * (size_t)i + 1] * w[3 * (size_t)i + 1];
        a2 += v[3 * (size_t)i + 2] * w[3 * (size_t)i + 2];
    }
    __shared__ double red[3][kDotThreads];
    red[0][threadIdx.x] = a0;
    red[1][threadIdx.x] = a1;
    red[2][threadIdx.x] = a2;
    __syncthreads();
    for (int s = kDotThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 3)
        partial[((size_t)j * nchunk + chunk) * 3 + threadIdx.x] = red[threadIdx.x][0];
}

// One Gram-Schmidt pass's dot products h_j = V_j . w for j < nj, fused
// with their finalisation: block (chunk, j) writes its partial sums, and the
// last block of column j to finish (counted in count[j], which it resets)
// adds the partials in chunk order into hpass[j] and the Hessenberg column
// hcol[j] (= hpass on the first pass, += on the second).  Deterministic.
template <typename B>
__global__ void __launch_bounds__(kDotThreads) gs_dots_kernel(const B *__restrict__ V, size_t vstride,
                                                              const double *__restrict__ w, int N, int nchunk,
                                                              double *__restrict__ partial,
                                                              unsigned *__restrict__ count,
                                                              double *__restrict__ hpass, double *__restrict__ hcol,
                                                              int first, const int *__restrict__ skip) {
    if (skip && *skip) return;   // a second pass that is not needed
    const int chunk = blockIdx.x, j = blockIdx.y;
    const B *v = V + (size_t)j * vstride;
    const int lo = chunk * kChunk, hi = min(N, lo + kChunk);
    // a thread's few products are summed in the basis type, the rest in FP64
    B ab[3] = {B(0), B(0), B(0)};
    for (int i = lo + threadIdx.x; i < hi; i += kDotThreads)
        for (int c = 0; c < 3; ++c) ab[c] += v[3 * (size_t)i + c] * (B)w[3 * (size_t)i + c];
    double a[3] = {(double)ab[0], (double)ab[1], (double)ab[2]};
    __shared__ double red[kDotThreads / 32][3];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    for (int c = 0; c < 3; ++c)
        for (int off = 16; off > 0; off >>= 1) a[c] += __shfl_xor_sync(0xffffffffu, a[c], off);
    if (lane == 0)
        for (int c = 0; c < 3; ++c) red[wp][c] = a[c];
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int q = 0; q < kDotThreads / 32; ++q) t += red[q][threadIdx.x];
        partial[((size_t)j * nchunk + chunk) * 3 + threadIdx.x] = t;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&count[j], 1u) == (unsigned)(nchunk - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x < 3) {
        const int c = threadIdx.x;
        double t = 0.0;
        for (int ch = 0; ch < nchunk; ++ch) t += __ldcg(partial + ((size_t)j * nchunk + ch) * 3 + c);
        hpass[3 * j + c] = t;
        hcol[3 * j + c] = first ? t : hcol[3 * j + c] + t;
    }
    if (threadIdx.x == 0) count[j] = 0u;
}

// h[j][c] (= or +=) sum_chunk partial
__global__ void dots_finalize_kernel(const double *__restrict__ partial, int nchunk, int nj,
                                     double *__restrict__ h, int accumulate) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nj * 3) return;
    int j = t / 3, c = t - 3 * j;
    double s = 0.0;
    for (int ch = 0; ch < nchunk; ++ch) s += partial[((size_t)j * nchunk + ch) * 3 + c];
    h[t] = accumulate ? h[t] + s : s;
}

// nrm[c] = sqrt(sum_chunk partial) (the norms of one [N][3] vector)
__global__ void norm_finalize_kernel(const double *__restrict__ partial, int nchunk, double *__restrict__ nrm) {
    int c = threadIdx.x;
    if (c >= 3) return;
    double s = 0.0;
    for (int ch = 0; ch < nchunk; ++ch) s += partial[(size_t)ch * 3 + c];
    nrm[c] = sqrt(fmax(s, 0.0));
}

// out[i][c] = in[i][c] / nrm[c] (0 where nrm[c] is 0); out2, the operator's
// input buffer when it has one, gets the same (stored) value
__global__ void scale_kernel(const double *__restrict__ in, const double *__restrict__ nrm,
                             double *__restrict__ out, int N, double *__restrict__ out2 = nullptr) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * N) return;
    int c = t % 3;
    double n = nrm[c];
    const double v = (n > 0.0) ? in[t] / n : 0.0;
    out[t] = v;
    if (out2) out2[t] = v;
}

// The same for an FP32 basis: one reciprocal per channel and block, the
// element rounded to FP32 and the operator's buffer given that FP32 value
__global__ void scale32_kernel(const double *__restrict__ in, const double *__restrict__ nrm,
                               float *__restrict__ out, int N, double *__restrict__ out2) {
    __shared__ double inv[3];
    if (threadIdx.x < 3) {
        const double n = nrm[threadIdx.x];
        inv[threadIdx.x] = n > 0.0 ? 1.0 / n : 0.0;
    }
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * N) return;
    const float v = (float)(in[t] * inv[t % 3]);
    out[t] = v;
    if (out2) out2[t] = (double)v;
}

// r = b - Ax
__global__ void residual_kernel(const double *__restrict__ b, const double *__restrict__ Ax,
                                double *__restrict__ r, int n3) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n3) r[t] = b[t] - Ax[t];
}

// sqrt of a finalized sum of squares
__global__ void sqrt3_kernel(double *v) {
    int c = threadIdx.x;
    if (c < 3) v[c] = sqrt(fmax(v[c], 0.0));
}

struct GivensState {
    // per channel
    double *R;      // [3][m][m] column-major upper triangle: R[c][k*m + j]
    double *cs;     // [3][m]
    double *sn;     // [3][m]
    double *e;      // [3][m+1]
    double *y;      // [3][m]
    int *active;    // [3]
    int *kc;        // [3] columns used in this cycle
    double *resid;  // [3] current |e[k+1]|
    const int *fault = nullptr;   // the operator's wait-limit flag, or null
};

// Start of a cycle: e = (beta, 0, ...); active = beta > thr.
__global__ void cycle_start_kernel(GivensState g, const double *__restrict__ beta,
                                   const double *__restrict__ thr, int m) {
    int c = threadIdx.x;
    if (c >= 3) return;
    for (int k = 0; k <= m; ++k) g.e[c * (m + 1) + k] = 0.0;
    g.e[c * (m + 1)] = beta[c];
    g.active[c] = beta[c] > thr[c] ? 1 : 0;
    g.kc[c] = 0;
    g.resid[c] = beta[c];
}

// One Givens step for channel c by one warp (lane 0 runs the sequential
// chain), the new column and the earlier rotations staged in smem (3 (k + 1)
// doubles) when it is given, else read from global memory.
__device__ void givens_step_warp(GivensState g, const double *__restrict__ hcol, const double *__restrict__ hnext,
                                 const double *__restrict__ thr, int k, int m, int c, int lane, double *smem) {
    if (!g.active[c]) return;
    const double *gcs = g.cs + c * m, *gsn = g.sn + c * m;
    double *col, *cs, *sn;
    if (smem) {
        col = smem;
        cs = col + (k + 1);
        sn = cs + (k + 1);
        for (int j = lane; j <= k; j += 32) col[j] = hcol[3 * j + c];
        for (int j = lane; j < k; j += 32) {
            cs[j] = gcs[j];
            sn[j] = gsn[j];
        }
    } else {
        col = g.R + (size_t)c * m * m + (size_t)k * m;
        cs = g.cs + c * m;
        sn = g.sn + c * m;
        for (int j = lane; j <= k; j += 32) col[j] = hcol[3 * j + c];
    }
    __syncwarp();
    if (lane == 0) {
        for (int j = 0; j < k; ++j) {
            double a = col[j], b = col[j + 1];
            col[j] = cs[j] * a + sn[j] * b;
            col[j + 1] = -sn[j] * a + cs[j] * b;
        }
        double *e = g.e + c * (m + 1);
        double hn = hnext[c];
        double den = hypot(col[k], hn);
        double cc = (den > 0.0) ? col[k] / den : 1.0;
        double ss = (den > 0.0) ? hn / den : 0.0;
        g.cs[c * m + k] = cc;
        g.sn[c * m + k] = ss;
        col[k] = den;
        e[k + 1] = -ss * e[k];
        e[k] = cc * e[k];
        double res = fabs(e[k + 1]);
        g.resid[c] = res;
        g.kc[c] = k + 1;
        if (res <= thr[c] || !(hn > 0.0) || !(den > 0.0)) g.active[c] = 0;
        if (g.fault && *g.fault) g.active[c] = 0;   // the operator gave up a wait: end the cycle
    }
    __syncwarp();
    if (smem) {
        double *R = g.R + (size_t)c * m * m + (size_t)k * m;
        for (int j = lane; j <= k; j += 32) R[j] = col[j];
    }
}

constexpr int kOrthThreads = 192;   // 3 x 64 elements per block: an element's channel is its index mod 3

// One Gram-Schmidt pass's update w -= V h with the squared norms of the
// result (and, on the first pass, of w before it) summed per block; the last
// block to finish (counter, which it resets) adds the block sums in block
// order, sets hnext = ||w|| per channel, on the first pass decides whether
// the second one is needed (skip), and runs the Givens step when this is the
// last pass of the iteration.  pass 1 returns at once when skip is set.
// Dynamic shared memory: 9 (k + 1) doubles for the Givens step, or none (the
// step then works in global memory).
template <typename B>
__global__ void __launch_bounds__(kOrthThreads) orth_norm_givens_kernel(
    const B *__restrict__ V, size_t vstride, const double *__restrict__ h, int nj, double *__restrict__ w,
    int N, double *__restrict__ npart, int pass, int *__restrict__ skip, unsigned *__restrict__ counter,
    double *__restrict__ hnext, GivensState g, const double *__restrict__ hcol, const double *__restrict__ thr,
    int k, int m, int staged) {
    if (pass == 1 && *skip) return;
    extern __shared__ double gsm[];
    __shared__ double sq[2][kOrthThreads];
    __shared__ bool last;
    __shared__ int keep[3];
    const int t = blockIdx.x * kOrthThreads + threadIdx.x;
    double a = 0.0, a0 = 0.0;
    if (t < 3 * N) {
        const int c = t % 3;
        a = a0 = w[t];
        if constexpr (sizeof(B) == 8) {
            int j = 0;
            for (; j + 4 <= nj; j += 4) {
                const double v0 = V[(size_t)j * vstride + t], v1 = V[(size_t)(j + 1) * vstride + t];
                const double v2 = V[(size_t)(j + 2) * vstride + t], v3 = V[(size_t)(j + 3) * vstride + t];
                a -= h[3 * j + c] * v0;
                a -= h[3 * (j + 1) + c] * v1;
                a -= h[3 * (j + 2) + c] * v2;
                a -= h[3 * (j + 3) + c] * v3;
            }
            for (; j < nj; ++j) a -= h[3 * j + c] * V[(size_t)j * vstride + t];
        } else {
            // FP32 basis: (V h)[t] summed in FP32, eight loads in flight
            float sv = 0.f;
            int j = 0;
            for (; j + 8 <= nj; j += 8) {
                float v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = V[(size_t)(j + u) * vstride + t];
#pragma unroll
                for (int u = 0; u < 8; ++u) sv = fmaf((float)h[3 * (j + u) + c], v[u], sv);
            }
            for (; j < nj; ++j) sv = fmaf((float)h[3 * j + c], V[(size_t)j * vstride + t], sv);
            a -= (double)sv;
        }
        w[t] = a;
    }
    sq[0][threadIdx.x] = a * a;
    sq[1][threadIdx.x] = a0 * a0;
    __syncthreads();
    if (threadIdx.x < 3) {
        double s1 = 0.0, s0 = 0.0;
        for (int u = threadIdx.x; u < kOrthThreads; u += 3) {
            s1 += sq[0][u];
            s0 += sq[1][u];
        }
        npart[6 * blockIdx.x + threadIdx.x] = s1;
        npart[6 * blockIdx.x + 3 + threadIdx.x] = s0;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1u;
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (c < 3) {
        double s1 = 0.0, s0 = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32) {
            s1 += __ldcg(npart + 6 * b + c);
            s0 += __ldcg(npart + 6 * b + 3 + c);
        }
        for (int off = 16; off > 0; off >>= 1) {
            s1 += __shfl_xor_sync(0xffffffffu, s1, off);
            s0 += __shfl_xor_sync(0xffffffffu, s0, off);
        }
        if (lane == 0) {
            hnext[c] = sqrt(fmax(s1, 0.0));
            keep[c] = s1 >= kReorthEta2 * s0;
        }
    }
    __syncthreads();
    bool givens = true;
    if (pass == 0) {
        givens = keep[0] && keep[1] && keep[2];   // no second pass: this is the last
        if (threadIdx.x == 0) *skip = givens ? 1 : 0;
    }
    if (threadIdx.x == 0) *counter = 0u;
    __threadfence();
    if (givens && c < 3) givens_step_warp(g, hcol, hnext, thr, k, m, c, lane, staged ? gsm + (size_t)c * 3 * (k + 1) : nullptr);
}

// Back substitution R y = e for each channel (kc[c] columns).
__global__ void backsolve_kernel(GivensState g, int m) {
    int c = threadIdx.x;
    if (c >= 3) return;
    int n = g.kc[c];
    const double *R = g.R + (size_t)c * m * m;
    double *y = g.y + c * m;
    const double *e = g.e + c * (m + 1);
    for (int i = n - 1; i >= 0; --i) {
        double s = e[i];
        for (int j = i + 1; j < n; ++j) s -= R[(size_t)j * m + i] * y[j];
        double d = R[(size_t)i * m + i];
        y[i] = (d != 0.0) ? s / d : 0.0;
    }
    for (int i = n; i < m; ++i) y[i] = 0.0;
}

// x[i][c] += sum_{j < kc[c]} y[c][j] V_j[i][c]
template <typename B>
__global__ void solution_update_kernel(GivensState g, const B *__restrict__ V, size_t vstride,
                                       double *__restrict__ x, int N, int m) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    for (int c = 0; c < 3; ++c) {
        int n = g.kc[c];
        const double *y = g.y + c * m;
        double a = x[3 * (size_t)i + c];
        for (int j = 0; j < n; ++j) a += y[j] * (double)V[(size_t)j * vstride + 3 * (size_t)i + c];
        x[3 * (size_t)i + c] = a;
    }
}

}  // namespace

struct GmresWork {
    int N = 0, m = 0, nchunk = 0;
    DevBuf<double> V, w, r, Ax, partial, hcol, hpass, hnext, small, npart;
    DevBuf<float> V32;   // the basis of solves that keep it in FP32
    DevBuf<double> R, cs, sn, e, y;
    DevBuf<int> flags;
    DevBuf<unsigned> count;   // [m + 1] blocks done per column (gs_dots_kernel), kept at zero
    double *host = nullptr;   // pinned: resid[3], active-as-double[3], norms[3]
    int *poll = nullptr;      // pinned [kPollRing][3] copies of the active flags
    double *pollr = nullptr;  // pinned [kPollRing][3] copies of the residual estimates
    cudaEvent_t ev[kPollRing] = {};
    ~GmresWork() {
        if (host) cudaFreeHost(host);
        if (poll) cudaFreeHost(poll);
        if (pollr) cudaFreeHost(pollr);
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
    }
    cudaError_t ensure(int N_, int m_) {
        if (N_ == N && m_ == m) return cudaSuccess;
        N = N_;
        m = m_;
        nchunk = (N + kChunk - 1) / kChunk;
        cudaError_t e_;
#define DC_TRY(x)               \
    if ((e_ = (x)) != cudaSuccess) \
        return e_;
        DC_TRY(V.alloc((size_t)(m + 1) * N * 3));
        DC_TRY(V32.alloc((size_t)(m + 1) * N * 3));
        DC_TRY(w.alloc((size_t)N * 3));
        DC_TRY(r.alloc((size_t)N * 3));
        DC_TRY(Ax.alloc((size_t)N * 3));
        DC_TRY(partial.alloc((size_t)(m + 1) * nchunk * 3));
        DC_TRY(count.alloc((size_t)(m + 2)));   // gs_dots columns, then the orth_norm_givens counter
        DC_TRY(npart.alloc((size_t)6 * ((3 * (size_t)N + kOrthThreads - 1) / kOrthThreads)));
        DC_TRY(hcol.alloc((size_t)(m + 1) * 3));
        DC_TRY(hpass.alloc((size_t)(m + 1) * 3));
        DC_TRY(hnext.alloc(3));
        DC_TRY(small.alloc(32));
        DC_TRY(R.alloc((size_t)3 * m * m));
        DC_TRY(cs.alloc((size_t)3 * m));
        DC_TRY(sn.alloc((size_t)3 * m));
        DC_TRY(e.alloc((size_t)3 * (m + 1)));
        DC_TRY(y.alloc((size_t)3 * m));
        DC_TRY(flags.alloc(8));
        if (!host) DC_TRY(cudaMallocHost(reinterpret_cast<void **>(&host), 16 * sizeof(double)));
        if (!poll) DC_TRY(cudaMallocHost(reinterpret_cast<void **>(&poll), kPollRing * 3 * sizeof(int)));
        if (!pollr) DC_TRY(cudaMallocHost(reinterpret_cast<void **>(&pollr), kPollRing * 3 * sizeof(double)));
        for (auto &e : ev)
            if (!e) DC_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
#undef DC_TRY
        return cudaSuccess;
    }
    GivensState gs() {
        GivensState g;
        g.R = R.ptr;
        g.cs = cs.ptr;
        g.sn = sn.ptr;
        g.e = e.ptr;
        g.y = y.ptr;
        g.active = flags.ptr;
        g.kc = flags.ptr + 3;
        g.resid = small.ptr + 8;
        return g;
    }
};

GmresWork *gmres_work_create() { return new GmresWork(); }

namespace {
__global__ void axpy_kernel(double *__restrict__ x, const double *__restrict__ d, int n3) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n3) x[t] += d[t];
}
// y[i][c] = a[c] x[i][c] + b[c] z[i][c] (z may be null: then b[c] alone)
__global__ void combine3_kernel(const double *x, const double *z, double *y, int n3,
                                double a0, double a1, double a2, double b0, double b1, double b2) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n3) return;
    int c = t % 3;
    double a = c == 0 ? a0 : (c == 1 ? a1 : a2), b = c == 0 ? b0 : (c == 1 ? b1 : b2);
    // a = 0 ignores x (it may hold anything, even non-finite values)
    y[t] = (a != 0.0 ? a * x[t] : 0.0) + b * (z ? z[t] : 1.0);
}
__global__ void mask3_kernel(double *__restrict__ v, int n3, int k0, int k1, int k2) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n3) return;
    int c = t % 3;
    int keep = c == 0 ? k0 : (c == 1 ? k1 : k2);
    if (!keep) v[t] = 0.0;
}
}  // namespace

cudaError_t vec_residual(const double *b, const double *Ax, double *r, int n3, cudaStream_t st) {
    residual_kernel<<<(n3 + 255) / 256, 256, 0, st>>>(b, Ax, r, n3); note_launch();
    return cudaGetLastError();
}

cudaError_t vec_axpy(double *x, const double *d, int n3, cudaStream_t st) {
    axpy_kernel<<<(n3 + 255) / 256, 256, 0, st>>>(x, d, n3); note_launch();
    return cudaGetLastError();
}

cudaError_t vec_combine3(const double *x, const double *z, double *y, int N, const double a[3],
                         const double b[3], cudaStream_t st) {
    int n3 = 3 * N;
    combine3_kernel<<<(n3 + 255) / 256, 256, 0, st>>>(x, z, y, n3, a[0], a[1], a[2], b[0], b[1], b[2]);
    note_launch();
    return cudaGetLastError();
}

cudaError_t vec_mask3(double *v, int N, const int keep[3], cudaStream_t st) {
    int n3 = 3 * N;
    mask3_kernel<<<(n3 + 255) / 256, 256, 0, st>>>(v, n3, keep[0], keep[1], keep[2]); note_launch();
    return cudaGetLastError();
}
void gmres_work_destroy(GmresWork *w) { delete w; }

namespace {

// nrm[c] = || v[:, c] ||_2 (device), through the deterministic dot kernels.
cudaError_t norms(GmresWork &W, const double *v, double *nrm, cudaStream_t st) {
    dim3 grid(W.nchunk, 1);
    dots_partial_kernel<<<grid, kDotThreads, 0, st>>>(v, 0, v, W.N, W.nchunk, W.partial.ptr); note_launch();
    dots_finalize_kernel<<<1, 32, 0, st>>>(W.partial.ptr, W.nchunk, 1, nrm, 0); note_launch();
    sqrt3_kernel<<<1, 32, 0, st>>>(nrm); note_launch();
    return cudaGetLastError();
}

__global__ void add_into_kernel(double *__restrict__ dst, const double *__restrict__ src, int n,
                                int assign) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) dst[t] = assign ? src[t] : dst[t] + src[t];
}

}  // namespace

cudaError_t vec_norms3(GmresWork *Wp, const double *v, int N, double host_out[3], cudaStream_t st) {
    GmresWork &W = *Wp;
    cudaError_t e = W.ensure(N, W.m > 0 ? W.m : 1);
    if (e != cudaSuccess) return e;
    if ((e = norms(W, v, W.small.ptr + 16, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(host_out, W.small.ptr + 16, 3 * sizeof(double), cudaMemcpyDeviceToHost,
                             st)) != cudaSuccess)
        return e;
    return cudaStreamSynchronize(st);
}

cudaError_t vec_dots3(GmresWork *Wp, const double *u, const double *v, int N, double host_out[3],
                      cudaStream_t st) {
    GmresWork &W = *Wp;
    cudaError_t e = W.ensure(N, W.m > 0 ? W.m : 1);
    if (e != cudaSuccess) return e;
    dim3 grid(W.nchunk, 1);
    dots_partial_kernel<<<grid, kDotThreads, 0, st>>>(u, 0, v, N, W.nchunk, W.partial.ptr); note_launch();
    dots_finalize_kernel<<<1, 32, 0, st>>>(W.partial.ptr, W.nchunk, 1, W.small.ptr + 20, 0); note_launch();
    if ((e = cudaMemcpyAsync(host_out, W.small.ptr + 20, 3 * sizeof(double), cudaMemcpyDeviceToHost,
                             st)) != cudaSuccess)
        return e;
    return cudaStreamSynchronize(st);
}

cudaError_t gmres_solve(GmresWork *Wp, Operator &A, int N, const double *b, double *x, bool x0_zero, bool trust_estimate,
                        double tol,
                        int restart, int max_iter, cudaStream_t st, GmresResult &res,
                        std::string &err) {
    GmresWork &W = *Wp;
    res = GmresResult();
    int m = restart < 1 ? 1 : restart;
    if (max_iter < m) m = max_iter < 1 ? 1 : max_iter;
    cudaError_t ce = W.ensure(N, m);
    if (ce != cudaSuccess) {
        err = std::string("gmres workspace: ") + cudaGetErrorString(ce);
        return ce;
    }
    const size_t vs = (size_t)N * 3;
    const int th = 256;
    // the column counters of gs_dots_kernel start at zero (each last block
    // resets its own; this guards against a launch that failed midway)
    if ((ce = cudaMemsetAsync(W.count.ptr, 0, W.count.bytes(), st)) != cudaSuccess) return ce;
    GivensState gs = W.gs();
    gs.fault = A.fault_flag();
    double *bnorm = W.small.ptr;        // [3]
    double *thr = W.small.ptr + 3;      // [3]
    double *beta = W.small.ptr + 12;    // [3] (slots 8..10 hold resid)
    // ||b|| and thresholds tol * ||b||
    if ((ce = norms(W, b, bnorm, st)) != cudaSuccess) return ce;
    double hb[3];
    if ((ce = cudaMemcpyAsync(hb, bnorm, 3 * sizeof(double), cudaMemcpyDeviceToHost, st)) !=
        cudaSuccess)
        return ce;
    if ((ce = cudaStreamSynchronize(st)) != cudaSuccess) return ce;
    double hthr[3];
    for (int c = 0; c < 3; ++c) hthr[c] = tol * hb[c];
    if ((ce = cudaMemcpyAsync(thr, hthr, 3 * sizeof(double), cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
        return ce;
    // An inner solve (stopped by the Givens estimate at a tolerance far above
    // FP32 rounding, on an operator with its own input / output buffers)
    // keeps its basis in FP32: half the bytes, and the Gram-Schmidt products
    // at the FP32 rate; the operator is applied to the stored FP32 vectors,
    // so the Arnoldi relation holds for them.  Other solves keep FP64.
    const bool bufs = A.in_buffer() && A.out_buffer();
    const bool b32 = bufs && trust_estimate && tol >= kBasis32MinTol;
    int total = 0;
    bool done_all = false;
    // a cycle that ends with every channel converged by the Givens estimate
    // while the recomputed residual has not even halved since the cycle
    // began means the operator's own error (an inexact, e.g. FP32, matvec)
    // is reached: stop, the caller's refinement takes over
    bool est_done = false;
    double prev_beta[3] = {0, 0, 0};
    bool first = true;
    while (true) {
        // r = b - A x ; beta = ||r||  (r = b for a zero start)
        if (first && x0_zero) {
            if ((ce = cudaMemcpyAsync(W.r.ptr, b, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, st)) !=
                cudaSuccess)
                return ce;
        } else {
            if ((ce = A.apply(x, W.Ax.ptr, st)) != cudaSuccess) return ce;
            res.n_matvec++;
            residual_kernel<<<(3 * N + th - 1) / th, th, 0, st>>>(b, W.Ax.ptr, W.r.ptr, 3 * N); note_launch();
        }
        first = false;
        if ((ce = norms(W, W.r.ptr, beta, st)) != cudaSuccess) return ce;
        double hbeta[3];
        if ((ce = cudaMemcpyAsync(hbeta, beta, 3 * sizeof(double), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess)
            return ce;
        if ((ce = cudaStreamSynchronize(st)) != cudaSuccess) return ce;
        bool any = false;
        for (int c = 0; c < 3; ++c) {
            res.rel_resid[c] = hb[c] > 0 ? hbeta[c] / hb[c] : 0.0;
            res.true_rel_resid[c] = res.rel_resid[c];
            if (hbeta[c] > hthr[c]) any = true;
        }
        if (!any) {
            done_all = true;
            break;
        }
        if (total >= max_iter) break;
        if (est_done) {
            bool progress = false;
            for (int c = 0; c < 3; ++c)
                if (hbeta[c] > hthr[c] && hbeta[c] < 0.5 * prev_beta[c]) progress = true;
            if (!progress) {
                res.stagnated = 1;
                break;
            }
        }
        for (int c = 0; c < 3; ++c) prev_beta[c] = hbeta[c];
        est_done = false;
        cycle_start_kernel<<<1, 32, 0, st>>>(gs, beta, thr, m); note_launch();
        // an operator with its own input / output buffers reads v_k from the
        // former (written by the scale kernels) and leaves A v_k in the latter
        double *in_buf = A.in_buffer(), *out_buf = A.out_buffer();
        double *wv = bufs ? out_buf : W.w.ptr;
        if (b32) scale32_kernel<<<(3 * N + th - 1) / th, th, 0, st>>>(W.r.ptr, beta, W.V32.ptr, N, in_buf);
        else scale_kernel<<<(3 * N + th - 1) / th, th, 0, st>>>(W.r.ptr, beta, W.V.ptr, N, bufs ? in_buf : nullptr);
        note_launch();
        int k = 0;
        for (; k < m && total < max_iter; ++k) {
            double *vk = W.V.ptr + (size_t)k * vs;
            if ((ce = bufs ? A.apply_buffers(st) : A.apply(vk, wv, st)) != cudaSuccess) return ce;
            res.n_matvec++;
            // CGS2: two passes of h = V^T w, w -= V h
            // classical Gram-Schmidt, h = V^T w, w -= V h, and h_{k+1,k} =
            // ||w|| per channel; the second pass runs only when the first
            // one cancelled too much of w (its kernels read the flag)
            int *skip = W.flags.ptr + 6;   // after active[3], kc[3]
            const size_t gsm = (size_t)9 * (k + 1) * sizeof(double);
            const int staged = gsm <= kGivensSmem ? 1 : 0;
            const int nb = (3 * N + kOrthThreads - 1) / kOrthThreads;
            for (int pass = 0; pass < 2; ++pass) {
                dim3 grid(W.nchunk, k + 1);
                if (b32) {
                    gs_dots_kernel<float><<<grid, kDotThreads, 0, st>>>(
                        W.V32.ptr, vs, wv, N, W.nchunk, W.partial.ptr, W.count.ptr, W.hpass.ptr, W.hcol.ptr,
                        pass == 0, pass == 0 ? nullptr : skip);
                    orth_norm_givens_kernel<float><<<nb, kOrthThreads, staged ? gsm : 0, st>>>(
                        W.V32.ptr, vs, W.hpass.ptr, k + 1, wv, N, W.npart.ptr, pass, skip, W.count.ptr + (m + 1),
                        W.hnext.ptr, gs, W.hcol.ptr, thr, k, m, staged);
                } else {
                    gs_dots_kernel<double><<<grid, kDotThreads, 0, st>>>(
                        W.V.ptr, vs, wv, N, W.nchunk, W.partial.ptr, W.count.ptr, W.hpass.ptr, W.hcol.ptr,
                        pass == 0, pass == 0 ? nullptr : skip);
                    orth_norm_givens_kernel<double><<<nb, kOrthThreads, staged ? gsm : 0, st>>>(
                        W.V.ptr, vs, W.hpass.ptr, k + 1, wv, N, W.npart.ptr, pass, skip, W.count.ptr + (m + 1),
                        W.hnext.ptr, gs, W.hcol.ptr, thr, k, m, staged);
                }
                note_launch(2);
            }
            if (b32)
                scale32_kernel<<<(3 * N + th - 1) / th, th, 0, st>>>(wv, W.hnext.ptr,
                                                                     W.V32.ptr + (size_t)(k + 1) * vs, N, in_buf);
            else
                scale_kernel<<<(3 * N + th - 1) / th, th, 0, st>>>(wv, W.hnext.ptr, W.V.ptr + (size_t)(k + 1) * vs,
                                                                   N, bufs ? in_buf : nullptr);
            note_launch();
            total++;
            const int slot = k % kPollRing;
            if ((ce = cudaMemcpyAsync(W.poll + 3 * slot, gs.active, 3 * sizeof(int),
                                      cudaMemcpyDeviceToHost, st)) != cudaSuccess)
                return ce;
            if (trust_estimate && (ce = cudaMemcpyAsync(W.pollr + 3 * slot, gs.resid, 3 * sizeof(double),
                                                        cudaMemcpyDeviceToHost, st)) != cudaSuccess)
                return ce;
            if ((ce = cudaEventRecord(W.ev[slot], st)) != cudaSuccess) return ce;
            // flags of iteration k - kPollLag (slot reuse is safe: it was read
            // kPollLag iterations ago, before this iteration was enqueued)
            const int done = k - kPollLag;
            if (done >= 0) {
                const int ps = done % kPollRing;
                if ((ce = cudaEventSynchronize(W.ev[ps])) != cudaSuccess) return ce;
                const int *f = W.poll + 3 * ps;
                if (!f[0] && !f[1] && !f[2]) {
                    est_done = true;
                    break;
                }
                // When the estimates of iterations done - 1 and done, extrapolated
                // geometrically, put every active channel within kPredictMargin of
                // its threshold at iteration k, wait for k before enqueuing k + 1:
                // a wrong guess costs one host round trip, a right one saves an
                // iteration that would only be discarded.
                if (trust_estimate && done >= 1 && k + 1 < m && total < max_iter) {
                    const double *r1 = W.pollr + 3 * ps, *r0 = W.pollr + 3 * ((done - 1) % kPollRing);
                    bool near = true;
                    for (int c = 0; c < 3; ++c) {
                        if (!f[c]) continue;
                        const double q = r0[c] > 0.0 ? fmin(1.0, r1[c] / r0[c]) : 1.0;
                        if (!(r1[c] * q <= kPredictMargin * hthr[c])) near = false;
                    }
                    if (near) {
                        if ((ce = cudaEventSynchronize(W.ev[slot])) != cudaSuccess) return ce;
                        const int *fk = W.poll + 3 * slot;
                        if (!fk[0] && !fk[1] && !fk[2]) {
                            est_done = true;
                            break;
                        }
                    }
                }
            }
        }
        backsolve_kernel<<<1, 32, 0, st>>>(gs, m); note_launch();
        if (b32) solution_update_kernel<float><<<(N + th - 1) / th, th, 0, st>>>(gs, W.V32.ptr, vs, x, N, m);
        else solution_update_kernel<double><<<(N + th - 1) / th, th, 0, st>>>(gs, W.V.ptr, vs, x, N, m);
        note_launch();
        int hkc[3];
        if ((ce = cudaMemcpyAsync(hkc, gs.kc, 3 * sizeof(int), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess)
            return ce;
        if ((ce = cudaStreamSynchronize(st)) != cudaSuccess) return ce;
        for (int c = 0; c < 3; ++c) res.iters[c] += hkc[c];
        if (est_done && trust_estimate) {
            // the caller recomputes the residual with its own (more exact)
            // operator: stop at the Givens estimate
            double hres[3];
            if ((ce = cudaMemcpyAsync(hres, gs.resid, 3 * sizeof(double), cudaMemcpyDeviceToHost, st)) !=
                cudaSuccess)
                return ce;
            if ((ce = cudaStreamSynchronize(st)) != cudaSuccess) return ce;
            for (int c = 0; c < 3; ++c) res.rel_resid[c] = hb[c] > 0 ? hres[c] / hb[c] : 0.0;
            done_all = true;
            break;
        }
    }
    res.converged = done_all ? 1 : 0;
    return cudaGetLastError();
}

}  // namespace dc
