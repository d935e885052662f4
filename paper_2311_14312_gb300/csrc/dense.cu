// Plain dense FP64 form (the brute-force hybrid method of Sec. 4.5 / Table 1)
// and the small elementwise kernels shared by every form.
//
//  - K1  interpolation  sigma_bar = Pbar Pring^-1 sigma_ring   (Eq. 19)
//  - K9  dense hybrid rows  A_G = Gbar Pbar Pring^-1, A_F alike (Eq. 19, 27)
//        and the FP64 direct-sum layer potential at pixels (Eq. 23)
//  - K12 output conversion / 8-bit quantisation
#include <cuda_runtime.h>

#include "dc_internal.h"
#include "segint.cuh"

namespace dc {

namespace {

// ----------------------------------------------------------------- K1 --
__global__ void interp_kernel(const double *__restrict__ lam, const double *__restrict__ nv,
                              double *__restrict__ sv, int S, int s, int g) {
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
    sv[3 * (size_t)k + 0] = a0;
    sv[3 * (size_t)k + 1] = a1;
    sv[3 * (size_t)k + 2] = a2;
}

// ------------------------------------------------------ K9 assembly ----
// One thread per (target row i, panel j): the s segment integrals of panel
// j at node i, folded through Lambda into the g columns of that panel.
template <int MAXG>
__global__ void dense_assemble_kernel(const double *__restrict__ seg, const double *__restrict__ segw,
                                      const double *__restrict__ nxy, const int *__restrict__ nseg,
                                      const int *__restrict__ nseg2, const double *__restrict__ lam,
                                      double *__restrict__ AG, double *__restrict__ AF, int N,
                                      int n_panels, int s, int g) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y;
    if (j >= n_panels) return;
    double qx = nxy[2 * i], qy = nxy[2 * i + 1];
    int own1 = nseg[i], own2 = nseg2[i];
    double accG[MAXG], accF[MAXG];
#pragma unroll
    for (int m = 0; m < MAXG; ++m) accG[m] = accF[m] = 0.0;
    for (int kk = 0; kk < s; ++kk) {
        int k = j * s + kk;
        const double *q = seg + 4 * (size_t)k;
        double G, F;
        seg_gf_f64(qx, qy, __ldg(q), __ldg(q + 1), __ldg(q + 2), __ldg(q + 3), __ldg(segw + k),
                   k == own1 || k == own2, G, F);
        const double *lr = lam + (size_t)kk * g;
#pragma unroll
        for (int m = 0; m < MAXG; ++m) {
            if (m < g) {
                double l = __ldg(lr + m);
                accG[m] += G * l;
                accF[m] += F * l;
            }
        }
    }
    double *rg = AG + (size_t)i * N + (size_t)j * g;
    double *rf = AF + (size_t)i * N + (size_t)j * g;
#pragma unroll
    for (int m = 0; m < MAXG; ++m) {
        if (m < g) {
            rg[m] = accG[m];
            rf[m] = accF[m];
        }
    }
}

// y[i][c] = sum_col A[i][col] x[col][c]; one warp per row, fixed order.
__global__ void dense_gemv_kernel(const double *__restrict__ A, int N, const double *__restrict__ x,
                                  double *__restrict__ y) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= N) return;
    const double *row = A + (size_t)warp * N;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int col = lane; col < N; col += 32) {
        double a = __ldg(row + col);
        a0 += a * __ldg(x + 3 * (size_t)col + 0);
        a1 += a * __ldg(x + 3 * (size_t)col + 1);
        a2 += a * __ldg(x + 3 * (size_t)col + 2);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, off);
        a1 += __shfl_xor_sync(0xffffffffu, a1, off);
        a2 += __shfl_xor_sync(0xffffffffu, a2, off);
    }
    if (lane == 0) {
        y[3 * (size_t)warp + 0] = a0;
        y[3 * (size_t)warp + 1] = a1;
        y[3 * (size_t)warp + 2] = a2;
    }
}

// ------------------------------------------------ K9 direct-sum eval ----
// Each thread owns one target; segments stream through shared memory in
// tiles of blockDim.x.  Targets come either from a viewport grid or from
// an explicit point list.
constexpr int kEvalThreads = 128;

struct SegTile {
    double x1[kEvalThreads], y1[kEvalThreads], x2[kEvalThreads], y2[kEvalThreads];
    double w[kEvalThreads];
    double sb[kEvalThreads][3], mb[kEvalThreads][3];
};

__device__ void dense_eval_body(double qx, double qy, bool active, const double *__restrict__ seg,
                                const double *__restrict__ segw, const double *__restrict__ sbar,
                                const double *__restrict__ mbar, int S, SegTile &t,
                                double &u0, double &u1, double &u2) {
    u0 = u1 = u2 = 0.0;
    for (int base = 0; base < S; base += kEvalThreads) {
        int k = base + threadIdx.x;
        __syncthreads();
        if (k < S) {
            t.x1[threadIdx.x] = seg[4 * (size_t)k + 0];
            t.y1[threadIdx.x] = seg[4 * (size_t)k + 1];
            t.x2[threadIdx.x] = seg[4 * (size_t)k + 2];
            t.y2[threadIdx.x] = seg[4 * (size_t)k + 3];
            t.w[threadIdx.x] = segw[k];
            for (int c = 0; c < 3; ++c) {
                t.sb[threadIdx.x][c] = sbar[3 * (size_t)k + c];
                t.mb[threadIdx.x][c] = mbar[3 * (size_t)k + c];
            }
        }
        __syncthreads();
        int cnt = min(kEvalThreads, S - base);
        if (active) {
            for (int j = 0; j < cnt; ++j) {
                double G, F;
                seg_gf_f64(qx, qy, t.x1[j], t.y1[j], t.x2[j], t.y2[j], t.w[j], false, G, F);
                u0 += G * t.sb[j][0] + F * t.mb[j][0];
                u1 += G * t.sb[j][1] + F * t.mb[j][1];
                u2 += G * t.sb[j][2] + F * t.mb[j][2];
            }
        }
    }
}

__global__ void __launch_bounds__(kEvalThreads)
dense_eval_grid_kernel(const double *__restrict__ seg, const double *__restrict__ segw,
                       const double *__restrict__ sbar, const double *__restrict__ mbar, int S,
                       VpDev vp, double *__restrict__ u) {
    __shared__ SegTile tile;
    long long npix = (long long)vp.width * vp.height;
    long long pix = (long long)blockIdx.x * kEvalThreads + threadIdx.x;
    bool active = pix < npix;
    double qx = 0.0, qy = 0.0;
    if (active) {
        int r = (int)(pix / vp.width), c = (int)(pix - (long long)r * vp.width);
        qx = vp.x0 + (c + 0.5) * vp.dx;
        qy = vp.y0 + (r + 0.5) * vp.dy;
    }
    double u0, u1, u2;
    dense_eval_body(qx, qy, active, seg, segw, sbar, mbar, S, tile, u0, u1, u2);
    if (active) {
        double *o = u + 3 * pix;
        o[0] = u0;
        o[1] = u1;
        o[2] = u2;
    }
}

__global__ void __launch_bounds__(kEvalThreads)
dense_eval_points_kernel(const double *__restrict__ seg, const double *__restrict__ segw,
                         const double *__restrict__ sbar, const double *__restrict__ mbar, int S,
                         const double *__restrict__ xy, int n, double *__restrict__ u) {
    __shared__ SegTile tile;
    int i = blockIdx.x * kEvalThreads + threadIdx.x;
    bool active = i < n;
    double qx = active ? xy[2 * i] : 0.0, qy = active ? xy[2 * i + 1] : 0.0;
    double u0, u1, u2;
    dense_eval_body(qx, qy, active, seg, segw, sbar, mbar, S, tile, u0, u1, u2);
    if (active) {
        u[3 * (size_t)i + 0] = u0;
        u[3 * (size_t)i + 1] = u1;
        u[3 * (size_t)i + 2] = u2;
    }
}

// ------------------------------------------ panel block preconditioner --
// Diagonal blocks of G_H: B_j[m][n] = sum_{k in panel j} w_k int_{S_k} G(p, q_jm) dS
// Lambda[k][n] (the self-interaction of panel j, Eq. 19), one warp per panel:
// one lane per row, or with g <= 16 two lanes per row splitting the
// segments.  Segments within kBlockNearSeg chord lengths of the node (and
// its own, singular) take the FP64 closed form, the others the FP32 one on
// FP64 relative coordinates (smooth terms; the blocks only precondition).
// As in the coarse level's near pairs, the first sweep does the FP32 terms
// and lists the near (row, segment) entries, whose FP64 closed forms the
// warp then computes with all lanes busy; each row adds its entries in
// list order (entries beyond the list's room are computed in place).
constexpr double kBlockNearSeg = 8.0;
constexpr int kBlockNearCap = 512;
template <int MAXG>
__global__ void __launch_bounds__(32) panel_blocks_kernel(const double *__restrict__ seg,
                                                          const double *__restrict__ segw,
                                                          const double *__restrict__ nxy, const int *__restrict__ nseg,
                                                          const int *__restrict__ nseg2,
                                                          const double *__restrict__ lam,
                                                          double *__restrict__ blocks, int s, int g) {
    __shared__ int nl_tag[kBlockNearCap];   // row m << 16 | segment kk
    __shared__ double nl_g[kBlockNearCap];
    const int j = blockIdx.x, lane = threadIdx.x;
    const int halves = g <= 16 ? 2 : 1;
    const int m = halves == 2 ? (lane & 15) : lane, part = halves == 2 ? (lane >> 4) : 0;
    const bool valid = m < g;
    const int i = j * g + (valid ? m : 0);
    const double qx = nxy[2 * i], qy = nxy[2 * i + 1];
    const int own1 = nseg[i], own2 = nseg2[i];
    double acc[MAXG];
#pragma unroll
    for (int n = 0; n < MAXG; ++n) acc[n] = 0.0;
    int listed = 0;   // the same in every lane
    const int sweeps = (s + halves - 1) / halves;
    for (int it = 0; it < sweeps; ++it) {
        const int kk = part + it * halves;
        const bool act = valid && kk < s;
        const int k = j * s + (act ? kk : 0);
        const double *q = seg + 4 * (size_t)k;
        const double ax = q[0] - qx, ay = q[1] - qy, bx = q[2] - qx, by = q[3] - qy;
        const double dx = q[2] - q[0], dy = q[3] - q[1];
        const bool own = k == own1 || k == own2;
        const bool near = act && (own || seg_is_near(ax, ay, bx, by, dx, dy, kBlockNearSeg));
        const unsigned bal = __ballot_sync(0xffffffffu, near);
        double G = 0.0;
        bool add = false;
        if (near) {
            const int pos = listed + __popc(bal & ((1u << lane) - 1u));
            if (pos < kBlockNearCap) {
                nl_tag[pos] = (m << 16) | kk;
            } else {
                double F;
                seg_gf_f64(qx, qy, q[0], q[1], q[2], q[3], segw[k], own, G, F);
                add = true;
            }
        } else if (act) {
            G = segw[k] * (double)seg_g_far_f32(ax, ay, bx, by, dx, dy);
            add = true;
        }
        if (add) {
            const double *lr = lam + (size_t)kk * g;
#pragma unroll
            for (int n = 0; n < MAXG; ++n)
                if (n < g) acc[n] += G * lr[n];
        }
        listed += __popc(bal);
    }
    __syncwarp();
    const int n_list = min(listed, kBlockNearCap);
    for (int u = lane; u < n_list; u += 32) {
        const int mi = nl_tag[u] >> 16, k = j * s + (nl_tag[u] & 0xffff);
        const int ii = j * g + mi;
        const double *q = seg + 4 * (size_t)k;
        double G, F;
        seg_gf_f64(nxy[2 * ii], nxy[2 * ii + 1], q[0], q[1], q[2], q[3], segw[k], k == nseg[ii] || k == nseg2[ii],
                   G, F);
        nl_g[u] = G;
    }
    __syncwarp();
    if (halves == 2) {
#pragma unroll
        for (int n = 0; n < MAXG; ++n) acc[n] += __shfl_down_sync(0xffffffffu, acc[n], 16);
    }
    if (!valid || part != 0) return;
    for (int u = 0; u < n_list; ++u) {
        if ((nl_tag[u] >> 16) != m) continue;
        const double G = nl_g[u];
        const double *lr = lam + (size_t)(nl_tag[u] & 0xffff) * g;
#pragma unroll
        for (int n = 0; n < MAXG; ++n)
            if (n < g) acc[n] += G * lr[n];
    }
    double *row = blocks + ((size_t)j * g + m) * g;
#pragma unroll
    for (int n = 0; n < MAXG; ++n)
        if (n < g) row[n] = acc[n];
}

// In-place inverse of each g x g block by Gauss-Jordan elimination with
// partial pivoting in shared memory; info[j] = 1 if a pivot vanished.
__global__ void invert_blocks_kernel(double *__restrict__ blocks, int g, int *__restrict__ info) {
    __shared__ double a[kMaxG][2 * kMaxG + 1];
    __shared__ int piv;
    int j = blockIdx.x, t = threadIdx.x;   // t = column of the augmented matrix
    double *B = blocks + (size_t)j * g * g;
    for (int r = 0; r < g; ++r) {
        if (t < g) a[r][t] = B[r * g + t];
        if (t < g) a[r][g + t] = (r == t) ? 1.0 : 0.0;
    }
    __syncthreads();
    int bad = 0;
    for (int c = 0; c < g; ++c) {
        if (t == 0) {
            int best = c;
            for (int r = c + 1; r < g; ++r)
                if (fabs(a[r][c]) > fabs(a[best][c])) best = r;
            piv = best;
        }
        __syncthreads();
        int pr = piv;
        if (t < 2 * g && pr != c) {
            double tmp = a[c][t];
            a[c][t] = a[pr][t];
            a[pr][t] = tmp;
        }
        __syncthreads();
        double d = a[c][c];
        if (d == 0.0) bad = 1;
        __syncthreads();
        if (t < 2 * g && d != 0.0) a[c][t] /= d;
        __syncthreads();
        for (int r = 0; r < g; ++r) {
            if (r == c) continue;
            double f = a[r][c];
            __syncthreads();
            if (t < 2 * g) a[r][t] -= f * a[c][t];
            __syncthreads();
        }
    }
    for (int r = 0; r < g; ++r)
        if (t < g) B[r * g + t] = a[r][g + t];
    if (t == 0) info[j] = bad;
}

// y[j g + m][c] = sum_n inv_j[m][n] x[j g + n][c]
__global__ void block_apply_kernel(const double *__restrict__ inv, int n_panels, int g,
                                   const double *__restrict__ x, double *__restrict__ y) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_panels * g) return;
    int j = i / g, m = i - j * g;
    const double *row = inv + ((size_t)j * g + m) * g;
    const double *xs = x + (size_t)j * g * 3;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int n = 0; n < g; ++n) {
        double v = row[n];
        a0 += v * xs[3 * n + 0];
        a1 += v * xs[3 * n + 1];
        a2 += v * xs[3 * n + 2];
    }
    y[3 * (size_t)i + 0] = a0;
    y[3 * (size_t)i + 1] = a1;
    y[3 * (size_t)i + 2] = a2;
}

// ---------------------------------------------------------------- K12 --
__device__ __forceinline__ unsigned char quantise8(double v) {
    v = fmin(fmax(v, 0.0), 1.0);
    return (unsigned char)floor(255.0 * v + 0.5);
}

template <typename TIn>
__global__ void write_outputs_kernel(const TIn *__restrict__ u, long long n3, void *rgb,
                                     int rgb_dtype, unsigned char *rgb8) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n3) return;
    double v = (double)u[i];
    if (rgb) {
        if (rgb_dtype == DC_F64) static_cast<double *>(rgb)[i] = v;
        else static_cast<float *>(rgb)[i] = (float)v;
    }
    if (rgb8) rgb8[i] = quantise8(v);
}

__global__ void mu_kernel(const double *__restrict__ up, const double *__restrict__ um,
                          double *__restrict__ mu, int n3) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n3) mu[i] = up[i] - um[i];
}

__global__ void rhs_kernel(const double *__restrict__ up, const double *__restrict__ um,
                           const double *__restrict__ fmu, double *__restrict__ b, int n3) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n3) b[i] = 0.5 * (up[i] + um[i]) - fmu[i];
}

}  // namespace

cudaError_t launch_interp(const DevGeom &G, const double *node_vals, double *seg_vals,
                          cudaStream_t st) {
    int th = 256;
    interp_kernel<<<(G.S + th - 1) / th, th, 0, st>>>(G.lambda.ptr, node_vals, seg_vals, G.S, G.s,
                                                      G.g); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_dense_assemble(const DevGeom &G, double *AG, double *AF, cudaStream_t st) {
    int th = 64;
    dim3 grid((G.n_panels + th - 1) / th, G.N);
#define DC_ASM(MG)                                                                              \
    dense_assemble_kernel<MG><<<grid, th, 0, st>>>(G.seg.ptr, G.segw.ptr, G.node_xy.ptr,        \
                                                   G.node_seg.ptr, G.node_seg2.ptr,             \
                                                   G.lambda.ptr, AG, AF, G.N, G.n_panels, G.s, \
                                                   G.g)
    if (G.g <= 4) DC_ASM(4);
    else if (G.g <= 8) DC_ASM(8);
    else if (G.g <= 16) DC_ASM(16);
    else DC_ASM(32);
#undef DC_ASM
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_dense_gemv(const double *A, int N, const double *x, double *y, cudaStream_t st) {
    int th = 256;
    long long threads = (long long)N * 32;
    dense_gemv_kernel<<<(unsigned)((threads + th - 1) / th), th, 0, st>>>(A, N, x, y); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_dense_eval_grid(const DevGeom &G, const double *sbar, const double *mbar,
                                   const VpDev &vp, double *u, cudaStream_t st) {
    long long npix = (long long)vp.width * vp.height;
    if (npix == 0) return cudaSuccess;
    unsigned blocks = (unsigned)((npix + kEvalThreads - 1) / kEvalThreads);
    dense_eval_grid_kernel<<<blocks, kEvalThreads, 0, st>>>(G.seg.ptr, G.segw.ptr, sbar, mbar, G.S,
                                                            vp, u); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_dense_eval_points(const DevGeom &G, const double *sbar, const double *mbar,
                                     const double *xy, int n, double *u, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    dense_eval_points_kernel<<<(n + kEvalThreads - 1) / kEvalThreads, kEvalThreads, 0, st>>>(
        G.seg.ptr, G.segw.ptr, sbar, mbar, G.S, xy, n, u); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_panel_block_inverse(const DevGeom &G, double *inv, int *info, cudaStream_t st) {
    int th = 32;
#define DC_PB(MG)                                                                                 \
    panel_blocks_kernel<MG><<<G.n_panels, th, 0, st>>>(G.seg.ptr, G.segw.ptr, G.node_xy.ptr,      \
                                                       G.node_seg.ptr, G.node_seg2.ptr,           \
                                                       G.lambda.ptr, inv, G.s, G.g)
    if (G.g <= 4) DC_PB(4);
    else if (G.g <= 8) DC_PB(8);
    else if (G.g <= 16) DC_PB(16);
    else DC_PB(32);
#undef DC_PB
    note_launch();
    invert_blocks_kernel<<<G.n_panels, 2 * kMaxG, 0, st>>>(inv, G.g, info); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_block_apply(const double *inv, int n_panels, int g, const double *x, double *y,
                               cudaStream_t st) {
    int n = n_panels * g, th = 256;
    block_apply_kernel<<<(n + th - 1) / th, th, 0, st>>>(inv, n_panels, g, x, y); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_write_outputs(const double *u, long long n, void *rgb, int rgb_dtype,
                                 unsigned char *rgb8, cudaStream_t st) {
    long long n3 = 3 * n;
    if (n3 == 0) return cudaSuccess;
    int th = 256;
    write_outputs_kernel<double><<<(unsigned)((n3 + th - 1) / th), th, 0, st>>>(u, n3, rgb,
                                                                                 rgb_dtype, rgb8); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_write_outputs_f32(const float *u, long long n, void *rgb, int rgb_dtype,
                                     unsigned char *rgb8, cudaStream_t st) {
    long long n3 = 3 * n;
    if (n3 == 0) return cudaSuccess;
    int th = 256;
    write_outputs_kernel<float><<<(unsigned)((n3 + th - 1) / th), th, 0, st>>>(u, n3, rgb,
                                                                               rgb_dtype, rgb8); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_mu(const DevGeom &G, double *mu, cudaStream_t st) {
    int n3 = 3 * G.N, th = 256;
    mu_kernel<<<(n3 + th - 1) / th, th, 0, st>>>(G.u_plus.ptr, G.u_minus.ptr, mu, n3); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_rhs(const DevGeom &G, const double *Fmu, double *b, cudaStream_t st) {
    int n3 = 3 * G.N, th = 256;
    rhs_kernel<<<(n3 + th - 1) / th, th, 0, st>>>(G.u_plus.ptr, G.u_minus.ptr, Fmu, b, n3); note_launch();
    return cudaGetLastError();
}

}  // namespace dc
