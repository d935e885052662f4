// Quadtree anti-aliasing (Sec. 7) and the device-side pieces it needs: an
// exclusive scan, and leaf location plus counting sort of arbitrary points
// for the FMM evaluation kernels.
//
// A pixel whose closed square meets a closed segment of the solve polyline
// is refined in a quadtree of its own: a cell of level k < m that meets a
// segment splits into its four quarters (lower-left, lower-right,
// upper-left, upper-right), every other cell is one sample at its centre
// with weight 4^-k, and the pixel's colour is the weighted sum (the
// area-weighted mean of Sec. 7).  Pixels that meet no segment keep the
// render's centre sample.  Corners and centres are x0 + (c + f) dx with a
// dyadic fraction f, and the segment / rectangle test uses explicitly
// rounded products and differences (no contraction into FMAs), so every
// decision is the IEEE result of the written expression.
#include <cuda_runtime.h>

#include <climits>
#include <string>

#include "dc_internal.h"
#include "fmm_impl.h"

namespace dc {

// ------------------------------------------------------------- scan ----
namespace {

constexpr int kScanThreads = 256, kScanPer = 8, kScanTile = kScanThreads * kScanPer;

// Exclusive scan of one tile of 2048 elements per block; the block's total
// goes to bsum[blockIdx.x].  in and out may alias (each thread reads its
// own elements before writing them).
template <typename TI, typename TO>
__global__ void __launch_bounds__(kScanThreads) scan_tile_kernel(const TI *in, TO *out, long long n,
                                                                 long long *bsum) {
    __shared__ long long wtot[kScanThreads / 32];
    const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanPer;
    long long v[kScanPer];
    long long s = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        const long long i = base + k;
        v[k] = i < n ? (long long)in[i] : 0;
        s += v[k];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wtot[w] = x;
    __syncthreads();
    if (w == 0) {
        long long t = lane < kScanThreads / 32 ? wtot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < kScanThreads / 32) wtot[lane] = t;
    }
    __syncthreads();
    long long ex = x - s + (w > 0 ? wtot[w - 1] : 0);
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        const long long i = base + k;
        if (i < n) out[i] = (TO)ex;
        ex += v[k];
    }
    if (threadIdx.x == kScanThreads - 1) bsum[blockIdx.x] = ex;
}

template <typename TO>
__global__ void scan_add_kernel(TO *out, long long n, const long long *boff) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (TO)((long long)out[i] + boff[i / kScanTile]);
}

template <typename TI, typename TO>
cudaError_t scan_rec(const TI *in, TO *out, long long n, ScanWork &w, int depth, cudaStream_t st) {
    if (depth >= ScanWork::kLevels) return cudaErrorInvalidValue;
    const long long nb = (n + kScanTile - 1) / kScanTile;
    cudaError_t e = w.lv[depth].ensure(size_t(nb));
    if (e != cudaSuccess) return e;
    long long *bs = w.lv[depth].ptr;
    scan_tile_kernel<TI, TO><<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, n, bs);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (nb == 1) return cudaMemcpyAsync(w.total.ptr, bs, sizeof(long long), cudaMemcpyDeviceToDevice, st);
    if ((e = scan_rec<long long, long long>(bs, bs, nb, w, depth + 1, st)) != cudaSuccess) return e;
    scan_add_kernel<TO><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out, n, bs);
    note_launch();
    return cudaGetLastError();
}

}  // namespace

cudaError_t scan_exclusive(const int *in, int *out, long long n, ScanWork &w, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    cudaError_t e = w.total.ensure(1);
    if (e != cudaSuccess) return e;
    return scan_rec<int, int>(in, out, n, w, 0, st);
}

// ------------------------------------------------ points into leaves ----
namespace {

__global__ void locate_count_kernel(const double *__restrict__ xy, int n, const int *__restrict__ child0,
                                    const double *__restrict__ cc, double x0, double y0, double w0,
                                    int *__restrict__ leaf_of, int *__restrict__ cnt, int *__restrict__ bad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x = xy[2 * i], y = xy[2 * i + 1];
    if (!(x >= x0 && x < x0 + w0 && y >= y0 && y < y0 + w0)) {
        leaf_of[i] = -1;
        atomicExch(bad, 1);
        return;
    }
    int c = 0;
    for (int guard = 0; guard < 64 && child0[c] >= 0; ++guard)
        c = child0[c] + (x >= cc[2 * c] ? 1 : 0) + (y >= cc[2 * c + 1] ? 2 : 0);
    leaf_of[i] = c;
    atomicAdd(&cnt[c], 1);
}

__global__ void chunks_kernel(const int *__restrict__ cnt, int *__restrict__ chunks, int n_cells, int item) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n_cells) chunks[c] = (cnt[c] + item - 1) / item;
    if (c == n_cells) chunks[c] = 0;
}

__global__ void scatter_points_kernel(const double *__restrict__ xy, int n, const int *__restrict__ leaf_of,
                                      const int *__restrict__ start, int *__restrict__ fill,
                                      int *__restrict__ perm, double *__restrict__ sxy) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = leaf_of[i];
    if (c < 0) return;
    const int pos = start[c] + atomicAdd(&fill[c], 1);
    perm[pos] = i;
    sxy[2 * pos] = xy[2 * i];
    sxy[2 * pos + 1] = xy[2 * i + 1];
}

// one work item per chunk of `item` points of a leaf
template <bool F32>
__global__ void items_kernel(const int *__restrict__ cnt, const int *__restrict__ start,
                             const int *__restrict__ ioff, int n_cells, int item, Tile *__restrict__ t32,
                             int4 *__restrict__ t64) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    const int k = cnt[c];
    for (int j = 0, q = ioff[c]; j < k; j += item, ++q) {
        const int m = min(item, k - j);
        if (F32) t32[q] = Tile{c, start[c] + j, 0, m, 0, 0};
        else t64[q] = make_int4(c, start[c] + j, m, 0);
    }
}

}  // namespace

cudaError_t PointSort::run(const double *xy, int n, const int *child0, const double *cc, int n_cells,
                           double x0, double y0, double w0, int item, bool f32, cudaStream_t st,
                           int &n_items, bool &outside) {
    n_items = 0;
    outside = false;
    cudaError_t e;
    if ((e = leaf_of.ensure(size_t(n))) != cudaSuccess || (e = cnt.ensure(size_t(n_cells) + 1)) != cudaSuccess ||
        (e = start.ensure(size_t(n_cells) + 1)) != cudaSuccess ||
        (e = ioff.ensure(size_t(n_cells) + 1)) != cudaSuccess || (e = perm.ensure(size_t(n))) != cudaSuccess ||
        (e = sxy.ensure(2 * size_t(n))) != cudaSuccess || (e = flag.ensure(1)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(cnt.ptr, 0, sizeof(int) * (size_t(n_cells) + 1), st)) != cudaSuccess ||
        (e = cudaMemsetAsync(flag.ptr, 0, sizeof(int), st)) != cudaSuccess)
        return e;
    const int th = 256;
    locate_count_kernel<<<(n + th - 1) / th, th, 0, st>>>(xy, n, child0, cc, x0, y0, w0, leaf_of.ptr, cnt.ptr,
                                                          flag.ptr);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = scan_exclusive(cnt.ptr, start.ptr, n_cells + 1, scan, st)) != cudaSuccess) return e;
    chunks_kernel<<<(n_cells + 1 + th - 1) / th, th, 0, st>>>(cnt.ptr, ioff.ptr, n_cells, item);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = scan_exclusive(ioff.ptr, ioff.ptr, n_cells + 1, scan, st)) != cudaSuccess) return e;
    long long tot = 0;
    int bad = 0;
    if ((e = cudaMemcpyAsync(&tot, scan.total.ptr, sizeof(long long), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&bad, flag.ptr, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return e;
    if (bad) {
        outside = true;
        return cudaSuccess;
    }
    n_items = int(tot);
    // the leaf counters become fill counters
    if ((e = cudaMemsetAsync(flag.ptr, 0, sizeof(int), st)) != cudaSuccess) return e;
    if (f32) {
        if ((e = items32.ensure(size_t(std::max(n_items, 1)))) != cudaSuccess) return e;
    } else {
        if ((e = items64.ensure(size_t(std::max(n_items, 1)))) != cudaSuccess) return e;
    }
    if (f32)
        items_kernel<true><<<(n_cells + th - 1) / th, th, 0, st>>>(cnt.ptr, start.ptr, ioff.ptr, n_cells, item,
                                                                   items32.ptr, nullptr);
    else
        items_kernel<false><<<(n_cells + th - 1) / th, th, 0, st>>>(cnt.ptr, start.ptr, ioff.ptr, n_cells, item,
                                                                    nullptr, items64.ptr);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(cnt.ptr, 0, sizeof(int) * size_t(n_cells), st)) != cudaSuccess) return e;
    scatter_points_kernel<<<(n + th - 1) / th, th, 0, st>>>(xy, n, leaf_of.ptr, start.ptr, cnt.ptr, perm.ptr,
                                                            sxy.ptr);
    note_launch();
    return cudaGetLastError();
}

// ----------------------------------------------------- anti-aliasing ----
namespace {

constexpr int kAaStack = 32;

// Closed segment p-q against the closed rectangle [x0, x1] x [y0, y1]:
// the boxes overlap and the corners are not all strictly on one side of
// the segment's line (separating axes).
__device__ __forceinline__ bool seg_meets_rect(double px, double py, double qx, double qy, double x0, double y0,
                                               double x1, double y1) {
    const double lox = fmin(px, qx), hix = fmax(px, qx), loy = fmin(py, qy), hiy = fmax(py, qy);
    if (!(hix >= x0 && lox <= x1 && hiy >= y0 && loy <= y1)) return false;
    const double ex = __dsub_rn(qx, px), ey = __dsub_rn(qy, py);
    const double s0 = __dsub_rn(__dmul_rn(ex, __dsub_rn(y0, py)), __dmul_rn(ey, __dsub_rn(x0, px)));
    const double s1 = __dsub_rn(__dmul_rn(ex, __dsub_rn(y0, py)), __dmul_rn(ey, __dsub_rn(x1, px)));
    const double s2 = __dsub_rn(__dmul_rn(ex, __dsub_rn(y1, py)), __dmul_rn(ey, __dsub_rn(x0, px)));
    const double s3 = __dsub_rn(__dmul_rn(ex, __dsub_rn(y1, py)), __dmul_rn(ey, __dsub_rn(x1, px)));
    const bool pos = s0 > 0.0 && s1 > 0.0 && s2 > 0.0 && s3 > 0.0;
    const bool neg = s0 < 0.0 && s1 < 0.0 && s2 < 0.0 && s3 < 0.0;
    return !(pos || neg);
}

// x0 + f dx with the product and the sum each rounded once
__device__ __forceinline__ double grid_coord(double x0, double f, double d) { return __dadd_rn(x0, __dmul_rn(f, d)); }

__device__ __forceinline__ double clamp_idx(double v, double lo, double hi) { return fmin(fmax(v, lo), hi); }

// Pixels whose closed square meets segment s, one thread per (segment,
// viewport).  pass 0 counts them per pixel; pass 1 lists the segment under
// each (positions from the counts' scan).  The column and row ranges are a
// superset (one pixel of padding); the exact test decides.
__global__ void aa_touch_kernel(const double *__restrict__ seg, int S, const VpDev *__restrict__ vps,
                                int *__restrict__ cnt, const int *__restrict__ off, int *__restrict__ ids,
                                int pass) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const VpDev vp = vps[blockIdx.y];
    if (vp.width <= 0 || vp.height <= 0) return;
    const double px = seg[4 * s], py = seg[4 * s + 1], qx = seg[4 * s + 2], qy = seg[4 * s + 3];
    const double lox = fmin(px, qx), hix = fmax(px, qx), loy = fmin(py, qy), hiy = fmax(py, qy);
    const double Wm = vp.width - 1, Hm = vp.height - 1;
    const double fc0 = floor((lox - vp.x0) / vp.dx) - 1.0, fc1 = floor((hix - vp.x0) / vp.dx) + 1.0;
    const double fr0 = floor((loy - vp.y0) / vp.dy) - 1.0, fr1 = floor((hiy - vp.y0) / vp.dy) + 1.0;
    if (!(fc1 >= 0.0 && fc0 <= Wm && fr1 >= 0.0 && fr0 <= Hm)) return;
    const int c0 = (int)clamp_idx(fc0, 0.0, Wm), c1 = (int)clamp_idx(fc1, 0.0, Wm);
    const int R0 = (int)clamp_idx(fr0, 0.0, Hm), R1 = (int)clamp_idx(fr1, 0.0, Hm);
    const double ex = qx - px, ey = qy - py;
    for (int c = c0; c <= c1; ++c) {
        // rows the segment can reach over columns c - 1 .. c + 1
        int r0 = R0, r1 = R1;
        if (ex != 0.0) {
            const double xa = vp.x0 + (c - 1) * vp.dx, xb = vp.x0 + (c + 2) * vp.dx;
            const double ta = fmin(fmax((xa - px) / ex, 0.0), 1.0), tb = fmin(fmax((xb - px) / ex, 0.0), 1.0);
            const double ya = py + ta * ey, yb = py + tb * ey;
            const double g0 = floor((fmin(ya, yb) - vp.y0) / vp.dy) - 1.0;
            const double g1 = floor((fmax(ya, yb) - vp.y0) / vp.dy) + 1.0;
            r0 = max(R0, (int)clamp_idx(g0, 0.0, Hm));
            r1 = min(R1, (int)clamp_idx(g1, 0.0, Hm));
        }
        const double x0 = grid_coord(vp.x0, (double)c, vp.dx), x1 = grid_coord(vp.x0, (double)(c + 1), vp.dx);
        for (int r = r0; r <= r1; ++r) {
            const double y0 = grid_coord(vp.y0, (double)r, vp.dy), y1 = grid_coord(vp.y0, (double)(r + 1), vp.dy);
            if (!seg_meets_rect(px, py, qx, qy, x0, y0, x1, y1)) continue;
            const long long p = vp.offset + (long long)r * vp.width + c;
            if (pass == 0) atomicAdd(&cnt[p], 1);
            else ids[off[p] + atomicAdd(&cnt[p], 1)] = s;
        }
    }
}

__global__ void aa_flags_kernel(const int *__restrict__ off, int *__restrict__ flag, long long n) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) flag[p] = off[p + 1] > off[p] ? 1 : 0;
    if (p == n) flag[p] = 0;
}

__global__ void aa_compact_kernel(const int *__restrict__ off, const int *__restrict__ eidx, long long n,
                                  long long *__restrict__ edge) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n && off[p + 1] > off[p]) edge[eidx[p]] = p;
}

__device__ __forceinline__ int find_vp(const VpDev *vps, int n_vp, long long p) {
    int lo = 0, hi = n_vp - 1;   // last viewport with offset <= p and pixels
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (vps[mid].offset <= p) lo = mid;
        else hi = mid - 1;
    }
    while (lo > 0 && (long long)vps[lo].width * vps[lo].height == 0) --lo;
    return lo;
}

// One thread per edge pixel: depth-first walk of its cells (children in
// the order lower-left, lower-right, upper-left, upper-right).  PASS 0
// counts the samples, PASS 1 writes them (centre, weight) from soff[e].
template <int PASS>
__global__ void aa_subdiv_kernel(const long long *__restrict__ edge, int n_edge, const VpDev *__restrict__ vps,
                                 int n_vp, const int *__restrict__ off, const int *__restrict__ ids,
                                 const double *__restrict__ seg, int levels, int *__restrict__ ns,
                                 const int *__restrict__ soff, double *__restrict__ sxy, double *__restrict__ sw) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_edge) return;
    const long long p = edge[e];
    const VpDev vp = vps[find_vp(vps, n_vp, p)];
    const long long loc = p - vp.offset;
    const int r = int(loc / vp.width), c = int(loc % vp.width);
    const int a = off[p], b = off[p + 1];
    unsigned char sk[kAaStack];
    int si[kAaStack], sj[kAaStack];
    int top = 0, count = 0;
    sk[0] = 0;
    si[0] = 0;
    sj[0] = 0;
    top = 1;
    const int base = PASS == 1 ? soff[e] : 0;
    while (top > 0) {
        --top;
        const int k = sk[top], i = si[top], j = sj[top];
        const double h = ldexp(1.0, -k);
        const double x0 = grid_coord(vp.x0, c + i * h, vp.dx), x1 = grid_coord(vp.x0, c + (i + 1) * h, vp.dx);
        const double y0 = grid_coord(vp.y0, r + j * h, vp.dy), y1 = grid_coord(vp.y0, r + (j + 1) * h, vp.dy);
        bool hit = false;
        if (k < levels)
            for (int t = a; t < b && !hit; ++t) {
                const double *q = seg + 4 * (size_t)ids[t];
                hit = seg_meets_rect(q[0], q[1], q[2], q[3], x0, y0, x1, y1);
            }
        if (!hit || top + 4 > kAaStack) {
            if (PASS == 1) {
                const int o = base + count;
                sxy[2 * (size_t)o] = grid_coord(vp.x0, c + (i + 0.5) * h, vp.dx);
                sxy[2 * (size_t)o + 1] = grid_coord(vp.y0, r + (j + 0.5) * h, vp.dy);
                sw[o] = h * h;
            }
            ++count;
            continue;
        }
        // pushed in reverse so that they pop in the child order
        for (int q = 3; q >= 0; --q) {
            sk[top] = (unsigned char)(k + 1);
            si[top] = 2 * i + (q & 1);
            sj[top] = 2 * j + (q >> 1);
            ++top;
        }
    }
    if (PASS == 0) ns[e] = count;
}

__device__ __forceinline__ unsigned char aa_quantise8(double v) {   // the render's output rule
    v = fmin(fmax(v, 0.0), 1.0);
    return (unsigned char)floor(255.0 * v + 0.5);
}

__global__ void aa_reduce_kernel(const long long *__restrict__ edge, int n_edge, const int *__restrict__ soff,
                                 const double *__restrict__ sw, const double *__restrict__ u, void *rgb,
                                 int rgb_dtype, unsigned char *rgb8) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_edge) return;
    const long long p = edge[e];
    double acc[3] = {0.0, 0.0, 0.0};
    for (int j = soff[e]; j < soff[e + 1]; ++j) {
        const double w = sw[j];
        for (int ch = 0; ch < 3; ++ch) acc[ch] += w * u[3 * (size_t)j + ch];
    }
    for (int ch = 0; ch < 3; ++ch) {
        const size_t o = 3 * (size_t)p + ch;
        if (rgb) {
            if (rgb_dtype == DC_F64) static_cast<double *>(rgb)[o] = acc[ch];
            else static_cast<float *>(rgb)[o] = (float)acc[ch];
        }
        if (rgb8) rgb8[o] = aa_quantise8(acc[ch]);
    }
}

}  // namespace

cudaError_t AaWork::prepare(const DevGeom &G, const VpDev *vps_host, int n_vp, long long total_px, int levels,
                            cudaStream_t st, std::string &err) {
    n_edge = 0;
    n_samples = 0;
    if (total_px <= 0 || n_vp <= 0 || G.S == 0) return cudaSuccess;
    if (total_px >= INT_MAX) {
        err = "anti-aliasing: at most 2^31 - 2 pixels per call";
        return cudaErrorInvalidValue;
    }
    const long long n = total_px;
    cudaError_t e;
    if ((e = vps.ensure(size_t(n_vp))) != cudaSuccess ||
        (e = cudaMemcpyAsync(vps.ptr, vps_host, sizeof(VpDev) * n_vp, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cnt.ensure(size_t(n) + 1)) != cudaSuccess || (e = off.ensure(size_t(n) + 1)) != cudaSuccess ||
        (e = cudaMemsetAsync(cnt.ptr, 0, sizeof(int) * (size_t(n) + 1), st)) != cudaSuccess)
        return e;
    const int th = 256;
    const dim3 tg((G.S + th - 1) / th, n_vp);
    aa_touch_kernel<<<tg, th, 0, st>>>(G.seg.ptr, G.S, vps.ptr, cnt.ptr, nullptr, nullptr, 0);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = scan_exclusive(cnt.ptr, off.ptr, n + 1, scan, st)) != cudaSuccess) return e;
    long long entries = 0;
    if ((e = cudaMemcpyAsync(&entries, scan.total.ptr, sizeof(long long), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return e;
    if (entries >= INT_MAX) {
        err = "anti-aliasing: too many (pixel, segment) incidences in one call";
        return cudaErrorInvalidValue;
    }
    if (entries == 0) return cudaSuccess;
    if ((e = ids.ensure(size_t(entries))) != cudaSuccess ||
        (e = cudaMemsetAsync(cnt.ptr, 0, sizeof(int) * (size_t(n) + 1), st)) != cudaSuccess)
        return e;
    aa_touch_kernel<<<tg, th, 0, st>>>(G.seg.ptr, G.S, vps.ptr, cnt.ptr, off.ptr, ids.ptr, 1);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const unsigned gp = (unsigned)((n + 1 + th - 1) / th);
    aa_flags_kernel<<<gp, th, 0, st>>>(off.ptr, cnt.ptr, n);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = scan_exclusive(cnt.ptr, cnt.ptr, n + 1, scan, st)) != cudaSuccess) return e;
    long long ne = 0;
    if ((e = cudaMemcpyAsync(&ne, scan.total.ptr, sizeof(long long), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return e;
    n_edge = int(ne);
    if ((e = edge.ensure(size_t(n_edge))) != cudaSuccess || (e = ns.ensure(size_t(n_edge) + 1)) != cudaSuccess ||
        (e = soff.ensure(size_t(n_edge) + 1)) != cudaSuccess ||
        (e = cudaMemsetAsync(ns.ptr, 0, sizeof(int) * (size_t(n_edge) + 1), st)) != cudaSuccess)
        return e;
    aa_compact_kernel<<<gp, th, 0, st>>>(off.ptr, cnt.ptr, n, edge.ptr);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const unsigned ge = (unsigned)((n_edge + th - 1) / th);
    aa_subdiv_kernel<0><<<ge, th, 0, st>>>(edge.ptr, n_edge, vps.ptr, n_vp, off.ptr, ids.ptr, G.seg.ptr, levels,
                                           ns.ptr, nullptr, nullptr, nullptr);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = scan_exclusive(ns.ptr, soff.ptr, (long long)n_edge + 1, scan, st)) != cudaSuccess) return e;
    long long nsamp = 0;
    if ((e = cudaMemcpyAsync(&nsamp, scan.total.ptr, sizeof(long long), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return e;
    if (nsamp >= INT_MAX) {
        err = "anti-aliasing: too many samples in one call; lower aa_levels";
        return cudaErrorInvalidValue;
    }
    n_samples = int(nsamp);
    if ((e = sxy.ensure(2 * size_t(n_samples))) != cudaSuccess || (e = sw.ensure(size_t(n_samples))) != cudaSuccess ||
        (e = u.ensure(3 * size_t(n_samples))) != cudaSuccess)
        return e;
    aa_subdiv_kernel<1><<<ge, th, 0, st>>>(edge.ptr, n_edge, vps.ptr, n_vp, off.ptr, ids.ptr, G.seg.ptr, levels,
                                           nullptr, soff.ptr, sxy.ptr, sw.ptr);
    note_launch();
    return cudaGetLastError();
}

cudaError_t AaWork::finish(void *rgb, int rgb_dtype, unsigned char *rgb8, cudaStream_t st) {
    if (n_edge == 0) return cudaSuccess;
    aa_reduce_kernel<<<(n_edge + 255) / 256, 256, 0, st>>>(edge.ptr, n_edge, soff.ptr, sw.ptr, u.ptr, rgb,
                                                           rgb_dtype, rgb8);
    note_launch();
    return cudaGetLastError();
}

}  // namespace dc
