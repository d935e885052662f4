// The quadtree's clipping of segments into pieces on the device (Sec. 5.1,
// 5.2, App. E.5), level by level: the cells of a level and their split
// decisions stay on the host (a few thousand cells), the pieces (about one
// per segment and level) are cut on the device.  Within a cell the pieces
// are kept in segment order, so a split cell hands each child its pieces in
// that order too (a stable partition by quadrant, ranks from warp ballots),
// and the result is the host build's, piece for piece: the same cuts, the
// same children, the same endpoints by the same IEEE operations (products
// and sums rounded one at a time, no contraction).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <string>
#include <vector>

#include "dc_internal.h"
#include "tree.h"

namespace dc {
namespace {

constexpr int kCutThreads = 256;
constexpr int kChunk = 2048;   // pieces per block: large cells take several blocks

// One block's share of a cell: pieces [p0, p0 + n) of the current arrays,
// in order; the chunks of a cell are consecutive.
struct CellJob {
    double xm, ym;        // the cell's midlines
    int p0, n;
    int split;            // 1: the pieces go to the 4 children, 0: leaf
    int out;              // leaf: first output position of this chunk's kept pieces
    int cstart[4];        // split: first position of this chunk's pieces of each child
};

// The sub-intervals of piece [ta, tb] of segment q cut at the midlines
// (xm, ym), by quadrant: has = bit mask, u[q], v[q] the interval in q.
__device__ __forceinline__ int cut_piece(const double *q, double ta, double tb, double xm, double ym, double u[4],
                                         double v[4]) {
    const double dx = __dsub_rn(q[2], q[0]), dy = __dsub_rn(q[3], q[1]);
    double c[4];
    int nc = 0;
    c[nc++] = ta;
    if (dx != 0.0) {
        const double tx = __ddiv_rn(__dsub_rn(xm, q[0]), dx);
        if (tx > ta && tx < tb) c[nc++] = tx;
    }
    if (dy != 0.0) {
        const double ty = __ddiv_rn(__dsub_rn(ym, q[1]), dy);
        if (ty > ta && ty < tb) c[nc++] = ty;
    }
    c[nc++] = tb;
    for (int i = 1; i < nc; ++i)
        for (int k = i; k > 0 && c[k] < c[k - 1]; --k) {
            const double x = c[k];
            c[k] = c[k - 1];
            c[k - 1] = x;
        }
    int has = 0;
    for (int i = 0; i + 1 < nc; ++i) {
        const double a = c[i], b = c[i + 1];
        if (!(b > a)) continue;
        const double tm = __dmul_rn(0.5, __dadd_rn(a, b));
        const double px = __dadd_rn(q[0], __dmul_rn(tm, dx)), py = __dadd_rn(q[1], __dmul_rn(tm, dy));
        const int qd = (px >= xm ? 1 : 0) + (py >= ym ? 2 : 0);
        has |= 1 << qd;
        u[qd] = a;
        v[qd] = b;
    }
    return has;
}

// Block-wide ranks of up to 4 flags per thread, in thread order, carried
// across batches in base[4]; returns the batch totals in tot[4].
__device__ __forceinline__ void block_ranks(int has, int rank[4], int *base, int tot[4]) {
    __shared__ int wsum[kCutThreads / 32][4];
    __shared__ int wpre[kCutThreads / 32][4];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    unsigned bal[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        bal[q] = __ballot_sync(0xffffffffu, (has >> q) & 1);
        if (lane == 0) wsum[w][q] = __popc(bal[q]);
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        const int q = threadIdx.x;
        int acc = base[q];
        for (int k = 0; k < kCutThreads / 32; ++k) {
            wpre[k][q] = acc;
            acc += wsum[k][q];
        }
        tot[q] = acc - base[q];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) rank[q] = wpre[w][q] + __popc(bal[q] & lt);
}

// pass 0: per split cell the pieces of each child, per leaf the pieces kept
// (longer than 1e-12 in the parameter); pass 1: the pieces written.
template <int PASS>
__global__ void __launch_bounds__(kCutThreads) cut_kernel(const CellJob *__restrict__ jobs,
                                                          const double *__restrict__ seg, const int *__restrict__ ps,
                                                          const double *__restrict__ pa, const double *__restrict__ pb,
                                                          int *__restrict__ counts, int *__restrict__ ns,
                                                          double *__restrict__ na, double *__restrict__ nb,
                                                          int *__restrict__ out_seg, double *__restrict__ out_xy) {
    __shared__ int base[4], tot[4];
    const CellJob J = jobs[blockIdx.x];
    if (threadIdx.x < 4) base[threadIdx.x] = 0;
    __syncthreads();
    for (int b0 = 0; b0 < J.n; b0 += kCutThreads) {
        const int i = b0 + threadIdx.x;
        const bool live = i < J.n;
        int has = 0;
        double u[4] = {0, 0, 0, 0}, v[4] = {0, 0, 0, 0};
        int sg = 0;
        double ta = 0.0, tb = 0.0;
        if (live) {
            sg = ps[J.p0 + i];
            ta = pa[J.p0 + i];
            tb = pb[J.p0 + i];
            if (J.split) has = cut_piece(seg + 4 * (size_t)sg, ta, tb, J.xm, J.ym, u, v);
            else has = (tb - ta > 1e-12) ? 1 : 0;
        }
        int rank[4];
        block_ranks(has, rank, base, tot);
        if (PASS == 1 && live) {
            if (J.split) {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if ((has >> q) & 1) {
                        const int o = J.cstart[q] + rank[q];
                        ns[o] = sg;
                        na[o] = u[q];
                        nb[o] = v[q];
                    }
            } else if (has) {
                const int o = J.out + rank[0];
                const double *q = seg + 4 * (size_t)sg;
                const double dx = __dsub_rn(q[2], q[0]), dy = __dsub_rn(q[3], q[1]);
                out_seg[o] = sg;
                out_xy[4 * (size_t)o + 0] = ta == 0.0 ? q[0] : __dadd_rn(q[0], __dmul_rn(ta, dx));
                out_xy[4 * (size_t)o + 1] = ta == 0.0 ? q[1] : __dadd_rn(q[1], __dmul_rn(ta, dy));
                out_xy[4 * (size_t)o + 2] = tb == 1.0 ? q[2] : __dadd_rn(q[0], __dmul_rn(tb, dx));
                out_xy[4 * (size_t)o + 3] = tb == 1.0 ? q[3] : __dadd_rn(q[1], __dmul_rn(tb, dy));
            }
        }
        __syncthreads();
        if (threadIdx.x < 4) base[threadIdx.x] += tot[threadIdx.x];
        __syncthreads();
    }
    if (PASS == 0 && threadIdx.x < 4) counts[4 * blockIdx.x + threadIdx.x] = base[threadIdx.x];
}

__global__ void init_pieces_kernel(int S, int *__restrict__ ps, double *__restrict__ pa, double *__restrict__ pb) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= S) return;
    ps[k] = k;
    pa[k] = 0.0;
    pb[k] = 1.0;
}

}  // namespace

bool build_quadtree_device(const double *seg_dev, const std::vector<double> &seg_xy, const double domain[4],
                           int leaf_size, int max_depth, Tree &t, void *stream, std::string &err) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    t = Tree();
    const int S = int(seg_xy.size() / 4);
    if (!quadtree_root(seg_xy, domain, t, err)) return false;
    auto cuda_err = [&](cudaError_t e) {
        err = std::string("build_tree (device clipping): ") + cudaGetErrorString(e);
        return false;
    };
    // piece arrays: current and next level, and the leaves' output
    size_t cap = std::max<size_t>(2 * (size_t)S + 64, 1024);
    DevBuf<int> ps[2], out_seg;
    DevBuf<double> pa[2], pb[2], out_xy;
    DevBuf<CellJob> jobs;
    DevBuf<int> counts;
    cudaError_t e;
    for (int k = 0; k < 2; ++k)
        if ((e = ps[k].alloc(cap)) != cudaSuccess || (e = pa[k].alloc(cap)) != cudaSuccess ||
            (e = pb[k].alloc(cap)) != cudaSuccess)
            return cuda_err(e);
    if ((e = out_seg.alloc(cap)) != cudaSuccess || (e = out_xy.alloc(4 * cap)) != cudaSuccess) return cuda_err(e);
    if (S > 0) {
        init_pieces_kernel<<<(S + 255) / 256, 256, 0, st>>>(S, ps[0].ptr, pa[0].ptr, pb[0].ptr);
        note_launch();
    }
    t.level.push_back(0);
    t.parent.push_back(-1);
    t.child0.push_back(-1);
    t.ix.push_back(0);
    t.iy.push_back(0);
    t.level_start.push_back(0);
    std::vector<int> p0 = {0}, pn = {S};   // pieces of the current level's cells
    std::vector<int> leaf_out(1, -1), leaf_cnt(1, 0);
    int cur = 0, lev = 0, first = 0, n_out = 0;
    std::vector<CellJob> hj;
    std::vector<int> hc, job_cell;
    const auto t0 = std::chrono::steady_clock::now();
    while (true) {
        const int n_level = int(p0.size());
        const int next_first = t.n_cells();
        hj.clear();
        job_cell.clear();
        int n_split = 0;
        for (int j = 0; j < n_level; ++j) {
            const int c = first + j;
            CellJob J{};
            J.xm = t.cx(c);
            J.ym = t.cy(c);
            J.split = (pn[j] > leaf_size && lev < max_depth) ? 1 : 0;
            for (int a = 0; a == 0 || a < pn[j]; a += kChunk) {   // one job for an empty cell
                J.p0 = p0[j] + a;
                J.n = std::min(kChunk, pn[j] - a);
                hj.push_back(J);
                job_cell.push_back(j);
            }
            if (J.split) {
                ++n_split;
                t.child0[c] = t.n_cells();
                for (int q = 0; q < 4; ++q) {
                    t.level.push_back(lev + 1);
                    t.parent.push_back(c);
                    t.child0.push_back(-1);
                    t.ix.push_back(2 * t.ix[c] + (q & 1));
                    t.iy.push_back(2 * t.iy[c] + (q >> 1));
                }
            }
        }
        const int n_jobs = int(hj.size());
        // pass 0: counts per child / kept per leaf, per chunk
        if ((e = jobs.ensure(n_jobs)) != cudaSuccess || (e = counts.ensure(4 * (size_t)n_jobs)) != cudaSuccess)
            return cuda_err(e);
        if ((e = cudaMemcpyAsync(jobs.ptr, hj.data(), sizeof(CellJob) * n_jobs, cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
            return cuda_err(e);
        cut_kernel<0><<<n_jobs, kCutThreads, 0, st>>>(jobs.ptr, seg_dev, ps[cur].ptr, pa[cur].ptr, pb[cur].ptr,
                                                      counts.ptr, nullptr, nullptr, nullptr, nullptr, nullptr);
        note_launch();
        hc.resize(4 * (size_t)n_jobs);
        if ((e = cudaGetLastError()) != cudaSuccess ||
            (e = cudaMemcpyAsync(hc.data(), counts.ptr, sizeof(int) * 4 * n_jobs, cudaMemcpyDeviceToHost, st)) !=
                cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return cuda_err(e);
        // children's piece ranges (child cell order), each chunk's place in
        // them, and the leaves' output
        std::vector<int> np0, npn;
        np0.reserve(4 * (size_t)n_split);
        npn.reserve(4 * (size_t)n_split);
        leaf_out.resize(t.n_cells(), -1);
        leaf_cnt.resize(t.n_cells(), 0);
        int nxt_total = 0;
        for (int a = 0; a < n_jobs;) {
            const int j = job_cell[a], c = first + j;
            int b = a;
            while (b < n_jobs && job_cell[b] == j) ++b;   // the cell's chunks [a, b)
            if (hj[a].split) {
                for (int q = 0; q < 4; ++q) {
                    np0.push_back(nxt_total);
                    for (int k = a; k < b; ++k) {
                        hj[k].cstart[q] = nxt_total;
                        nxt_total += hc[4 * k + q];
                    }
                    npn.push_back(nxt_total - np0.back());
                }
            } else {
                leaf_out[c] = n_out;
                for (int k = a; k < b; ++k) {
                    hj[k].out = n_out;
                    n_out += hc[4 * k];
                }
                leaf_cnt[c] = n_out - leaf_out[c];
            }
            a = b;
        }
        const int nxt = 1 - cur;
        auto grow = [&](DevBuf<int> &bi, DevBuf<double> &b1, DevBuf<double> &b2, size_t need) -> cudaError_t {
            if (need <= bi.n) return cudaSuccess;
            cudaError_t r;
            DevBuf<int> ti;
            DevBuf<double> t1, t2;
            if ((r = ti.alloc(2 * need)) != cudaSuccess || (r = t1.alloc(2 * need)) != cudaSuccess ||
                (r = t2.alloc(2 * need)) != cudaSuccess)
                return r;
            std::swap(bi.ptr, ti.ptr);
            std::swap(bi.n, ti.n);
            std::swap(b1.ptr, t1.ptr);
            std::swap(b1.n, t1.n);
            std::swap(b2.ptr, t2.ptr);
            std::swap(b2.n, t2.n);
            return cudaSuccess;
        };
        if ((e = grow(ps[nxt], pa[nxt], pb[nxt], (size_t)nxt_total)) != cudaSuccess) return cuda_err(e);
        if ((size_t)n_out > out_seg.n) {   // keep what is written: copy into larger buffers
            DevBuf<int> os;
            DevBuf<double> ox;
            if ((e = os.alloc(2 * (size_t)n_out)) != cudaSuccess || (e = ox.alloc(8 * (size_t)n_out)) != cudaSuccess ||
                (e = cudaMemcpyAsync(os.ptr, out_seg.ptr, sizeof(int) * out_seg.n, cudaMemcpyDeviceToDevice, st)) !=
                    cudaSuccess ||
                (e = cudaMemcpyAsync(ox.ptr, out_xy.ptr, sizeof(double) * out_xy.n, cudaMemcpyDeviceToDevice, st)) !=
                    cudaSuccess ||
                (e = cudaStreamSynchronize(st)) != cudaSuccess)
                return cuda_err(e);
            std::swap(out_seg.ptr, os.ptr);
            std::swap(out_seg.n, os.n);
            std::swap(out_xy.ptr, ox.ptr);
            std::swap(out_xy.n, ox.n);
        }
        // pass 1: the pieces written
        if ((e = cudaMemcpyAsync(jobs.ptr, hj.data(), sizeof(CellJob) * n_jobs, cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
            return cuda_err(e);
        cut_kernel<1><<<n_jobs, kCutThreads, 0, st>>>(jobs.ptr, seg_dev, ps[cur].ptr, pa[cur].ptr, pb[cur].ptr,
                                                       nullptr, ps[nxt].ptr, pa[nxt].ptr, pb[nxt].ptr, out_seg.ptr,
                                                       out_xy.ptr);
        note_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(e);
        if (n_split == 0) break;
        ++lev;
        t.level_start.push_back(next_first);
        first = next_first;
        p0.swap(np0);
        pn.swap(npn);
        cur = nxt;
    }
    t.depth = lev;
    t.level_start.push_back(t.n_cells());
    const int nC = t.n_cells();
    leaf_out.resize(nC, -1);
    leaf_cnt.resize(nC, 0);
    t.piece_start.assign(nC, 0);
    t.piece_count.assign(nC, 0);
    for (int c = 0; c < nC; ++c)
        if (t.is_leaf(c)) {
            t.piece_start[c] = leaf_out[c];
            t.piece_count[c] = leaf_cnt[c];
        }
    t.pc_seg.resize(n_out);
    t.pc_xy.resize(4 * (size_t)n_out);
    if (n_out > 0 &&
        ((e = cudaMemcpyAsync(t.pc_seg.data(), out_seg.ptr, sizeof(int) * n_out, cudaMemcpyDeviceToHost, st)) !=
             cudaSuccess ||
         (e = cudaMemcpyAsync(t.pc_xy.data(), out_xy.ptr, sizeof(double) * 4 * n_out, cudaMemcpyDeviceToHost, st)) !=
             cudaSuccess))
        return cuda_err(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_err(e);
    const auto t1 = std::chrono::steady_clock::now();
    quadtree_lists(t);
    t.ms_cut = std::chrono::duration<double, std::milli>(t1 - t0).count();
    t.ms_lists = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t1).count();
    return true;
}

}  // namespace dc
