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

// ------------------------------------------------------------ lists --
// Lists 1-4 on the device, entry for entry the host construction's (same
// order within each list: the colleagues, list 2 and list 3 in the order
// their loops produce them, lists 1 and 4 sorted).
constexpr int kMaxColl = 8, kMaxV = 27, kDfsStack = 64;

struct CellsDev {
    const int *level, *parent, *child0;
    const long long *ix, *iy;
};

__device__ __forceinline__ bool touches_dev(const CellsDev &t, int a, int b) {
    if (t.level[a] > t.level[b]) {
        const int x = a;
        a = b;
        b = x;
    }
    const int d = t.level[b] - t.level[a];
    const long long ax0 = t.ix[a] << d, ax1 = (t.ix[a] + 1) << d;
    const long long ay0 = t.iy[a] << d, ay1 = (t.iy[a] + 1) << d;
    const long long bx0 = t.ix[b], bx1 = t.ix[b] + 1, by0 = t.iy[b], by1 = t.iy[b] + 1;
    return bx1 >= ax0 && bx0 <= ax1 && by1 >= ay0 && by0 <= ay1;
}

// colleagues of the cells [c0, c1) of one level (their parents' are known)
__global__ void coll_kernel(CellsDev t, int c0, int c1, int *__restrict__ coll, int *__restrict__ ncoll) {
    const int c = c0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= c1) return;
    const int P = t.parent[c];
    int n = 0;
    auto consider = [&](int Q) {
        if (t.child0[Q] < 0) return;
        for (int q = 0; q < 4; ++q) {
            const int D = t.child0[Q] + q;
            if (D != c && touches_dev(t, c, D) && n < kMaxColl) coll[kMaxColl * c + n++] = D;
        }
    };
    consider(P);
    for (int i = 0; i < ncoll[P]; ++i) consider(coll[kMaxColl * P + i]);
    ncoll[c] = n;
}

// list 2 into fixed slots
__global__ void v_kernel(CellsDev t, int nC, const int *__restrict__ coll, const int *__restrict__ ncoll,
                         int *__restrict__ vtmp, int *__restrict__ vcnt) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nC) return;
    int n = 0;
    if (t.level[c] >= 2) {
        const int P = t.parent[c];
        for (int i = 0; i < ncoll[P]; ++i) {
            const int Q = coll[kMaxColl * P + i];
            if (t.child0[Q] < 0) continue;
            for (int q = 0; q < 4; ++q) {
                const int D = t.child0[Q] + q;
                if (!touches_dev(t, c, D) && n < kMaxV) vtmp[kMaxV * c + n++] = D;
            }
        }
    }
    vcnt[c] = n;
}

__global__ void compact_kernel(const int *__restrict__ tmp, int slots, const int *__restrict__ cnt,
                               const int *__restrict__ ptr, int nC, int *__restrict__ idx) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nC) return;
    for (int i = 0; i < cnt[c]; ++i) idx[ptr[c] + i] = tmp[(size_t)slots * c + i];
}

// lists 1 (without the coarser neighbours) and 3 of each leaf by the host's
// descent through the colleagues; PASS 0 counts, PASS 1 writes
template <int PASS>
__global__ void uw_kernel(CellsDev t, int nC, const int *__restrict__ coll, const int *__restrict__ ncoll,
                          int *__restrict__ ucnt, int *__restrict__ wcnt, const int *__restrict__ uoff,
                          const int *__restrict__ woff, int *__restrict__ uidx, int *__restrict__ widx,
                          int *__restrict__ bad) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nC) return;
    if (t.child0[b] >= 0) {
        if (PASS == 0) ucnt[b] = wcnt[b] = 0;
        return;
    }
    int nu = 0, nw = 0;
    auto put_u = [&](int v) {
        if (PASS == 1) uidx[uoff[b] + nu] = v;
        ++nu;
    };
    auto put_w = [&](int v) {
        if (PASS == 1) widx[woff[b] + nw] = v;
        ++nw;
    };
    put_u(b);
    int stack[kDfsStack];
    int top = 0;
    for (int i = 0; i < ncoll[b]; ++i) stack[top++] = coll[kMaxColl * b + i];
    while (top > 0) {
        const int C = stack[--top];
        if (t.child0[C] < 0) {
            put_u(C);
            continue;
        }
        for (int q = 0; q < 4; ++q) {
            const int D = t.child0[C] + q;
            if (touches_dev(t, b, D)) {
                if (top < kDfsStack) stack[top++] = D;
                else atomicExch(bad, 1);
            } else {
                put_w(D);
            }
        }
    }
    if (PASS == 0) {
        ucnt[b] = nu;
        wcnt[b] = nw;
    }
}

// the coarser adjacent leaves (U[d] gains b) and list 4 (X[d] gains b for d
// in W[b]): PASS 0 counts per d, PASS 1 writes after d's own entries
template <int PASS>
__global__ void dual_kernel(CellsDev t, int nC, const int *__restrict__ uoff, const int *__restrict__ ucnt,
                            const int *__restrict__ uidx, const int *__restrict__ woff, const int *__restrict__ wcnt,
                            const int *__restrict__ widx, int *__restrict__ uadd, int *__restrict__ xcnt,
                            const int *__restrict__ ufptr, int *__restrict__ uslot, int *__restrict__ ufidx,
                            const int *__restrict__ xptr, int *__restrict__ xslot, int *__restrict__ xidx) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nC || t.child0[b] >= 0) return;
    for (int i = 0; i < ucnt[b]; ++i) {
        const int d = uidx[uoff[b] + i];
        if (t.level[d] > t.level[b]) {
            if (PASS == 0) atomicAdd(&uadd[d], 1);
            else ufidx[ufptr[d] + ucnt[d] + atomicAdd(&uslot[d], 1)] = b;
        }
    }
    for (int i = 0; i < wcnt[b]; ++i) {
        const int d = widx[woff[b] + i];
        if (PASS == 0) atomicAdd(&xcnt[d], 1);
        else xidx[xptr[d] + atomicAdd(&xslot[d], 1)] = b;
    }
}

__global__ void ucopy_kernel(int nC, const int *__restrict__ uoff, const int *__restrict__ ucnt,
                             const int *__restrict__ uidx, const int *__restrict__ ufptr, int *__restrict__ ufidx) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nC) return;
    for (int i = 0; i < ucnt[c]; ++i) ufidx[ufptr[c] + i] = uidx[uoff[c] + i];
}

// each list sorted (lists 1 and 4; a few dozen entries each)
__global__ void sort_lists_kernel(int nC, const int *__restrict__ ptr, int *__restrict__ idx) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nC) return;
    int *a = idx + ptr[c];
    const int n = ptr[c + 1] - ptr[c];
    for (int i = 1; i < n; ++i) {
        const int v = a[i];
        int k = i - 1;
        while (k >= 0 && a[k] > v) {
            a[k + 1] = a[k];
            --k;
        }
        a[k + 1] = v;
    }
}

}  // namespace

// Lists 1-4 of t (cells set) on the device; false with err on a failure.
static bool quadtree_lists_device(Tree &t, cudaStream_t st, std::string &err) {
    const int nC = t.n_cells();
    auto fail = [&](cudaError_t e) {
        err = std::string("build_tree (device lists): ") + cudaGetErrorString(e);
        return false;
    };
    DevBuf<int> level, parent, child0, coll, ncoll, vtmp, vcnt, vptr, ucnt, wcnt, uoff, woff, uidx, widx;
    DevBuf<int> uadd, xcnt, ufcnt, ufptr, uslot, ufidx, xptr, xslot, xidx, bad, vidx;
    DevBuf<long long> ix, iy;
    ScanWork sw;
    cudaError_t e;
    auto up = [&](auto &buf, const auto &v) -> cudaError_t {
        cudaError_t r = buf.alloc(std::max<size_t>(v.size(), 1));
        if (r != cudaSuccess) return r;
        return cudaMemcpyAsync(buf.ptr, v.data(), v.size() * sizeof(v[0]), cudaMemcpyHostToDevice, st);
    };
    const size_t n1 = size_t(nC) + 1;
    if ((e = up(level, t.level)) != cudaSuccess || (e = up(parent, t.parent)) != cudaSuccess ||
        (e = up(child0, t.child0)) != cudaSuccess || (e = up(ix, t.ix)) != cudaSuccess ||
        (e = up(iy, t.iy)) != cudaSuccess || (e = coll.alloc(kMaxColl * (size_t)nC)) != cudaSuccess ||
        (e = ncoll.alloc(nC)) != cudaSuccess || (e = vtmp.alloc(kMaxV * (size_t)nC)) != cudaSuccess ||
        (e = vcnt.alloc(n1)) != cudaSuccess || (e = vptr.alloc(n1)) != cudaSuccess ||
        (e = ucnt.alloc(n1)) != cudaSuccess || (e = wcnt.alloc(n1)) != cudaSuccess ||
        (e = uoff.alloc(n1)) != cudaSuccess || (e = woff.alloc(n1)) != cudaSuccess ||
        (e = uadd.alloc(n1)) != cudaSuccess || (e = xcnt.alloc(n1)) != cudaSuccess ||
        (e = ufcnt.alloc(n1)) != cudaSuccess || (e = ufptr.alloc(n1)) != cudaSuccess ||
        (e = uslot.alloc(n1)) != cudaSuccess || (e = xptr.alloc(n1)) != cudaSuccess ||
        (e = xslot.alloc(n1)) != cudaSuccess || (e = bad.alloc(1)) != cudaSuccess)
        return fail(e);
    CellsDev cd{level.ptr, parent.ptr, child0.ptr, ix.ptr, iy.ptr};
    const int th = 128, gC = (nC + th - 1) / th;
    if ((e = cudaMemsetAsync(ncoll.ptr, 0, sizeof(int) * nC, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(bad.ptr, 0, sizeof(int), st)) != cudaSuccess)
        return fail(e);
    for (int l = 1; l <= t.depth; ++l) {   // colleagues, top down
        const int c0 = t.level_start[l], c1 = t.level_start[l + 1];
        if (c1 > c0) {
            coll_kernel<<<(c1 - c0 + th - 1) / th, th, 0, st>>>(cd, c0, c1, coll.ptr, ncoll.ptr);
            note_launch();
        }
    }
    // sizes of every list, one scan each, then the entries
    auto zero_tail = [&](DevBuf<int> &b) { return cudaMemsetAsync(b.ptr + nC, 0, sizeof(int), st); };
    v_kernel<<<gC, th, 0, st>>>(cd, nC, coll.ptr, ncoll.ptr, vtmp.ptr, vcnt.ptr);
    uw_kernel<0><<<gC, th, 0, st>>>(cd, nC, coll.ptr, ncoll.ptr, ucnt.ptr, wcnt.ptr, nullptr, nullptr, nullptr,
                                    nullptr, bad.ptr);
    note_launch(2);
    if ((e = zero_tail(vcnt)) != cudaSuccess || (e = zero_tail(ucnt)) != cudaSuccess ||
        (e = zero_tail(wcnt)) != cudaSuccess || (e = scan_exclusive(vcnt.ptr, vptr.ptr, nC + 1, sw, st)) != cudaSuccess ||
        (e = scan_exclusive(ucnt.ptr, uoff.ptr, nC + 1, sw, st)) != cudaSuccess ||
        (e = scan_exclusive(wcnt.ptr, woff.ptr, nC + 1, sw, st)) != cudaSuccess)
        return fail(e);
    std::vector<int> tot(3);
    if ((e = cudaMemcpyAsync(&tot[0], vptr.ptr + nC, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&tot[1], uoff.ptr + nC, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&tot[2], woff.ptr + nC, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return fail(e);
    if ((e = vidx.alloc(std::max(tot[0], 1))) != cudaSuccess || (e = uidx.alloc(std::max(tot[1], 1))) != cudaSuccess ||
        (e = widx.alloc(std::max(tot[2], 1))) != cudaSuccess)
        return fail(e);
    compact_kernel<<<gC, th, 0, st>>>(vtmp.ptr, kMaxV, vcnt.ptr, vptr.ptr, nC, vidx.ptr);
    uw_kernel<1><<<gC, th, 0, st>>>(cd, nC, coll.ptr, ncoll.ptr, ucnt.ptr, wcnt.ptr, uoff.ptr, woff.ptr, uidx.ptr,
                                    widx.ptr, bad.ptr);
    note_launch(2);
    if ((e = cudaMemsetAsync(uadd.ptr, 0, sizeof(int) * n1, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(xcnt.ptr, 0, sizeof(int) * n1, st)) != cudaSuccess)
        return fail(e);
    dual_kernel<0><<<gC, th, 0, st>>>(cd, nC, uoff.ptr, ucnt.ptr, uidx.ptr, woff.ptr, wcnt.ptr, widx.ptr, uadd.ptr,
                                      xcnt.ptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
    note_launch();
    // list 1 = own entries + coarser neighbours; list 4
    std::vector<int> h_ucnt(n1), h_uadd(n1), h_xcnt(n1);
    if ((e = cudaMemcpyAsync(h_ucnt.data(), ucnt.ptr, sizeof(int) * n1, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(h_uadd.data(), uadd.ptr, sizeof(int) * n1, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(h_xcnt.data(), xcnt.ptr, sizeof(int) * n1, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return fail(e);
    t.u_ptr.assign(n1, 0);
    t.x_ptr.assign(n1, 0);
    for (int c = 0; c < nC; ++c) {
        t.u_ptr[c + 1] = t.u_ptr[c] + h_ucnt[c] + h_uadd[c];
        t.x_ptr[c + 1] = t.x_ptr[c] + h_xcnt[c];
    }
    if ((e = up(ufptr, t.u_ptr)) != cudaSuccess || (e = up(xptr, t.x_ptr)) != cudaSuccess ||
        (e = ufidx.alloc(std::max(t.u_ptr[nC], 1))) != cudaSuccess ||
        (e = xidx.alloc(std::max(t.x_ptr[nC], 1))) != cudaSuccess ||
        (e = cudaMemsetAsync(uslot.ptr, 0, sizeof(int) * n1, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(xslot.ptr, 0, sizeof(int) * n1, st)) != cudaSuccess)
        return fail(e);
    ucopy_kernel<<<gC, th, 0, st>>>(nC, uoff.ptr, ucnt.ptr, uidx.ptr, ufptr.ptr, ufidx.ptr);
    dual_kernel<1><<<gC, th, 0, st>>>(cd, nC, uoff.ptr, ucnt.ptr, uidx.ptr, woff.ptr, wcnt.ptr, widx.ptr, nullptr,
                                      nullptr, ufptr.ptr, uslot.ptr, ufidx.ptr, xptr.ptr, xslot.ptr, xidx.ptr);
    sort_lists_kernel<<<gC, th, 0, st>>>(nC, ufptr.ptr, ufidx.ptr);
    sort_lists_kernel<<<gC, th, 0, st>>>(nC, xptr.ptr, xidx.ptr);
    note_launch(4);
    // back to the host tree
    std::vector<int> hv(n1), hw(n1);
    t.v_idx.resize(tot[0]);
    t.w_idx.resize(tot[2]);
    t.u_idx.resize(t.u_ptr[nC]);
    t.x_idx.resize(t.x_ptr[nC]);
    int hbad = 0;
    if ((e = cudaMemcpyAsync(hv.data(), vptr.ptr, sizeof(int) * n1, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(hw.data(), woff.ptr, sizeof(int) * n1, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (tot[0] && (e = cudaMemcpyAsync(t.v_idx.data(), vidx.ptr, sizeof(int) * tot[0], cudaMemcpyDeviceToHost, st)) !=
                       cudaSuccess) ||
        (tot[2] && (e = cudaMemcpyAsync(t.w_idx.data(), widx.ptr, sizeof(int) * tot[2], cudaMemcpyDeviceToHost, st)) !=
                       cudaSuccess) ||
        (t.u_ptr[nC] && (e = cudaMemcpyAsync(t.u_idx.data(), ufidx.ptr, sizeof(int) * t.u_ptr[nC],
                                             cudaMemcpyDeviceToHost, st)) != cudaSuccess) ||
        (t.x_ptr[nC] && (e = cudaMemcpyAsync(t.x_idx.data(), xidx.ptr, sizeof(int) * t.x_ptr[nC],
                                             cudaMemcpyDeviceToHost, st)) != cudaSuccess) ||
        (e = cudaMemcpyAsync(&hbad, bad.ptr, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return fail(e);
    if (hbad) {
        err = "build_tree (device lists): descent stack exceeded";
        return false;
    }
    t.v_ptr.swap(hv);
    t.w_ptr.swap(hw);
    return true;
}

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
    if (!quadtree_lists_device(t, st, err)) return false;
    t.ms_cut = std::chrono::duration<double, std::milli>(t1 - t0).count();
    t.ms_lists = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t1).count();
    return true;
}

}  // namespace dc
