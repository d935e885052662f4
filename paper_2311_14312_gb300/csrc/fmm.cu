// FMM on the non-uniform quadtree (App. E, Alg. 8) for the combined single
// + double layer potential of Eq. 23 over clipped segments.
//
// Complex-variable form (App. E.1): G(p,q) = -(1/2pi) Re log(q - p) and
// F(p,q) = (1/2pi) Re[n(p) / (q - p)], n = -i w for a segment with unit
// tangent w.  Expansions are kept scaled by the cell width r:
//     Mt_k = int ((p - c)/r)^k sigma dS + (F part)    (outgoing, Eq. 56/60)
//     Lt_l = u_l r^l / l!                              (incoming, Eq. 62)
// so that every translation matrix depends only on the child quadrant (M2M
// Eq. 71, L2L Eq. 73) or on the integer offset of two same-level cells (M2L
// Eq. 69), plus an additive -log(r) Mt_0 term on Lt_0.  Segment moments
// (App. F, Eq. 76-79) use division-free recurrences:
//   P2M  Mt_k = omega l [ sigma S_k/(k+1) - i mu (w/r) S_{k-1} ],
//        S_k = sum_j bh^j ah^(k-j)  (ah, bh = scaled endpoints)
//   P2L  Lt_l = omega l alpha beta [ sigma T_{l-2}/(l(l-1)) + i mu w T_{l-1}/(l r) ],
//        T_m = sum_j alpha^j beta^(m-j), alpha = 1/ah, beta = 1/bh (l >= 2)
// with the log terms of l = 0, 1 written out.  Evaluation (Alg. 8 last loop)
// fuses L2P (Eq. 64), list-3 M2P (Eq. 61) and list-1 P2P (closed forms,
// App. D) per target.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <cmath>
#include <complex>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "evalnodes.cuh"
#include "fmm_impl.h"
#include "passes.cuh"
#include "passes_tc.cuh"
#include "segint.cuh"

namespace dc {

// initial state of the tensor-core M2L's flags: no wait ran out, no tile
// held back by the test hook
static const int kTcErrInit[2] = {0, -1};

namespace {

using cd = std::complex<double>;

// ----------------------------------------------------- complex helpers --
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) {
    return make_double2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ double2 cscale(double2 a, double s) {
    return make_double2(a.x * s, a.y * s);
}
__device__ __forceinline__ double2 cinv(double2 a) {
    double d = 1.0 / (a.x * a.x + a.y * a.y);
    return make_double2(a.x * d, -a.y * d);
}
// principal log
__device__ __forceinline__ double2 clog(double2 a) {
    return make_double2(0.5 * log(a.x * a.x + a.y * a.y), atan2(a.y, a.x));
}
// acc += m * v (complex)
__device__ __forceinline__ void cfma(double2 &acc, double2 m, double2 v) {
    acc.x += m.x * v.x - m.y * v.y;
    acc.y += m.x * v.y + m.y * v.x;
}



// ------------------------------------------------------------- eval ----
struct Acc3 {
    double v[3];
};

__device__ __forceinline__ void eval_point(const DevTree &t, int leaf, double qx, double qy,
                                           int own1, int own2, int P1,
                                           const double2 *__restrict__ M,
                                           const double2 *__restrict__ L,
                                           const double *__restrict__ sbar,
                                           const double *__restrict__ mbar, int use_s, int use_m,
                                           Acc3 &u, long long &pairs) {
    double e0 = 0, e1 = 0, e2 = 0;   // expansion parts, times 2 pi
    // L2P (Eq. 64)
    {
        double w = t.cw[leaf];
        double2 z = make_double2((qx - t.cc[2 * leaf]) / w, (qy - t.cc[2 * leaf + 1]) / w);
        const double2 *Lc = L + (size_t)leaf * 3 * P1;
        double2 s0 = Lc[P1 - 1], s1 = Lc[2 * P1 - 1], s2 = Lc[3 * P1 - 1];
        for (int k = P1 - 2; k >= 0; --k) {
            s0 = cadd(cmul(s0, z), Lc[k]);
            s1 = cadd(cmul(s1, z), Lc[P1 + k]);
            s2 = cadd(cmul(s2, z), Lc[2 * P1 + k]);
        }
        e0 += s0.x;
        e1 += s1.x;
        e2 += s2.x;
    }
    // M2P over list 3 (Eq. 61)
    for (int e = t.w_ptr[leaf]; e < t.w_ptr[leaf + 1]; ++e) {
        int src = t.w_idx[e];
        double w = t.cw[src];
        double zx = qx - t.cc[2 * src], zy = qy - t.cc[2 * src + 1];
        double2 iz = cinv(make_double2(zx / w, zy / w));
        double lz = 0.5 * log(zx * zx + zy * zy);
        const double2 *Ms = M + (size_t)src * 3 * P1;
        double2 s[3];
        for (int c = 0; c < 3; ++c) s[c] = cscale(Ms[c * P1 + P1 - 1], 1.0 / (P1 - 1));
        for (int k = P1 - 2; k >= 1; --k)
            for (int c = 0; c < 3; ++c) s[c] = cadd(cmul(s[c], iz), cscale(Ms[c * P1 + k], 1.0 / k));
        for (int c = 0; c < 3; ++c) s[c] = cmul(s[c], iz);
        e0 += s[0].x - lz * Ms[0].x;
        e1 += s[1].x - lz * Ms[P1].x;
        e2 += s[2].x - lz * Ms[2 * P1].x;
    }
    double u0 = e0 * kInv2Pi, u1 = e1 * kInv2Pi, u2 = e2 * kInv2Pi;
    // P2P over list 1 (App. D closed forms)
    for (int e = t.u_ptr[leaf]; e < t.u_ptr[leaf + 1]; ++e) {
        int src = t.u_idx[e];
        int p0 = t.pstart[src], pn = t.pcount[src];
        pairs += pn;
        for (int i = p0; i < p0 + pn; ++i) {
            const double *q = t.pc + 4 * (size_t)i;
            int seg = t.pseg[i];
            double G, F;
            seg_gf_f64(qx, qy, q[0], q[1], q[2], q[3], t.pw[i], seg == own1 || seg == own2, G, F);
            if (use_s) {
                u0 += G * sbar[3 * (size_t)seg + 0];
                u1 += G * sbar[3 * (size_t)seg + 1];
                u2 += G * sbar[3 * (size_t)seg + 2];
            }
            if (use_m) {
                u0 += F * mbar[3 * (size_t)seg + 0];
                u1 += F * mbar[3 * (size_t)seg + 1];
                u2 += F * mbar[3 * (size_t)seg + 2];
            }
        }
    }
    u.v[0] = u0;
    u.v[1] = u1;
    u.v[2] = u2;
}

// Targets grouped by leaf (nodes or sorted points); result scattered to the
// original order.
__global__ void eval_targets_kernel(DevTree t, const int *__restrict__ leaves,
                                    const int *__restrict__ tstart, const int *__restrict__ tcount,
                                    const double *__restrict__ txy, const int *__restrict__ town1,
                                    const int *__restrict__ town2, const int *__restrict__ tperm,
                                    int P1, const double2 *__restrict__ M,
                                    const double2 *__restrict__ L, const double *__restrict__ sbar,
                                    const double *__restrict__ mbar, int use_s, int use_m,
                                    double *__restrict__ out) {
    int leaf = leaves[blockIdx.x];
    int s0 = tstart[leaf], n = tcount[leaf];
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        int ti = s0 + j;
        Acc3 u;
        long long pairs = 0;
        eval_point(t, leaf, txy[2 * ti], txy[2 * ti + 1], town1 ? town1[ti] : -1,
                   town2 ? town2[ti] : -1, P1, M, L, sbar, mbar, use_s, use_m, u, pairs);
        int o = tperm[ti];
        out[3 * (size_t)o + 0] = u.v[0];
        out[3 * (size_t)o + 1] = u.v[1];
        out[3 * (size_t)o + 2] = u.v[2];
    }
}



__device__ __forceinline__ unsigned char q8(double v) {
    v = fmin(fmax(v, 0.0), 1.0);
    return (unsigned char)floor(255.0 * v + 0.5);
}

__global__ void eval_tiles_kernel(DevTree t, const Tile *__restrict__ tiles, const VpDev *__restrict__ vps, int P1,
                                  const double2 *__restrict__ M, const double2 *__restrict__ L,
                                  const double *__restrict__ sbar, const double *__restrict__ mbar,
                                  void *rgb, int rgb_dtype, unsigned char *rgb8) {
    Tile tl = tiles[blockIdx.x];
    const VpDev vp = vps[tl.vp];
    int npx = tl.nr * tl.nc;
    for (int j = threadIdx.x; j < npx; j += blockDim.x) {
        int r = tl.r0 + j / tl.nc, c = tl.c0 + j % tl.nc;
        double qx = vp.x0 + (c + 0.5) * vp.dx, qy = vp.y0 + (r + 0.5) * vp.dy;
        Acc3 u;
        long long pairs = 0;
        eval_point(t, tl.leaf, qx, qy, -1, -1, P1, M, L, sbar, mbar, 1, 1, u, pairs);
        size_t o = 3 * ((size_t)vp.offset + (size_t)r * vp.width + c);
        for (int ch = 0; ch < 3; ++ch) {
            if (rgb) {
                if (rgb_dtype == DC_F64) static_cast<double *>(rgb)[o + ch] = u.v[ch];
                else static_cast<float *>(rgb)[o + ch] = (float)u.v[ch];
            }
            if (rgb8) rgb8[o + ch] = q8(u.v[ch]);
        }
    }
}

// ------------------------------------------------- host table builders --
double binom(int n, int k) {
    if (k < 0 || k > n) return 0.0;
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

int offset_code(int dx, int dy) { return (dx + 3) * 7 + (dy + 3); }

void build_tables(int p, std::vector<cd> &m2m, std::vector<cd> &l2l, std::vector<cd> &m2l) {
    int P1 = p + 1;
    m2m.assign(4 * P1 * P1, cd(0));
    l2l.assign(4 * P1 * P1, cd(0));
    for (int q = 0; q < 4; ++q) {
        cd d(((q & 1) - 0.5) / 2.0, ((q >> 1) - 0.5) / 2.0);   // child centre - parent centre, / parent width
        // M2M: Mt'_k = sum_{j<=k} C(k,j) d^(k-j) 2^-j Mt_j          (Eq. 71 scaled)
        for (int k = 0; k < P1; ++k)
            for (int j = 0; j <= k; ++j)
                m2m[(q * P1 + k) * P1 + j] = binom(k, j) * std::pow(d, k - j) * std::ldexp(1.0, -j);
        // L2L: Lt_l = sum_{k>=l} C(k,l) 2^-l d^(k-l) Lt'_k           (Eq. 73 scaled)
        for (int l = 0; l < P1; ++l)
            for (int k = l; k < P1; ++k)
                l2l[(q * P1 + l) * P1 + k] = binom(k, l) * std::ldexp(1.0, -l) * std::pow(d, k - l);
    }
    // M2L: Lt_l = sum_k (-1)^l C(l+k,k)/(l+k) D^-(l+k) Mt_k ; [0][0] = -log D (Eq. 69 scaled)
    m2l.assign(49 * P1 * P1, cd(0));
    for (int dx = -3; dx <= 3; ++dx)
        for (int dy = -3; dy <= 3; ++dy) {
            if (std::max(std::abs(dx), std::abs(dy)) < 2) continue;
            cd D(dx, dy), iD = 1.0 / D;
            cd *T = &m2l[size_t(offset_code(dx, dy)) * P1 * P1];
            for (int l = 0; l < P1; ++l)
                for (int k = 0; k < P1; ++k) {
                    if (l + k == 0) {
                        T[0] = -std::log(D);
                        continue;
                    }
                    double sgn = (l & 1) ? -1.0 : 1.0;
                    T[l * P1 + k] = sgn * binom(l + k, k) / double(l + k) * std::pow(iD, l + k);
                }
        }
}

// The 7 base M2L matrices (offsets (2,0) (2,1) (2,2) (3,0) (3,1) (3,2) (3,3)),
// transposed: base[b][k][l] = T_lk(B_b).
void build_base_tables(int p, std::vector<cd> &base) {
    const int P1 = p + 1;
    const int bases[7][2] = {{2, 0}, {2, 1}, {2, 2}, {3, 0}, {3, 1}, {3, 2}, {3, 3}};
    base.assign(7 * P1 * P1, cd(0));
    for (int b = 0; b < 7; ++b) {
        cd D(bases[b][0], bases[b][1]), iD = 1.0 / D;
        for (int l = 0; l < P1; ++l)
            for (int k = 0; k < P1; ++k) {
                cd v;
                if (l + k == 0) v = -std::log(D);
                else v = ((l & 1) ? -1.0 : 1.0) * binom(l + k, k) / double(l + k) * std::pow(iD, l + k);
                base[(size_t)b * P1 * P1 + k * P1 + l] = v;
            }
    }
}

// The tables of an expansion order, built once per process and kept (they
// depend on p alone; entries are never removed, so references stay valid).
struct OrderTables {
    std::vector<cd> m2m, l2l, m2l, base;
};
const OrderTables &order_tables(int p) {
    static std::mutex mu;
    static std::map<int, std::unique_ptr<OrderTables>> cache;
    std::lock_guard<std::mutex> lock(mu);
    std::unique_ptr<OrderTables> &t = cache[p];
    if (!t) {
        std::unique_ptr<OrderTables> n(new OrderTables());
        build_tables(p, n->m2m, n->l2l, n->m2l);
        build_base_tables(p, n->base);
        t = std::move(n);
    }
    return *t;
}

template <typename T>
cudaError_t upload(DevBuf<T> &buf, const std::vector<T> &v, cudaStream_t st) {
    cudaError_t e = buf.alloc(std::max<size_t>(v.size(), 1));
    if (e != cudaSuccess) return e;
    if (v.empty()) return cudaSuccess;
    return cudaMemcpyAsync(buf.ptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st);
}

// Leaf c's list-1 pieces, flattened in list order (block per cell; other
// cells have an empty range): idx = piece numbers, seg = their segments.
__global__ void uf_fill_kernel(const int *__restrict__ u_ptr, const int *__restrict__ u_idx,
                               const int *__restrict__ pstart, const int *__restrict__ pcount,
                               const int *__restrict__ pseg, const int *__restrict__ ufp, int *__restrict__ idx,
                               int *__restrict__ seg) {
    const int c = blockIdx.x;
    int o = ufp[c];
    if (ufp[c + 1] == o) return;
    for (int e = u_ptr[c]; e < u_ptr[c + 1]; ++e) {
        const int src = u_idx[e], p0 = pstart[src], n = pcount[src];
        for (int q = threadIdx.x; q < n; q += blockDim.x) {
            idx[o + q] = p0 + q;
            seg[o + q] = pseg[p0 + q];
        }
        o += n;
    }
}

cudaError_t upload_cd(DevBuf<double2> &buf, const std::vector<cd> &v, cudaStream_t st) {
    std::vector<double2> h(v.size());
    for (size_t i = 0; i < v.size(); ++i) h[i] = make_double2(v[i].real(), v[i].imag());
    return upload(buf, h, st);
}

}  // namespace

// ====================================================================== Impl
DevTree Fmm::Impl::dt() const {
    DevTree t;
    t.cc = cc.ptr;
    t.cw = cw.ptr;
    t.parent = parent.ptr;
    t.child0 = child0.ptr;
    t.quad = quad.ptr;
    t.pstart = pstart.ptr;
    t.pcount = pcount.ptr;
    t.pc = pc.ptr;
    t.pw = pw.ptr;
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
    return t;
}

passes::TreeView<double> Fmm::Impl::view64() const {
    passes::TreeView<double> v;
    v.iw = iw64.ptr;
    v.logw = logw64.ptr;
    v.parent = parent.ptr;
    v.child0 = child0.ptr;
    v.quad = quad.ptr;
    v.pstart = pstart.ptr;
    v.pcount = pcount.ptr;
    v.pw = pw.ptr;
    v.plen = plen64.ptr;
    v.pseg = pseg.ptr;
    v.v_ptr = v_ptr.ptr;
    v.v_idx = v_idx.ptr;
    v.v_code = v_code.ptr;
    v.x_ptr = x_ptr.ptr;
    v.x_idx = x_idx.ptr;
    v.x_off = nullptr;
    return v;
}

// Up and down passes for segment densities (sbar / mbar), FP64.
cudaError_t Fmm::Impl::passes(const double *sb, const double *mb, int use_s, int use_m,
                              cudaStream_t st, const Schedule &sc) {
    const int nC = tree.n_cells();
    size_t ebytes = (size_t)nC * 3 * P1 * sizeof(double2);
    cudaError_t e;
    if ((e = cudaMemsetAsync(M.ptr, 0, ebytes, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(L.ptr, 0, ebytes, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(Lm2l.ptr, 0, ebytes, st)) != cudaSuccess) return e;
    passes::TreeView<double> tv = view64();
    passes::PiecesF64 ps{pc.ptr, cc.ptr};
    if (n_p2m > 0) {
        if (rows_ready)
            passes::p2m_rows_ff_kernel<<<n_p2m, passes::kChunk, 0, st>>>(tv, p2m_leaves.ptr, sb, mb, use_s, use_m, P1,
                                                                       M.ptr, p2m_gff.ptr, p2m_fff.ptr);
        else
            passes::p2m_kernel<double, passes::PiecesF64><<<n_p2m, passes::kChunk, passes::p2m_smem<double>(P1), st>>>(
                tv, ps, p2m_leaves.ptr, sb, mb, use_s, use_m, P1, M.ptr);
        note_launch();
    }
    // per level, in float-float: the chain through the parents does less
    // arithmetic than translating every leaf to every ancestor
    for (int l = tree.depth - 1; l >= 2; --l) {
        const int lo = m2m_ptr[l], n = m2m_ptr[l + 1] - lo;
        if (n <= 0) continue;
        passes::m2m_ff_kernel<<<(n + 3) / 4, 128, passes::mlff_smem(P1), st>>>(child0.ptr, m2m_cells.ptr + lo, n, P1,
                                                                            m2mff.ptr, M.ptr);
        note_launch();
    }
    if (sc.n_m2l > 0) {
        int grid = std::min((sc.n_m2l + passes::kM2LffWarps - 1) / passes::kM2LffWarps, 4 * n_sms);
        passes::m2l_ff_kernel<<<grid, 32 * passes::kM2LffWarps, passes::m2l_ff_smem(P1), st>>>(
            tv, sc.m2l.ptr, sc.n_m2l, P1, baseff.ptr, M.ptr, Lm2l.ptr);
        note_launch();
    }
    if (sc.n_p2l > 0) {
        if (rows_ready)
            passes::p2l_rows_ff_kernel<<<sc.n_p2l, passes::kChunk, 0, st>>>(
                tv, sc.p2l.ptr, p2l_off.ptr, p2l_cnt.ptr, p2l_item.ptr, sb, mb, use_s, use_m, P1, Lm2l.ptr,
                p2l_gff.ptr, p2l_fff.ptr);
        else
            passes::p2l_kernel<double, passes::PiecesF64><<<sc.n_p2l, passes::kChunk, passes::p2l_smem<double>(P1), st>>>(
                tv, ps, sc.p2l.ptr, sb, mb, use_s, use_m, P1, Lm2l.ptr);
        note_launch();
    }
    for (int l = 2; l <= tree.depth; ++l) {   // per level: FP64 work per cell once
        const int lo = sc.l2l_ptr[l], n = sc.l2l_ptr[l + 1] - lo;
        if (n <= 0) continue;
        passes::l2l_ff_kernel<<<(n + 3) / 4, 128, 0, st>>>(tv, sc.l2l.ptr + lo, n, l, P1, l2lff.ptr, Lm2l.ptr, L.ptr);
        note_launch();
    }
    return cudaGetLastError();
}

evalnodes::NodeArgs<double> Fmm::Impl::node_args64(const int4 *items, const double *q64, const int *own1,
                                                    const int *own2, const int *perm, const double *sb,
                                                    const double *mb, int use_s, int use_m,
                                                    double *out) const {
    evalnodes::NodeArgs<double> a;
    a.u_ptr = u_ptr.ptr;
    a.u_idx = u_idx.ptr;
    a.w_ptr = w_ptr.ptr;
    a.w_idx = w_idx.ptr;
    a.pstart = pstart.ptr;
    a.pcount = pcount.ptr;
    a.pseg = pseg.ptr;
    a.pc64 = pc.ptr;
    a.cc64 = cc.ptr;
    a.pw = pw.ptr;
    a.iw = iw64.ptr;
    a.logw = logw64.ptr;
    a.items = items;
    a.q64 = q64;
    a.own1 = own1;
    a.own2 = own2;
    a.perm = perm;
    a.P1 = P1;
    a.M = M.ptr;
    a.L = L.ptr;
    a.sb = sb;
    a.mb = mb;
    a.use_s = use_s;
    a.use_m = use_m;
    a.out = out;
    a.uf_ptr = uf_ptr.ptr;
    a.uf_seg = uf_seg.ptr;
    return a;
}

namespace {
// b[i] = a[i] as (hi, lo) floats
__global__ void d2ff_kernel(const double *__restrict__ a, float2 *__restrict__ b, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v = a[i];
        const float h = (float)v;
        b[i] = make_float2(h, (float)(v - (double)h));
    }
}
}  // namespace

cudaError_t Fmm::Impl::eval_list64(const int4 *items, int n_items, const double *q64,
                                   const int *own1, const int *own2, const int *perm,
                                   const double *sb, const double *mb, int use_s, int use_m,
                                   double *out, cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    evalnodes::NodeArgs<double> a = node_args64(items, q64, own1, own2, perm, sb, mb, use_s, use_m, out);
    evalnodes::eval_nodes_kernel<double><<<n_items, 32 * evalnodes::kWarps, 0, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

cudaError_t Fmm::Impl::apply_nodes(const double *x, double *y, bool single, cudaStream_t st) {
    cudaError_t e = launch_interp(*D, x, single ? sbar.ptr : mbar.ptr, st);
    if (e != cudaSuccess) return e;
    int us = single ? 1 : 0, um = single ? 0 : 1;
    if ((e = passes(sbar.ptr, mbar.ptr, us, um, st, sched_nodes)) != cudaSuccess) return e;
    if (near_ready && far_ready && n_nt_items4 > 0) {   // float-float from stored coefficients
        const long long nS = 3LL * D->S;
        const size_t nE = (size_t)tree.n_cells() * 3 * P1;
        if ((e = dens_ff.ensure((size_t)nS)) != cudaSuccess || (e = Lff.ensure(nE)) != cudaSuccess ||
            (e = Mff.ensure(nE)) != cudaSuccess)
            return e;
        d2ff_kernel<<<4 * n_sms, 256, 0, st>>>(single ? sbar.ptr : mbar.ptr, dens_ff.ptr, nS);
        passes::rows_to_ff_kernel<<<4 * n_sms, 256, 0, st>>>(L.ptr, Lff.ptr, nE);
        passes::rows_to_ff_kernel<<<4 * n_sms, 256, 0, st>>>(M.ptr, Mff.ptr, nE);
        evalnodes::NodeArgs<double> a = node_args64(nt_items4.ptr, nt_xy.ptr, nt_own1.ptr, nt_own2.ptr,
                                                    nt_perm.ptr, sbar.ptr, mbar.ptr, us, um, y);
        evalnodes::near_apply_ff_kernel<<<n_nt_items4, 32 * evalnodes::kWarps, 0, st>>>(
            a, near_off.ptr, single ? near_gff.ptr : near_fff.ptr, dens_ff.ptr, far_off.ptr, farff.ptr, Lff.ptr,
            Mff.ptr);
        note_launch(4);
        return cudaGetLastError();
    }
    if (near_ready && n_nt_items4 > 0) {
        evalnodes::NodeArgs<double> a = node_args64(nt_items4.ptr, nt_xy.ptr, nt_own1.ptr, nt_own2.ptr,
                                                    nt_perm.ptr, sbar.ptr, mbar.ptr, us, um, y);
        evalnodes::near_apply_kernel<double><<<n_nt_items4, 32 * evalnodes::kWarps, 0, st>>>(
            a, near_off.ptr, single ? near_g64.ptr : near_f64.ptr, single ? sbar.ptr : mbar.ptr,
            far_ready ? far_off.ptr : nullptr, far_ready ? far64.ptr : nullptr);
        note_launch();
        return cudaGetLastError();
    }
    return eval_list64(nt_items4.ptr, n_nt_items4, nt_xy.ptr, nt_own1.ptr, nt_own2.ptr, nt_perm.ptr,
                       sbar.ptr, mbar.ptr, us, um, y, st);
}

namespace {
__global__ void narrow_real_kernel(const double *__restrict__ a, float *__restrict__ b, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}
}  // namespace

namespace {
// dst[r][k] = (float2) src[r][k] for k < P1d (the low orders of each row)
__global__ void narrow_rows_kernel(const double2 *__restrict__ src, int P1s, float2 *__restrict__ dst, int P1d,
                                   long long nrows) {
    const long long n = nrows * P1d;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / P1d;
        const int k = int(i - r * P1d);
        const double2 v = src[r * P1s + k];
        dst[i] = make_float2((float)v.x, (float)v.y);
    }
}
}  // namespace

// The near-field coefficients of the node operator, once per drawing, when
// they fit comfortably in device memory (else the near field is evaluated
// from the geometry at every application).
cudaError_t Fmm::Impl::build_near(cudaStream_t st) {
    near_ready = false;
    if (near_total <= 0 || n_nt_items4 == 0) return cudaSuccess;
    const size_t need = (size_t)near_total * (2 * sizeof(double) + (fp32 ? sizeof(float) : 0));
    size_t fr = 0, tot = 0;
    cudaError_t e = cudaMemGetInfo(&fr, &tot);
    if (e != cudaSuccess) return e;
    if (need > fr / 4) return cudaSuccess;
    if ((e = near_g64.alloc((size_t)near_total)) != cudaSuccess) return e;
    if ((e = near_f64.alloc((size_t)near_total)) != cudaSuccess) return e;
    evalnodes::NodeArgs<double> a = node_args64(nt_items4.ptr, nt_xy.ptr, nt_own1.ptr, nt_own2.ptr,
                                                nt_perm.ptr, nullptr, nullptr, 0, 0, nullptr);
    evalnodes::near_coef_kernel<<<n_nt_items4, 32 * evalnodes::kWarps, 0, st>>>(a, near_off.ptr,
                                                                               near_g64.ptr, near_f64.ptr);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (fp32) {
        if ((e = near_g32.alloc((size_t)near_total)) != cudaSuccess) return e;
        narrow_real_kernel<<<4 * n_sms, 256, 0, st>>>(near_g64.ptr, near_g32.ptr, near_total);
        note_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    near_ready = true;
    // far-field coefficients (L2P and list-3 M2P at the nodes), when they fit too
    const size_t need_far = (size_t)far_blocks * (P1 * sizeof(double2) + (fp32 ? P1i * sizeof(float2) : 0));
    if ((e = cudaMemGetInfo(&fr, &tot)) != cudaSuccess) return e;
    if (far_blocks <= 0 || need_far > fr / 4) return cudaSuccess;
    if ((e = far64.alloc((size_t)far_blocks * P1)) != cudaSuccess) return e;
    far_coef_launch(st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (fp32) {
        if ((e = far32.alloc((size_t)far_blocks * P1i)) != cudaSuccess) return e;
        narrow_rows_kernel<<<4 * n_sms, 256, 0, st>>>(far64.ptr, P1, far32.ptr, P1i, far_blocks);
        note_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    far_ready = true;
    // the FP64 node operator reads both in float-float (same sizes)
    if ((e = near_gff.alloc((size_t)near_total)) != cudaSuccess ||
        (e = near_fff.alloc((size_t)near_total)) != cudaSuccess ||
        (e = farff.alloc((size_t)far_blocks * P1)) != cudaSuccess)
        return e;
    d2ff_kernel<<<4 * n_sms, 256, 0, st>>>(near_g64.ptr, near_gff.ptr, near_total);
    d2ff_kernel<<<4 * n_sms, 256, 0, st>>>(near_f64.ptr, near_fff.ptr, near_total);
    passes::rows_to_ff_kernel<<<4 * n_sms, 256, 0, st>>>(far64.ptr, farff.ptr, (size_t)far_blocks * P1);
    note_launch(3);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    near_g64.release();
    near_f64.release();
    far64.release();
    return cudaSuccess;
}

void Fmm::Impl::far_coef_launch(cudaStream_t st) {
    evalnodes::NodeArgs<double> a = node_args64(nt_items4.ptr, nt_xy.ptr, nt_own1.ptr, nt_own2.ptr,
                                                nt_perm.ptr, nullptr, nullptr, 0, 0, nullptr);
    evalnodes::far_coef_kernel<<<n_nt_items4, 32 * evalnodes::kWarps, 0, st>>>(a, far_off.ptr, far64.ptr);
    note_launch();
}


// Per-piece P2M and per-(cell, list-4 piece) P2L coefficients, formed once per
// drawing in FP64 (and the P2M rows' low orders in FP32 for the inner
// operator) and kept resident: the passes then stream them instead of
// re-running the recurrences and logarithms (FP64 at 1/64 of the FP32 rate)
// at every operator application.  The FP32 P2L recomputes: its rows would
// cost more memory traffic than the arithmetic they save.  Skipped when the
// rows would take more than a quarter of the free device memory.
cudaError_t Fmm::Impl::build_rows(cudaStream_t st) {
    rows_ready = false;
    const long long np = (long long)tree.pc_seg.size();
    if (np == 0) return cudaSuccess;
    const size_t per64 = 2 * sizeof(double2) * (size_t)P1, per32 = fp32 ? sizeof(float2) * (size_t)P1i : 0;
    const size_t need = (size_t)(np + p2l_rows) * per64 + (size_t)np * per32;
    size_t fr = 0, tot = 0;
    cudaError_t e = cudaMemGetInfo(&fr, &tot);
    if (e != cudaSuccess) return e;
    if (need > fr / 4) return cudaSuccess;
    if ((e = p2m_g64.alloc((size_t)np * P1)) != cudaSuccess || (e = p2m_f64.alloc((size_t)np * P1)) != cudaSuccess)
        return e;
    if (p2l_rows > 0 && ((e = p2l_g64.alloc((size_t)p2l_rows * P1)) != cudaSuccess ||
                         (e = p2l_f64.alloc((size_t)p2l_rows * P1)) != cudaSuccess))
        return e;
    passes::TreeView<double> tv = view64();
    passes::PiecesF64 ps{pc.ptr, cc.ptr};
    if (n_p2m > 0) {
        passes::p2m_kernel<double, passes::PiecesF64><<<n_p2m, passes::kChunk, passes::p2m_smem<double>(P1), st>>>(
            tv, ps, p2m_leaves.ptr, nullptr, nullptr, 0, 0, P1, M.ptr, nullptr, nullptr, p2m_g64.ptr,
            p2m_f64.ptr);
        note_launch();
    }
    if (sched_all.n_p2l > 0 && p2l_rows > 0) {
        passes::p2l_kernel<double, passes::PiecesF64><<<sched_all.n_p2l, passes::kChunk, passes::p2l_smem<double>(P1), st>>>(
            tv, ps, sched_all.p2l.ptr, nullptr, nullptr, 0, 0, P1, Lm2l.ptr, p2l_off.ptr, nullptr, nullptr,
            p2l_g64.ptr, p2l_f64.ptr);
        note_launch();
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (fp32) {
        if ((e = p2m_g32.alloc((size_t)np * P1i)) != cudaSuccess) return e;
        narrow_rows_kernel<<<4 * n_sms, 256, 0, st>>>(p2m_g64.ptr, P1, p2m_g32.ptr, P1i, np);
        note_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // the FP64 passes read the rows as float-float (same size)
    auto to_ff = [&](DevBuf<double2> &src, DevBuf<float4> &dst) -> cudaError_t {
        cudaError_t r = dst.alloc(src.n);
        if (r != cudaSuccess || src.n == 0) return r;
        passes::rows_to_ff_kernel<<<4 * n_sms, 256, 0, st>>>(src.ptr, dst.ptr, src.n);
        note_launch();
        src.release();   // a device-wide wait in cudaFree, or held back
        return cudaGetLastError();
    };
    if ((e = to_ff(p2m_g64, p2m_gff)) != cudaSuccess || (e = to_ff(p2m_f64, p2m_fff)) != cudaSuccess ||
        (e = to_ff(p2l_g64, p2l_gff)) != cudaSuccess || (e = to_ff(p2l_f64, p2l_fff)) != cudaSuccess)
        return e;
    rows_ready = true;
    return cudaSuccess;
}

Fmm::Fmm() : impl_(new Impl()) {}
Fmm::~Fmm() = default;

dc_status Fmm::build(const dc_options &opt, const Geometry &G, const DevGeom &D, cudaStream_t st,
                     std::string &err) {
    Impl &I = *impl_;
    I.opt = opt;
    I.p = opt.p;
    I.P1 = opt.p + 1;
    I.D = &D;
    if (opt.form != DC_FORM_FMM64 && opt.form != DC_FORM_FMM32) {
        err = "FMM build called for a non-FMM form";
        return DC_ERR_ARG;
    }
    I.fp32 = (opt.form == DC_FORM_FMM32);
    auto t_prev = std::chrono::steady_clock::now();
    auto phase = [&](int i) {   // wall time of build phase i (the stream drained first)
        cudaStreamSynchronize(st);
        const auto t = std::chrono::steady_clock::now();
        I.build_ms[i] = std::chrono::duration<double, std::milli>(t - t_prev).count();
        t_prev = t;
    };
    // Both preconditioner levels depend on the discretisation alone: a host
    // thread plans the coarse level during the tree build; once the tree is
    // built a second one enqueues the device work of both levels on a stream
    // of their own, which runs beside the rest of the tree phase and the
    // schedules here (not beside the tree build, whose short kernels the
    // host waits for one by one); the build waits for it before the stored
    // coefficients.  Meanwhile frees of device memory on this thread are
    // deferred (cudaFree would wait for that stream too).  On an early
    // return the guard joins the threads and drains the stream.
    FreeDefer defer;
    // written by the helper threads: declared before their guard, which
    // joins them before these go out of scope
    cudaError_t pre_err = cudaSuccess;
    bool pre_oom = false;
    Impl::Prep32 prep;
    bool prep_failed = false;
    struct Overlap {
        // the coarse plan, the preconditioner's launches, the FP32 form's host arrays
        std::thread th_plan, th, th32;
        cudaStream_t drain = nullptr;
        ~Overlap() {
            if (th_plan.joinable()) th_plan.join();
            if (th.joinable()) th.join();
            if (th32.joinable()) th32.join();
            if (drain) cudaStreamSynchronize(drain);
        }
    } ov;
    {
        // the preconditioner's stream at the lowest priority and the tree's
        // at the highest: the tree build's short kernels, each waited for by
        // the host, are not queued behind the preconditioner's blocks
        cudaError_t e;
        int prio_lo = 0, prio_hi = 0;
        cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
        if (!I.pre_stream &&
            (e = cudaStreamCreateWithPriority(&I.pre_stream, cudaStreamNonBlocking, prio_lo)) != cudaSuccess) {
            err = std::string("fmm stream: ") + cudaGetErrorString(e);
            return DC_ERR_CUDA;
        }
        if (!I.tree_stream &&
            (e = cudaStreamCreateWithPriority(&I.tree_stream, cudaStreamNonBlocking, prio_hi)) != cudaSuccess) {
            err = std::string("fmm stream: ") + cudaGetErrorString(e);
            return DC_ERR_CUDA;
        }
        if (!I.pre_ev && (e = cudaEventCreateWithFlags(&I.pre_ev, cudaEventDisableTiming)) != cudaSuccess) {
            err = std::string("fmm event: ") + cudaGetErrorString(e);
            return DC_ERR_CUDA;
        }
        // the discretisation's device copy is complete on st before the
        // preconditioner's stream reads it
        if ((e = cudaEventRecord(I.pre_ev, st)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(I.pre_stream, I.pre_ev, 0)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(I.tree_stream, I.pre_ev, 0)) != cudaSuccess) {
            err = std::string("fmm event: ") + cudaGetErrorString(e);
            return DC_ERR_CUDA;
        }
        auto plan = [&I, &G, &opt, &pre_oom] {   // host work only
            try {
                if (!I.render_only) I.coarse.plan(G, opt.coarse_max);
            } catch (...) {
                pre_oom = true;
            }
        };
        try {
            ov.th_plan = std::thread(plan);
        } catch (...) {
            plan();
        }
    }
    if (!build_quadtree_device(D.seg.ptr, G.seg_xy, opt.domain, opt.leaf_size, opt.max_depth, I.tree,
                               I.tree_stream, err))
        return DC_ERR_GEOMETRY;
    {   // later work on st follows the tree's; the preconditioner's device work starts
        cudaError_t e;
        if ((e = cudaEventRecord(I.pre_ev, I.tree_stream)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(st, I.pre_ev, 0)) != cudaSuccess) {
            err = std::string("fmm event: ") + cudaGetErrorString(e);
            return DC_ERR_CUDA;
        }
        if (ov.th_plan.joinable()) ov.th_plan.join();
        int dev = 0;
        cudaGetDevice(&dev);
        DevPool *pool = current_pool();
        auto pre = [&I, &D, &pre_err, &pre_oom, dev, pool] {
            try {
                PoolScope ps(pool);
                cudaError_t r = cudaSetDevice(dev);
                if (r == cudaSuccess && !I.render_only && !pre_oom) r = I.coarse.launch(D, I.pre_stream);
                if (r == cudaSuccess) r = I.pinv.alloc((size_t)D.n_panels * D.g * D.g);
                if (r == cudaSuccess) r = I.pinfo.alloc((size_t)D.n_panels);
                if (r == cudaSuccess) r = launch_panel_block_inverse(D, I.pinv.ptr, I.pinfo.ptr, I.pre_stream);
                pre_err = r;
            } catch (...) {
                pre_oom = true;
            }
        };
        ov.drain = I.pre_stream;
        try {
            ov.th = std::thread(pre);
        } catch (...) {
            pre();   // no thread: enqueue from here
        }
    }
    if (I.P1 > 32) {
        err = "FMM forms support expansion orders p <= 31";
        return DC_ERR_UNSUPPORTED;
    }
    Tree &T = I.tree;
    const int nC = T.n_cells();
    // pieces below each cell; list entries whose source holds none are
    // dropped (their expansions vanish)
    std::vector<int> sub_pieces(nC, 0);
    for (int c = nC - 1; c >= 0; --c) {
        if (T.is_leaf(c)) sub_pieces[c] = T.piece_count[c];
        else
            for (int q = 0; q < 4; ++q) sub_pieces[c] += sub_pieces[T.child0[c] + q];
    }
    auto prune = [&](std::vector<int> &ptr, std::vector<int> &idx) {
        std::vector<int> np(ptr.size(), 0), ni;
        ni.reserve(idx.size());
        for (int c = 0; c + 1 < (int)ptr.size(); ++c) {
            for (int e = ptr[c]; e < ptr[c + 1]; ++e)
                if (sub_pieces[idx[e]] > 0) ni.push_back(idx[e]);
            np[c + 1] = int(ni.size());
        }
        ptr.swap(np);
        idx.swap(ni);
    };
    // Host work of the tree phase on three threads: the lists are pruned on
    // one, the multi-level M2M chunks (which read no list) are built on
    // another, while the cell and piece tables and the node order are
    // built here.  Each guard joins its thread before the variables it
    // uses go out of scope (on an early return too).
    struct Joiner {
        std::thread th;
        ~Joiner() {
            if (th.joinable()) th.join();
        }
        void run(std::function<void()> f) {
            try {
                th = std::thread(f);
            } catch (...) {
                f();   // no thread: run here
            }
        }
        void join() {
            if (th.joinable()) th.join();
        }
    };
    std::atomic<bool> helper_oom(false);
    auto guarded = [&helper_oom](auto f) {
        return [f, &helper_oom] {
            try {
                f();
            } catch (...) {
                helper_oom = true;
            }
        };
    };
    Joiner j_prune;
    j_prune.run(guarded([&] {
        prune(T.u_ptr, T.u_idx);
        prune(T.v_ptr, T.v_idx);
        prune(T.w_ptr, T.w_idx);
        prune(T.x_ptr, T.x_idx);
    }));
    // pass schedules: inner cells of level >= 2 with pieces, by level; the
    // leaf -> ancestor M2M pairs of every inner cell, chunked for the
    // one-launch upward pass (cells with several chunks get partial slots)
    std::vector<int> m2m_cells;
    std::vector<int4> mchunks, mred;
    std::vector<int> pair_leaf;
    std::vector<float4> pair_geo;
    int n_slots = 0;
    Joiner j_mchunks;
    j_mchunks.run(guarded([&] {
        I.m2m_ptr.assign(T.depth + 2, 0);
        for (int l = 0; l <= T.depth; ++l) {
            I.m2m_ptr[l] = int(m2m_cells.size());
            if (l >= 2)
                for (int c = T.level_start[l]; c < T.level_start[l + 1]; ++c)
                    if (!T.is_leaf(c) && sub_pieces[c] > 0) m2m_cells.push_back(c);
        }
        I.m2m_ptr[T.depth + 1] = int(m2m_cells.size());
        std::vector<int> stack, lv;
        for (int a : m2m_cells) {
            lv.clear();
            stack.assign(1, a);
            while (!stack.empty()) {
                const int c = stack.back();
                stack.pop_back();
                if (T.is_leaf(c)) {
                    if (T.piece_count[c] > 0) lv.push_back(c);
                } else {
                    for (int q = 3; q >= 0; --q)
                        if (sub_pieces[T.child0[c] + q] > 0) stack.push_back(T.child0[c] + q);
                }
            }
            const int beg = int(pair_leaf.size());
            pair_leaf.insert(pair_leaf.end(), lv.begin(), lv.end());
            const double wa = T.width(a), ax = T.cx(a), ay = T.cy(a);
            for (int lf : lv)
                pair_geo.push_back(make_float4((float)((T.cx(lf) - ax) / wa), (float)((T.cy(lf) - ay) / wa),
                                               (float)(T.width(lf) / wa), 0.f));
            const int nch = (int(lv.size()) + passes::kMultiLeaves - 1) / passes::kMultiLeaves;
            if (nch == 1) {
                mchunks.push_back(make_int4(a, beg, int(lv.size()), -1));
            } else if (nch > 1) {
                mred.push_back(make_int4(a, n_slots, nch, 0));
                for (int q = 0; q < nch; ++q) {
                    const int b = beg + q * passes::kMultiLeaves;
                    const int cnt = std::min(passes::kMultiLeaves, beg + int(lv.size()) - b);
                    mchunks.push_back(make_int4(a, b, cnt, n_slots++));
                }
            }
        }
    }));
    std::vector<double> cc(2 * nC), cw(nC), iw64(nC), logw64(nC);
    std::vector<int> quad(nC, 0);
    for (int c = 0; c < nC; ++c) {
        cc[2 * c] = T.cx(c);
        cc[2 * c + 1] = T.cy(c);
        cw[c] = T.width(c);
        iw64[c] = 1.0 / cw[c];
        logw64[c] = std::log(cw[c]);
        if (T.parent[c] >= 0) quad[c] = c - T.child0[T.parent[c]];
    }
    std::vector<double> pw(T.pc_seg.size()), plen64(T.pc_seg.size());
    for (size_t i = 0; i < pw.size(); ++i) {
        pw[i] = G.seg_w[T.pc_seg[i]];
        const double *q = &T.pc_xy[4 * i];
        plen64[i] = std::hypot(q[2] - q[0], q[3] - q[1]);
    }
    // list-2 entries: M2L symmetry code (base matrix, rotation, conjugation)
    const int bases[7][2] = {{2, 0}, {2, 1}, {2, 2}, {3, 0}, {3, 1}, {3, 2}, {3, 3}};
    auto sym_code = [&](int dx, int dy) {
        for (int b = 0; b < 7; ++b)
            for (int cj = 0; cj < 2; ++cj)
                for (int r = 0; r < 4; ++r) {
                    int x = bases[b][0], y = cj ? -bases[b][1] : bases[b][1];
                    for (int k = 0; k < r; ++k) {   // times i
                        int t = x;
                        x = -y;
                        y = t;
                    }
                    if (x == dx && y == dy) return b | (r << 3) | (cj << 5);
                }
        return -1;
    };
    int sym_tab[7][7];   // the codes of the offsets in [-3, 3]^2, looked up per entry
    for (int dx = -3; dx <= 3; ++dx)
        for (int dy = -3; dy <= 3; ++dy) sym_tab[dx + 3][dy + 3] = sym_code(dx, dy);
    std::vector<int> p2m;
    for (int c = 0; c < nC; ++c)
        if (T.is_leaf(c) && T.piece_count[c] > 0) p2m.push_back(c);
    I.n_p2m = int(p2m.size());
    // node targets sorted by leaf
    const int N = G.n_nodes();
    std::vector<int> leaf_of(N), cnt(nC, 0);
    // Tree::locate with the cell centres read from cc (the same values)
    auto locate = [&](double x, double y) {
        if (!(x >= T.x0 && x < T.x0 + T.w0 && y >= T.y0 && y < T.y0 + T.w0)) return -1;
        int c = 0;
        while (T.child0[c] >= 0) c = T.child0[c] + (x >= cc[2 * c] ? 1 : 0) + (y >= cc[2 * c + 1] ? 2 : 0);
        return c;
    };
    for (int i = 0; i < N; ++i) {
        int lf = locate(G.node_xy[2 * i], G.node_xy[2 * i + 1]);
        if (lf < 0) {
            err = "internal error: node outside the quadtree root";
            return DC_ERR_GEOMETRY;
        }
        leaf_of[i] = lf;
        cnt[lf]++;
    }
    j_prune.join();
    if (helper_oom) {
        err = "fmm build: host allocation failed";
        return DC_ERR_OOM;
    }
    std::vector<int> voff(T.v_idx.size()), vcode(T.v_idx.size());
    long long m2l_cnt = 0;
    for (int c = 0; c < nC; ++c)
        for (int e = T.v_ptr[c]; e < T.v_ptr[c + 1]; ++e) {
            int s = T.v_idx[e];
            int dx = int(T.ix[c] - T.ix[s]), dy = int(T.iy[c] - T.iy[s]);
            int code = (std::abs(dx) <= 3 && std::abs(dy) <= 3) ? sym_tab[dx + 3][dy + 3] : -1;
            if (std::abs(dx) > 3 || std::abs(dy) > 3 || code < 0) {
                err = "internal error: interaction-list offset out of range";
                return DC_ERR_GEOMETRY;
            }
            voff[e] = offset_code(dx, dy);
            vcode[e] = code;
            ++m2l_cnt;
        }
    I.m2l_cnt = m2l_cnt;
    std::vector<int> sub_nodes(cnt);
    for (int c = nC - 1; c >= 0; --c)
        if (!T.is_leaf(c))
            for (int q = 0; q < 4; ++q) sub_nodes[c] += sub_nodes[T.child0[c] + q];
    j_mchunks.join();
    if (helper_oom) {
        err = "fmm build: host allocation failed";
        return DC_ERR_OOM;
    }
    I.n_mchunks = int(mchunks.size());
    I.n_mred = int(mred.size());
    I.n_mslots = n_slots;
    std::vector<float> binom32(32 * 32, 0.f);
    for (int k = 0; k < 32; ++k)
        for (int j = 0; j <= k; ++j) binom32[k * 32 + j] = (float)binom(k, j);
    auto make_sched = [&](Schedule &sc, bool nodes_only, std::vector<int> &m2l_c,
                          std::vector<int> &p2l_c, std::vector<int> &l2l_c, std::vector<int> &walk_c) {
        sc.l2l_ptr.assign(T.depth + 2, 0);
        for (int l = 0; l <= T.depth; ++l) {
            sc.l2l_ptr[l] = int(l2l_c.size());
            if (l < 2) continue;
            for (int c = T.level_start[l]; c < T.level_start[l + 1]; ++c) {
                if (nodes_only && sub_nodes[c] == 0) continue;
                l2l_c.push_back(c);
                if (T.v_ptr[c + 1] > T.v_ptr[c]) m2l_c.push_back(c);
                if (T.x_ptr[c + 1] > T.x_ptr[c]) p2l_c.push_back(c);
                if (T.is_leaf(c)) walk_c.push_back(c);
            }
        }
        sc.l2l_ptr[T.depth + 1] = int(l2l_c.size());
        sc.n_m2l = int(m2l_c.size());
        sc.n_p2l = int(p2l_c.size());
        sc.n_walk = int(walk_c.size());
    };
    std::vector<int> am2l, ap2l, al2l, aw, nm2l, np2l, nl2l, nw;
    phase(0);   // quadtree, lists, tables, multi-level M2M chunks
    // the FP32 form's host arrays (tree and discretisation only) on a helper
    // thread while the schedules, preconditioner and coefficients are built
    if (I.fp32) {
        auto run = [&T, &G, &prep, &prep_failed] {
            try {
                Impl::prep32(T, G, prep);
            } catch (...) {
                prep_failed = true;
            }
        };
        try {
            ov.th32 = std::thread(run);
        } catch (...) {
            run();
        }
    }
    make_sched(I.sched_all, false, am2l, ap2l, al2l, aw);
    make_sched(I.sched_nodes, true, nm2l, np2l, nl2l, nw);
    // rows of the stored P2L coefficients: the pieces of each list-4 cell of
    // the full schedule (the node schedule's cells are among them)
    std::vector<long long> p2l_off(nC, -1);
    std::vector<int> p2l_cnt(nC, 0);
    std::vector<int2> p2l_item;   // (piece, list-4 entry) per row
    long long p2l_rows = 0;
    Joiner j_p2l;   // on a helper thread while the node items and tables are built
    j_p2l.run(guarded([&] {
        for (int c : ap2l) {
            p2l_off[c] = p2l_rows;
            for (int e = T.x_ptr[c]; e < T.x_ptr[c + 1]; ++e) {
                const int src = T.x_idx[e];
                for (int k = 0; k < T.piece_count[src]; ++k)
                    p2l_item.push_back(make_int2(T.piece_start[src] + k, e));
                p2l_rows += T.piece_count[src];
            }
            p2l_cnt[c] = int(p2l_rows - p2l_off[c]);
        }
    }));
    {
        cudaDeviceProp prop;
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess)
            I.n_sms = prop.multiProcessorCount;
    }
    std::vector<int> start(nC, 0), perm(N), own1(N), own2(N), leaves;
    std::vector<double> txy(2 * N);
    for (int c = 0, acc = 0; c < nC; ++c) {
        start[c] = acc;
        acc += cnt[c];
        if (cnt[c] > 0) leaves.push_back(c);
    }
    std::vector<int> fill(start);
    long long p2p = 0;
    for (int i = 0; i < N; ++i) {
        int j = fill[leaf_of[i]]++;
        perm[j] = i;
        txy[2 * j] = G.node_xy[2 * i];
        txy[2 * j + 1] = G.node_xy[2 * i + 1];
        own1[j] = G.node_seg[i];
        own2[j] = G.node_seg2[i];
        int lf = leaf_of[i];
        for (int e = T.u_ptr[lf]; e < T.u_ptr[lf + 1]; ++e) p2p += T.piece_count[T.u_idx[e]];
    }
    I.p2p_nodes = p2p;
    I.n_nt_leaves = int(leaves.size());
    std::vector<int4> items4;
    std::vector<long long> near_off;   // first near-field coefficient of each item
    long long near_total = 0;
    std::vector<long long> far_off;    // first far-field block of each item
    long long far_blocks = 0;
    for (int c : leaves) {
        int nU = 0;
        for (int e = T.u_ptr[c]; e < T.u_ptr[c + 1]; ++e) nU += T.piece_count[T.u_idx[e]];
        for (int j = 0; j < cnt[c]; j += evalnodes::kNodeItem) {
            const int nt = std::min(evalnodes::kNodeItem, cnt[c] - j);
            items4.push_back(make_int4(c, start[c] + j, nt, nU));
            near_off.push_back(near_total);
            near_total += (long long)nt * nU;
            far_off.push_back(far_blocks);
            far_blocks += (long long)nt * (1 + T.w_ptr[c + 1] - T.w_ptr[c]);
        }
    }
    I.n_nt_items4 = int(items4.size());
    I.near_total = near_total;
    I.far_blocks = far_blocks;
    const OrderTables &tab = order_tables(I.p);
    const std::vector<cd> &m2m = tab.m2m, &l2l = tab.l2l, &m2l = tab.m2l, &base = tab.base;
    const int p_inner = opt.p_inner > 0 ? std::min(opt.p_inner, I.p) : std::min(I.p, 12);
    I.P1i = p_inner + 1;
    const OrderTables &tabi = order_tables(p_inner);
    const std::vector<cd> &m2mi = tabi.m2m, &l2li = tabi.l2l, &basei = tabi.base;
    // the 56 (base, rotation, conjugation) variants in full for the
    // low-order M2L: F[b + 7 r + 28 cj][l][k] = conj^cj(B_b[k][l]) i^(-r (k + l))
    std::vector<cd> fulli(56 * (size_t)I.P1i * I.P1i);
    {
        const int Q = I.P1i;
        const cd ipow[4] = {cd(1, 0), cd(0, -1), cd(-1, 0), cd(0, 1)};   // i^(-n)
        for (int b = 0; b < 7; ++b)
            for (int r = 0; r < 4; ++r)
                for (int cj = 0; cj < 2; ++cj)
                    for (int l = 0; l < Q; ++l)
                        for (int k = 0; k < Q; ++k) {
                            cd v = basei[(size_t)b * Q * Q + (size_t)k * Q + l];
                            if (cj) v = std::conj(v);
                            fulli[((size_t)(b + 7 * r + 28 * cj) * Q + l) * Q + k] = v * ipow[(r * (k + l)) & 3];
                        }
    }
    // tensor-core M2L of the inner operator (p_i <= 15): G_v = the realified
    // F_v as TF32 hi / lo tiles in the canonical K-major layout, and the list-2
    // entries of the node schedule grouped by variant into tiles of up to
    // kTcPairs pairs
    std::vector<float> tc_tab;
    std::vector<int> tc_entries;
    std::vector<int4> tc_tiles;
    if (I.fp32 && I.P1i <= passes::kTcMaxP1 && opt.m2l_engine == DC_M2L_TENSOR) {
        const int Q = I.P1i;
        auto tf32 = [](float x) {   // round to nearest (ties away) at 10 mantissa bits
            uint32_t u;
            std::memcpy(&u, &x, 4);
            if ((u & 0x7F800000u) != 0x7F800000u) u = (u + 0x1000u) & 0xFFFFE000u;
            float r;
            std::memcpy(&r, &u, 4);
            return r;
        };
        tc_tab.assign((size_t)56 * 2 * 32 * passes::kTcK, 0.f);
        for (int v = 0; v < 56; ++v)
            for (int l = 0; l < Q; ++l)
                for (int k = 0; k < Q; ++k) {
                    const cd F = fulli[((size_t)v * Q + l) * Q + k];
                    const double g[2][2] = {{F.real(), -F.imag()}, {F.imag(), F.real()}};
                    for (int a = 0; a < 2; ++a)
                        for (int b = 0; b < 2; ++b) {
                            const float gf = (float)g[a][b], hi = tf32(gf), lo = tf32(gf - hi);
                            const size_t o = (size_t)passes::tc_offset(2 * l + a, 2 * k + b) / 4;
                            tc_tab[(size_t)v * 2 * 32 * passes::kTcK + o] = hi;
                            tc_tab[(size_t)v * 2 * 32 * passes::kTcK + 32 * passes::kTcK + o] = lo;
                        }
                }
        std::vector<std::vector<int>> byv(56);
        for (int c : nm2l)
            for (int e = T.v_ptr[c]; e < T.v_ptr[c + 1]; ++e) {
                const int code = vcode[e];
                byv[(code & 7) + 7 * ((code >> 3) & 3) + 28 * (code >> 5)].push_back(e);
            }
        for (int v = 0; v < 56; ++v) {
            const int first = int(tc_entries.size()), n = int(byv[v].size());
            tc_entries.insert(tc_entries.end(), byv[v].begin(), byv[v].end());
            for (int i = 0; i < n; i += passes::kTcPairs)
                tc_tiles.push_back(make_int4(v, first + i, std::min(passes::kTcPairs, n - i), 0));
        }
    }
    auto to_ff = [](const std::vector<cd> &v) {   // float-float: hi, then the rest
        std::vector<float4> f(v.size());
        for (size_t i = 0; i < v.size(); ++i) {
            const float hx = (float)v[i].real(), hy = (float)v[i].imag();
            f[i] = make_float4(hx, hy, (float)(v[i].real() - hx), (float)(v[i].imag() - hy));
        }
        return f;
    };
    auto lam_hilo = [](const std::vector<double> &v) {   // (hi, lo) float pairs
        std::vector<float2> f(v.size());
        for (size_t i = 0; i < v.size(); ++i) {
            const float h = (float)v[i];
            f[i] = make_float2(h, (float)(v[i] - (double)h));
        }
        return f;
    };
    auto to_f2 = [](const std::vector<cd> &v) {
        std::vector<float2> f(v.size());
        for (size_t i = 0; i < v.size(); ++i) f[i] = make_float2((float)v[i].real(), (float)v[i].imag());
        return f;
    };
    j_p2l.join();
    if (helper_oom) {
        err = "fmm build: host allocation failed";
        return DC_ERR_OOM;
    }
    I.p2l_rows = p2l_rows;
    cudaError_t e;
#define UP(buf, vec)                                                   \
    if ((e = upload(buf, vec, st)) != cudaSuccess) {                   \
        err = std::string("fmm upload: ") + cudaGetErrorString(e);      \
        return e == cudaErrorMemoryAllocation ? DC_ERR_OOM : DC_ERR_CUDA; \
    }
    UP(I.cc, cc);
    UP(I.cw, cw);
    UP(I.parent, T.parent);
    UP(I.child0, T.child0);
    UP(I.quad, quad);
    UP(I.pstart, T.piece_start);
    UP(I.pcount, T.piece_count);
    UP(I.pc, T.pc_xy);
    UP(I.pw, pw);
    UP(I.pseg, T.pc_seg);
    UP(I.u_ptr, T.u_ptr);
    UP(I.u_idx, T.u_idx);
    UP(I.v_ptr, T.v_ptr);
    UP(I.v_idx, T.v_idx);
    UP(I.v_off, voff);
    UP(I.w_ptr, T.w_ptr);
    UP(I.w_idx, T.w_idx);
    UP(I.x_ptr, T.x_ptr);
    UP(I.x_idx, T.x_idx);
    UP(I.p2m_leaves, p2m);
    UP(I.nt_leaves, leaves);
    UP(I.nt_start, start);
    UP(I.nt_count, cnt);
    UP(I.nt_perm, perm);
    UP(I.nt_own1, own1);
    UP(I.nt_own2, own2);
    UP(I.nt_xy, txy);
    UP(I.nt_items4, items4);
    UP(I.near_off, near_off);
    UP(I.far_off, far_off);
    UP(I.p2l_off, p2l_off);
    UP(I.p2l_cnt, p2l_cnt);
    UP(I.p2l_item, p2l_item);
    UP(I.iw64, iw64);
    UP(I.logw64, logw64);
    UP(I.plen64, plen64);
    UP(I.v_code, vcode);
    UP(I.m2m_cells, m2m_cells);
    {   // list-1 pieces of every leaf, flattened in list order: the offsets
        // here, the piece and segment numbers by uf_fill_kernel
        std::vector<int> ufp(nC + 1, 0);
        long long tot = 0;
        for (int c = 0; c < nC; ++c) {
            ufp[c] = int(tot);
            if (!T.is_leaf(c)) continue;
            for (int e = T.u_ptr[c]; e < T.u_ptr[c + 1]; ++e) tot += T.piece_count[T.u_idx[e]];
        }
        if (tot > INT_MAX) {
            err = "build_tree: too many list-1 pieces";
            return DC_ERR_UNSUPPORTED;
        }
        ufp[nC] = int(tot);
        UP(I.uf_ptr, ufp);
        if ((e = I.uf_idx.alloc(std::max<size_t>(tot, 1))) != cudaSuccess ||
            (e = I.uf_seg.alloc(std::max<size_t>(tot, 1))) != cudaSuccess) {
            err = std::string("fmm allocation: ") + cudaGetErrorString(e);
            return e == cudaErrorMemoryAllocation ? DC_ERR_OOM : DC_ERR_CUDA;
        }
        if (nC > 0) {
            uf_fill_kernel<<<nC, 128, 0, st>>>(I.u_ptr.ptr, I.u_idx.ptr, I.pstart.ptr, I.pcount.ptr, I.pseg.ptr,
                                               I.uf_ptr.ptr, I.uf_idx.ptr, I.uf_seg.ptr);
            note_launch();
        }
    }
    UP(I.mchunks, mchunks);
    UP(I.mred, mred);
    UP(I.pair_leaf, pair_leaf);
    UP(I.pair_geo, pair_geo);
    UP(I.binom32, binom32);
    if (I.fp32 && (e = I.mpart32.alloc((size_t)std::max(n_slots, 1) * 3 * I.P1i)) != cudaSuccess) {
        err = std::string("fmm allocation: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? DC_ERR_OOM : DC_ERR_CUDA;
    }
    UP(I.level_d, T.level);
    I.walk_nmax = std::min(passes::kWalkMax, std::max(1, T.depth - 1));
    auto make_chains = [&](const std::vector<int> &walk) {
        std::vector<int> ch(walk.size() * (size_t)(I.walk_nmax + 1), -1);
        for (size_t w = 0; w < walk.size(); ++w) {
            int *row = &ch[w * (I.walk_nmax + 1)];
            int n = 0;
            for (int c = walk[w]; c >= 0 && T.level[c] >= 2 && n < I.walk_nmax; c = T.parent[c]) row[1 + n++] = c;
            row[0] = n;
        }
        return ch;
    };
    UP(I.sched_all.chains, make_chains(aw));
    UP(I.sched_nodes.chains, make_chains(nw));
    UP(I.sched_all.walk, aw);
    UP(I.sched_all.l2l, al2l);
    UP(I.sched_nodes.l2l, nl2l);
    UP(I.sched_nodes.walk, nw);
    UP(I.sched_all.m2l, am2l);
    UP(I.sched_all.p2l, ap2l);
    UP(I.sched_nodes.m2l, nm2l);
    I.m2l_pairs_nodes = 0;
    for (int c : nm2l) I.m2l_pairs_nodes += T.v_ptr[c + 1] - T.v_ptr[c];
    UP(I.sched_nodes.p2l, np2l);
    if (!tc_tiles.empty()) {
        UP(I.tc_tab, tc_tab);
        UP(I.tc_entries, tc_entries);
        UP(I.tc_tiles, tc_tiles);
        I.n_tc_tiles = int(tc_tiles.size());
        if ((e = I.tc_y.alloc(T.v_idx.size() * 3 * 2 * (size_t)I.P1i)) != cudaSuccess ||
            (e = I.tc_err.alloc(2)) != cudaSuccess ||
            (e = cudaMemcpyAsync(I.tc_err.ptr, kTcErrInit, sizeof(kTcErrInit), cudaMemcpyHostToDevice, st)) !=
                cudaSuccess) {
            err = std::string("fmm allocation: ") + cudaGetErrorString(e);
            return e == cudaErrorMemoryAllocation ? DC_ERR_OOM : DC_ERR_CUDA;
        }
    }
#undef UP
    if ((e = upload_cd(I.m2m, m2m, st)) != cudaSuccess || (e = upload_cd(I.l2l, l2l, st)) != cudaSuccess ||
        (e = upload_cd(I.m2l, m2l, st)) != cudaSuccess || (e = I.M.alloc((size_t)nC * 3 * I.P1)) != cudaSuccess ||
        (e = I.L.alloc((size_t)nC * 3 * I.P1)) != cudaSuccess ||
        (e = upload_cd(I.base64, base, st)) != cudaSuccess ||
        (e = upload(I.baseff, to_ff(base), st)) != cudaSuccess ||
        (e = upload(I.m2mff, to_ff(m2m), st)) != cudaSuccess ||
        (e = upload(I.l2lff, to_ff(l2l), st)) != cudaSuccess ||
        (e = upload(I.m2m32i, to_f2(m2mi), st)) != cudaSuccess ||
        (e = upload(I.l2l32i, to_f2(l2li), st)) != cudaSuccess ||
        (e = upload(I.base32i, to_f2(basei), st)) != cudaSuccess ||
        (e = upload(I.m2lfull32i, to_f2(fulli), st)) != cudaSuccess ||
        (e = upload(I.lam_ff, lam_hilo(G.lambda), st)) != cudaSuccess ||
        (e = I.M32i.alloc((size_t)nC * 3 * I.P1i)) != cudaSuccess ||
        (e = I.L32i.alloc((size_t)nC * 3 * I.P1i)) != cudaSuccess ||
        (e = I.Lm2l32i.alloc((size_t)nC * 3 * I.P1i)) != cudaSuccess ||
        (e = I.Lm2l.alloc((size_t)nC * 3 * I.P1)) != cudaSuccess ||
        (e = I.sbar.alloc((size_t)3 * D.S)) != cudaSuccess ||
        (e = I.mbar.alloc((size_t)3 * D.S)) != cudaSuccess) {
        err = std::string("fmm allocation: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? DC_ERR_OOM : DC_ERR_CUDA;
    }
    // the other channel of interp output must be defined (zero) for passes
    cudaMemsetAsync(I.sbar.ptr, 0, I.sbar.bytes(), st);
    cudaMemsetAsync(I.mbar.ptr, 0, I.mbar.bytes(), st);
    // refinement buffers
    if ((e = I.ir_r.alloc((size_t)3 * D.N)) != cudaSuccess || (e = I.ir_d.alloc((size_t)3 * D.N)) != cudaSuccess ||
        (e = I.ir_t.alloc((size_t)3 * D.N)) != cudaSuccess) {
        err = std::string("fmm allocation: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? DC_ERR_OOM : DC_ERR_CUDA;
    }
    phase(1);   // schedules, node items, uploads
    // the two-level preconditioner (panel blocks + coarse space of panel
    // constants): wait for its thread and stream, then check both levels
    if (ov.th.joinable()) ov.th.join();
    if (pre_oom || pre_err != cudaSuccess) {
        err = pre_oom ? std::string("fmm preconditioner: host allocation failed")
                      : std::string("fmm preconditioner: ") + cudaGetErrorString(pre_err);
        return (pre_oom || pre_err == cudaErrorMemoryAllocation) ? DC_ERR_OOM : DC_ERR_CUDA;
    }
    if ((e = I.render_only ? cudaStreamSynchronize(I.pre_stream) : I.coarse.finish(I.pre_stream)) != cudaSuccess) {
        err = std::string("fmm preconditioner: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? DC_ERR_OOM : DC_ERR_CUDA;
    }
    ov.drain = nullptr;
    {
        std::vector<int> info(D.n_panels);
        e = cudaMemcpy(info.data(), I.pinfo.ptr, info.size() * sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            err = cudaGetErrorString(e);
            return DC_ERR_CUDA;
        }
        for (int j = 0; j < D.n_panels; ++j)
            if (info[j]) {
                err = "build_tree: singular self-interaction block on panel " + std::to_string(j);
                return DC_ERR_GEOMETRY;
            }
    }
    cudaFuncSetAttribute(passes::m2l_ff_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)passes::m2l_ff_smem(I.P1));
    cudaFuncSetAttribute(passes::m2l_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)passes::m2l_smem<double>(I.P1));
    cudaFuncSetAttribute(passes::p2l_kernel<double, passes::PiecesF64>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)passes::p2l_smem<double>(I.P1));
    cudaFuncSetAttribute(passes::p2m_kernel<double, passes::PiecesF64>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)passes::p2m_smem<double>(I.P1));
    cudaFuncSetAttribute(passes::p2l_flat_kernel<double, passes::PiecesF64>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)passes::p2l_flat_smem<double>(I.P1));
    cudaFuncSetAttribute(passes::m2m_ff_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)passes::mlff_smem(I.P1));
    phase(2);   // two-level preconditioner
    // The node near / far coefficients on a helper thread and the tree's
    // stream (free again) while the stored rows and the FP32 form are built
    // here; the helper's frees are held back and done with this thread's at
    // the end, so that no cudaFree waits for the other's kernels.
    cudaError_t near_err = cudaSuccess;
    bool near_oom = false;
    std::vector<std::pair<void *, size_t>> near_frees;
    struct Adopt {   // the helper's held frees join this thread's, on every return
        FreeDefer &d;
        std::vector<std::pair<void *, size_t>> &v;
        ~Adopt() { d.adopt(v); }
    } adopt_near{defer, near_frees};
    Joiner j_near;   // joined before the variables above go out of scope
    if (!I.render_only) {
        if ((e = cudaEventRecord(I.pre_ev, st)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(I.tree_stream, I.pre_ev, 0)) != cudaSuccess) {
            err = std::string("fmm event: ") + cudaGetErrorString(e);
            return DC_ERR_CUDA;
        }
        int dev = 0;
        cudaGetDevice(&dev);
        DevPool *pool = current_pool();
        j_near.run([&I, &near_err, &near_oom, &near_frees, dev, pool] {
            PoolScope ps(pool);
            FreeDefer held;
            try {
                near_err = cudaSetDevice(dev);
                if (near_err == cudaSuccess) near_err = I.build_near(I.tree_stream);
            } catch (...) {
                near_oom = true;
            }
            // its kernels are done before any block it released is recycled
            cudaStreamSynchronize(I.tree_stream);
            try {
                held.take(near_frees);
            } catch (...) {   // no room to hand them over: the guard frees them here
            }
        });
    }
    if ((e = I.build_rows(st)) != cudaSuccess) {
        err = std::string("stored P2M / P2L coefficients: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? DC_ERR_OOM : DC_ERR_CUDA;
    }
    phase(3);   // stored P2M / P2L rows
    if (ov.th32.joinable()) ov.th32.join();
    if (prep_failed) {
        err = "fmm32 build: host allocation failed";
        return DC_ERR_OOM;
    }
    dc_status r = I.fp32 ? I.build32(G, prep, txy, start, cnt, st, err) : DC_OK;
    phase(5);   // FP32 form
    j_near.join();
    if (near_oom || near_err != cudaSuccess) {
        err = near_oom ? std::string("near-field coefficients: host allocation failed")
                       : std::string("near-field coefficients: ") + cudaGetErrorString(near_err);
        return (near_oom || near_err == cudaErrorMemoryAllocation) ? DC_ERR_OOM : DC_ERR_CUDA;
    }
    if (!I.render_only && ((e = cudaEventRecord(I.pre_ev, I.tree_stream)) != cudaSuccess ||
                           (e = cudaStreamWaitEvent(st, I.pre_ev, 0)) != cudaSuccess)) {
        err = std::string("fmm event: ") + cudaGetErrorString(e);
        return DC_ERR_CUDA;
    }
    phase(4);   // near / far coefficients (the wait for them)
    return r;
}

void Fmm::build_timings(double out[6]) const {
    for (int i = 0; i < 6; ++i) out[i] = impl_->build_ms[i];
}

cudaError_t Fmm::prepare_eval(const double *sbar, const double *mbar, cudaStream_t st) {
    Impl &I = *impl_;
    I.render_pairs = 0;
    I.render_m2p = 0;
    I.render_flops = 0.0;
    I.render_eval_ms = 0.0;
    if (I.fp32) return I.prepare_render32(sbar, mbar, st);
    return I.passes(sbar, mbar, 1, 1, st, I.sched_all);
}

cudaError_t Fmm::apply_single_layer(const double *x, double *y, cudaStream_t st) {
    return impl_->apply_nodes(x, y, true, st);
}

cudaError_t Fmm::apply_double_layer(const double *x, double *y, cudaStream_t st) {
    return impl_->apply_nodes(x, y, false, st);
}

// w = M v: the two-level preconditioner, or the panel blocks alone when the
// coarse matrix could not be inverted.
cudaError_t Fmm::Impl::precond(const double *v, double *w, cudaStream_t st) {
    if (coarse.aggregated()) {   // coarse residual from the operator itself (FP32 in the FP32 form)
        cudaError_t e;
        if ((e = agg_py.ensure(3 * (size_t)D->N)) != cudaSuccess || (e = agg_gpy.ensure(3 * (size_t)D->N)) != cudaSuccess ||
            (e = coarse.apply_stage1(v, agg_py.ptr, st)) != cudaSuccess)
            return e;
        e = fp32 ? apply_nodes32(agg_py.ptr, agg_gpy.ptr, true, st) : apply_nodes(agg_py.ptr, agg_gpy.ptr, true, st);
        if (e != cudaSuccess) return e;
        return coarse.apply_stage2(pinv.ptr, v, agg_gpy.ptr, w, st);
    }
    if (coarse.ready()) return coarse.apply(pinv.ptr, v, w, st);
    return launch_block_apply(pinv.ptr, D->n_panels, D->g, v, w, st);
}

cudaError_t Fmm::apply_inner(const double *x, double *y, cudaStream_t st) {
    if (!impl_->fp32) return cudaErrorNotSupported;
    cudaError_t e;
    std::string msg;
    if (impl_->tc_err.ptr && (e = cudaMemsetAsync(impl_->tc_err.ptr, 0, sizeof(int), st)) != cudaSuccess) return e;
    if ((e = impl_->graph_matvec32(x, y, st)) != cudaSuccess) return e;
    return impl_->check_tc_wait(st, msg);
}

cudaError_t Fmm::apply_block_jacobi(const double *x, double *y, cudaStream_t st) {
    return launch_block_apply(impl_->pinv.ptr, impl_->D->n_panels, impl_->D->g, x, y, st);
}

cudaError_t Fmm::apply_precond(const double *x, double *y, cudaStream_t st) {
    return impl_->precond(x, y, st);
}

cudaError_t Fmm::apply_inner_raw(const double *x, double *y, cudaStream_t st) {
    if (!impl_->fp32) return cudaErrorNotSupported;
    cudaError_t e;
    std::string msg;
    if (impl_->tc_err.ptr && (e = cudaMemsetAsync(impl_->tc_err.ptr, 0, sizeof(int), st)) != cudaSuccess) return e;
    if ((e = impl_->apply_nodes32(x, y, true, st)) != cudaSuccess) return e;
    return impl_->check_tc_wait(st, msg);
}

namespace {
// v -> A M v with M the two-level preconditioner (right preconditioning).
struct PrecOp : Operator {
    Fmm::Impl *f;
    bool fp32 = false;
    cudaError_t apply(const double *v, double *y, cudaStream_t st) override {
        if (fp32) return f->graph_matvec32(v, y, st);
        cudaError_t e = f->precond(v, f->ir_t.ptr, st);
        if (e != cudaSuccess) return e;
        return f->apply_nodes(f->ir_t.ptr, y, true, st);
    }
    // the FP32 graph's own input and output: no copies in the Arnoldi loop
    double *in_buffer() override { return fp32 && f->graph_ensure() == cudaSuccess ? f->g_in.ptr : nullptr; }
    double *out_buffer() override { return fp32 && f->graph_ensure() == cudaSuccess ? f->g_out.ptr : nullptr; }
    cudaError_t apply_buffers(cudaStream_t st) override { return f->graph_launch(st); }
    const int *fault_flag() override { return fp32 ? f->tc_err.ptr : nullptr; }
};
}  // namespace

cudaError_t Fmm::solve(GmresWork *w, const double *b, double *x, const dc_options &opt,
                       cudaStream_t st, GmresResult &res, std::string &err, int *n_refine,
                       const double *Ax0) {
    cudaError_t e0;
    // Iterative refinement around right-preconditioned GMRES:
    //   r = b - A x            (FP64 FMM operator)
    //   z = GMRES(A' M, 0, r, tol')      A' = FP64 or FP32 FMM operator,
    //                                    M = two-level preconditioner: panel
    //                                    blocks of G_H inverted + a coarse
    //                                    space of panel constants
    //   x += M z
    // until ||r|| <= tol ||b|| per channel.  The preconditioner changes the
    // iteration, not the discrete solution of Eq. 27.
    Impl &I = *impl_;
    const int N = I.D->N;
    PrecOp op;
    op.f = &I;
    res = GmresResult();
    // the tensor-core M2L's wait-limit flag starts clear in every solve
    if (I.tc_err.ptr && (e0 = cudaMemsetAsync(I.tc_err.ptr, 0, sizeof(int), st)) != cudaSuccess) return e0;
    double bn[3], rn[3];
    cudaError_t e = vec_norms3(w, b, N, bn, st);
    if (e != cudaSuccess) return e;
    const int max_outer = I.fp32 ? 12 : 4;
    int used = 0;
    if (n_refine) *n_refine = 0;
    for (int outer = 0; outer <= max_outer; ++outer) {
        if (n_refine) *n_refine = outer;
        const double *Ax = Ax0;
        if (outer > 0 || !Ax0) {
            if ((e = I.apply_nodes(x, I.ir_t.ptr, true, st)) != cudaSuccess) return e;
            res.n_matvec++;
            Ax = I.ir_t.ptr;
        }
        if ((e = vec_residual(b, Ax, I.ir_r.ptr, 3 * N, st)) != cudaSuccess) return e;
        if ((e = vec_norms3(w, I.ir_r.ptr, N, rn, st)) != cudaSuccess) return e;
        int mask[3], any = 0;
        double need = 1.0;
        for (int c = 0; c < 3; ++c) {
            res.rel_resid[c] = bn[c] > 0 ? rn[c] / bn[c] : 0.0;
            res.true_rel_resid[c] = res.rel_resid[c];
            mask[c] = rn[c] > opt.gmres_tol * bn[c];
            any |= mask[c];
            if (mask[c]) need = std::min(need, opt.gmres_tol * bn[c] / rn[c]);
        }
        if (!any) {
            res.converged = 1;
            break;
        }
        if (outer == max_outer || used >= opt.gmres_max_iter) break;
        if ((e = vec_mask3(I.ir_r.ptr, N, mask, st)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(I.ir_d.ptr, 0, sizeof(double) * 3 * N, st)) != cudaSuccess) return e;
        const double floor32 = opt.inner_tol > 0.0 ? opt.inner_tol : 3e-5;
        double inner_tol = I.fp32 ? std::max(floor32, need) : std::max(0.5 * need, 1e-15);
        GmresResult inner;
        op.fp32 = I.fp32;
        e = gmres_solve(w, op, N, I.ir_r.ptr, I.ir_d.ptr, true, true, inner_tol, opt.gmres_restart,
                        opt.gmres_max_iter - used, st, inner, err);
        if (e != cudaSuccess) return e;
        if ((e = I.check_tc_wait(st, err)) != cudaSuccess) return e;
        int mx = 0;
        for (int c = 0; c < 3; ++c) {
            res.iters[c] += inner.iters[c];
            mx = std::max(mx, inner.iters[c]);
        }
        used += std::max(mx, 1);
        res.n_matvec += inner.n_matvec;
        if ((e = I.precond(I.ir_d.ptr, I.ir_t.ptr, st)) !=
            cudaSuccess)
            return e;
        if ((e = vec_axpy(x, I.ir_t.ptr, 3 * N, st)) != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

// cudaErrorTimeout when the tensor-core M2L's bounded wait ran out since the
// flag was last cleared (the library reports it as DC_ERR_TIMEOUT).
cudaError_t Fmm::Impl::check_tc_wait(cudaStream_t st, std::string &err) {
    if (!tc_err.ptr) return cudaSuccess;
    int flag = 0;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(&flag, tc_err.ptr, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return e;
    if (flag) {
        err = "tensor-core M2L: the MMAs of a tile did not complete within the wait limit";
        return cudaErrorTimeout;
    }
    return cudaSuccess;
}

cudaError_t Fmm::time_inner_m2l(int reps, cudaStream_t st, double out[6]) {
    return impl_->time_inner_m2l(reps, st, out);
}

void Fmm::set_eval_tile(int t) { impl_->opt.eval_tile = t; }

void Fmm::set_render_only(bool on) { impl_->render_only = on; }

void Fmm::compare_host_tree(const Geometry &G, double out[6]) const {
    const Tree &T = impl_->tree;
    Tree H;
    std::string err;
    out[0] = out[1] = 0.0;
    out[4] = T.ms_cut;
    out[5] = T.ms_lists;
    out[2] = T.n_cells();
    out[3] = double(T.pc_seg.size());
    if (!build_quadtree(G.seg_xy, impl_->opt.domain, impl_->opt.leaf_size, impl_->opt.max_depth, H, err)) return;
    // the lists as the build keeps them: entries whose source holds no pieces dropped
    std::vector<int> sub(H.n_cells(), 0);
    for (int c = H.n_cells() - 1; c >= 0; --c) {
        if (H.is_leaf(c)) sub[c] = H.piece_count[c];
        else
            for (int q = 0; q < 4; ++q) sub[c] += sub[H.child0[c] + q];
    }
    auto prune = [&](std::vector<int> &ptr, std::vector<int> &idx) {
        std::vector<int> np(ptr.size(), 0), ni;
        for (int c = 0; c + 1 < (int)ptr.size(); ++c) {
            for (int e = ptr[c]; e < ptr[c + 1]; ++e)
                if (sub[idx[e]] > 0) ni.push_back(idx[e]);
            np[c + 1] = int(ni.size());
        }
        ptr.swap(np);
        idx.swap(ni);
    };
    prune(H.u_ptr, H.u_idx);
    prune(H.v_ptr, H.v_idx);
    prune(H.w_ptr, H.w_idx);
    prune(H.x_ptr, H.x_idx);
    const bool same = H.x0 == T.x0 && H.y0 == T.y0 && H.w0 == T.w0 && H.depth == T.depth && H.level == T.level &&
                      H.parent == T.parent && H.child0 == T.child0 && H.ix == T.ix && H.iy == T.iy &&
                      H.level_start == T.level_start && H.piece_start == T.piece_start &&
                      H.piece_count == T.piece_count && H.pc_seg == T.pc_seg && H.pc_xy.size() == T.pc_xy.size() &&
                      H.u_ptr == T.u_ptr && H.u_idx == T.u_idx && H.v_ptr == T.v_ptr && H.v_idx == T.v_idx &&
                      H.w_ptr == T.w_ptr && H.w_idx == T.w_idx && H.x_ptr == T.x_ptr && H.x_idx == T.x_idx;
    out[0] = same ? 1.0 : 0.0;
    double d = 0.0;
    if (same)
        for (size_t i = 0; i < H.pc_xy.size(); ++i) d = std::max(d, std::fabs(H.pc_xy[i] - T.pc_xy[i]));
    out[1] = d;
}

cudaError_t Fmm::set_mma_skip_tile(int tile, cudaStream_t st) {
    Impl &I = *impl_;
    if (!I.tc_err.ptr) return cudaErrorNotSupported;
    return cudaMemcpyAsync(I.tc_err.ptr + 1, &tile, sizeof(int), cudaMemcpyHostToDevice, st);
}

namespace {
// Pixel index range [lo, hi) whose centres o + (i + 1/2) d lie in [a, b).
void pixel_range(double o, double d, int n, double a, double b, int &lo, int &hi) {
    auto centre = [&](long long i) { return o + (i + 0.5) * d; };
    auto first_ge = [&](double v) {
        double g = std::ceil((v - o) / d - 0.5);
        g = std::max(0.0, std::min(double(n), g));   // clamp before the cast
        long long i = (long long)g;
        while (i > 0 && centre(i - 1) >= v) --i;
        while (i < n && centre(i) < v) ++i;
        return int(i);
    };
    lo = first_ge(a);
    hi = first_ge(b);
}
}  // namespace

// The evaluation launch over the planned tiles (I.tiles, I.vps).
static dc_status launch_render(Fmm::Impl &I, int n_tiles, void *rgb, int rgb_dtype, unsigned char *rgb8,
                             const double *sbar, const double *mbar, cudaStream_t st, std::string &err) {
    if (n_tiles == 0) return DC_OK;
    cudaError_t e;
    if (I.eval_timing) {
        if (!I.ev0 && (e = cudaEventCreate(&I.ev0)) != cudaSuccess) return DC_ERR_CUDA;
        if (!I.ev1 && (e = cudaEventCreate(&I.ev1)) != cudaSuccess) return DC_ERR_CUDA;
        cudaEventRecord(I.ev0, st);
    }
    if (I.fp32)
        e = I.render_tiles32(n_tiles, rgb, rgb_dtype, rgb8, sbar, mbar, st);
    else {
        eval_tiles_kernel<<<n_tiles, 128, 0, st>>>(I.dt(), I.tiles.ptr, I.vps.ptr, I.P1,
                                                              I.M.ptr, I.L.ptr, sbar, mbar, rgb,
                                                              rgb_dtype, rgb8);
        note_launch();
        e = cudaGetLastError();
    }
    if (I.eval_timing) {
        cudaEventRecord(I.ev1, st);
        cudaEventSynchronize(I.ev1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, I.ev0, I.ev1);
        I.render_eval_ms += ms;
    }
    if (e != cudaSuccess) {
        err = cudaGetErrorString(e);
        return DC_ERR_CUDA;
    }
    return DC_OK;
}

dc_status Fmm::render_viewports(const VpDev *vpl, int n_vp, const double *sbar, const double *mbar,
                                void *rgb, int rgb_dtype, unsigned char *rgb8, cudaStream_t st,
                                std::string &err) {
    Impl &I = *impl_;
    const Tree &T = I.tree;
    for (int v = 0; v < n_vp; ++v) {
        const VpDev &vp = vpl[v];
        if (vp.width == 0 || vp.height == 0) continue;
        // every pixel centre must lie inside the root
        double xa = vp.x0 + 0.5 * vp.dx, xb = vp.x0 + (vp.width - 0.5) * vp.dx;
        double ya = vp.y0 + 0.5 * vp.dy, yb = vp.y0 + (vp.height - 0.5) * vp.dy;
        if (!(vp.dx > 0 && vp.dy > 0)) {
            err = "render_viewport: need x1 > x0 and y1 > y0";
            return DC_ERR_ARG;
        }
        if (!(xa >= T.x0 && xb < T.x0 + T.w0 && ya >= T.y0 && yb < T.y0 + T.w0)) {
            err = "render_viewport: pixel centres outside the quadtree root; widen options.domain";
            return DC_ERR_ARG;
        }
    }
    cudaError_t e;
    // the tile plan of the last call is kept on the device: the same
    // viewports (bit for bit) reuse it without rebuilding or uploading
    const bool same = I.plan_valid && I.plan_tile == I.opt.eval_tile && int(I.plan_vps.size()) == n_vp &&
                      (n_vp == 0 || std::memcmp(I.plan_vps.data(), vpl, sizeof(VpDev) * n_vp) == 0);
    if (same) {
        I.render_pairs += I.plan_pairs;
        I.render_m2p += I.plan_m2p;
        I.render_flops += I.plan_flops;
        return launch_render(I, I.plan_tiles, rgb, rgb_dtype, rgb8, sbar, mbar, st, err);
    }
    // the plan is built here while the stream runs the passes before the
    // render; its upload is ordered after them on the stream
    I.plan_valid = false;
    std::vector<Tile> tiles;
    std::vector<double> cost;   // estimated flops per tile
    int TW = kEvalTile, TH = kEvalTile;
    if (I.fp32) tile_shape(I.opt.eval_tile, TW, TH);
    long long pairs = 0;
    const long long m2p0 = I.render_m2p;
    const double flops0 = I.render_flops;
    for (int v = 0; v < n_vp; ++v) {
        const VpDev &vp = vpl[v];
        if (vp.width == 0 || vp.height == 0) continue;
        for (int c = 0; c < T.n_cells(); ++c) {
            if (!T.is_leaf(c)) continue;
            double w = T.width(c);
            double bx0 = T.x0 + double(T.ix[c]) * w, by0 = T.y0 + double(T.iy[c]) * w;
            int c0, c1, r0, r1;
            pixel_range(vp.x0, vp.dx, vp.width, bx0, bx0 + w, c0, c1);
            if (c1 <= c0) continue;
            pixel_range(vp.y0, vp.dy, vp.height, by0, by0 + w, r0, r1);
            if (r1 <= r0) continue;
            long long up = 0, npx = (long long)(c1 - c0) * (r1 - r0);
            for (int e2 = T.u_ptr[c]; e2 < T.u_ptr[c + 1]; ++e2) up += T.piece_count[T.u_idx[e2]];
            pairs += up * npx;
            long long wn = T.w_ptr[c + 1] - T.w_ptr[c];
            I.render_m2p += wn * npx;
            I.render_flops += 45.0 * double(up * npx) + 24.0 * I.P1 * double((1 + wn) * npx);
            for (int r = r0; r < r1; r += TH)
                for (int cc = c0; cc < c1; cc += TW) {
                    tiles.push_back({c, r, cc, std::min(TH, r1 - r), std::min(TW, c1 - cc), v});
                    const double tp = double(std::min(TH, r1 - r)) * std::min(TW, c1 - cc);
                    cost.push_back(tp * (45.0 * double(up) + 24.0 * I.P1 * double(1 + wn)));
                }
        }
    }
    {   // the most expensive tiles first (the persistent launch takes them in
        // order): a counting sort on the cost's binary logarithm in steps of
        // 1/16 octave, stable within a step (ties keep the generation order)
        constexpr int kSub = 16, kBins = 64 * kSub;
        std::vector<int> bin(tiles.size()), cnt(kBins + 1, 0);
        for (size_t i = 0; i < tiles.size(); ++i) {
            int e2 = 0;
            const double f = std::frexp(std::max(cost[i], 1.0), &e2);   // cost = f 2^e2, f in [0.5, 1)
            const int b = std::min(kBins - 1, std::max(0, e2 * kSub + int((2.0 * f - 1.0) * kSub)));
            bin[i] = kBins - 1 - b;   // descending cost
            cnt[bin[i] + 1]++;
        }
        for (int b = 0; b < kBins; ++b) cnt[b + 1] += cnt[b];
        std::vector<Tile> sorted(tiles.size());
        for (size_t i = 0; i < tiles.size(); ++i) sorted[cnt[bin[i]]++] = tiles[i];
        tiles.swap(sorted);
    }
    I.render_pairs += pairs;
    std::vector<VpDev> vv(vpl, vpl + n_vp);
    auto put = [&](auto &buf, const auto &v) -> cudaError_t {   // reuses the buffer when it is large enough
        cudaError_t r = buf.ensure(std::max<size_t>(v.size(), 1));
        if (r != cudaSuccess || v.empty()) return r;
        return cudaMemcpyAsync(buf.ptr, v.data(), v.size() * sizeof(v[0]), cudaMemcpyHostToDevice, st);
    };
    if (!tiles.empty() && ((e = put(I.tiles, tiles)) != cudaSuccess || (e = put(I.vps, vv)) != cudaSuccess)) {
        err = cudaGetErrorString(e);
        return DC_ERR_CUDA;
    }
    I.plan_vps = vv;
    I.plan_tile = I.opt.eval_tile;
    I.plan_tiles = int(tiles.size());
    I.plan_pairs = pairs;
    I.plan_m2p = I.render_m2p - m2p0;
    I.plan_flops = I.render_flops - flops0;
    I.plan_valid = true;
    return launch_render(I, I.plan_tiles, rgb, rgb_dtype, rgb8, sbar, mbar, st, err);
}


dc_status Fmm::eval_points(const double *xy, int n, const double *sbar, const double *mbar,
                           void *out, int out_dtype, cudaStream_t st, std::string &err) {
    Impl &I = *impl_;
    const Tree &T = I.tree;
    std::vector<double> h(2 * size_t(n));
    cudaError_t e = cudaMemcpyAsync(h.data(), xy, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        err = cudaGetErrorString(e);
        return DC_ERR_CUDA;
    }
    const int nC = T.n_cells();
    std::vector<int> leaf_of(n), cnt(nC, 0);
    for (int i = 0; i < n; ++i) {
        int lf = T.locate(h[2 * i], h[2 * i + 1]);
        if (lf < 0) {
            err = "eval_points: point outside the quadtree root; widen options.domain";
            return DC_ERR_ARG;
        }
        leaf_of[i] = lf;
        cnt[lf]++;
    }
    std::vector<int> start(nC), perm(n), leaves;
    std::vector<double> sxy(2 * size_t(n));
    for (int c = 0, acc = 0; c < nC; ++c) {
        start[c] = acc;
        acc += cnt[c];
        if (cnt[c]) leaves.push_back(c);
    }
    std::vector<int> fill(start);
    for (int i = 0; i < n; ++i) {
        int j = fill[leaf_of[i]]++;
        perm[j] = i;
        sxy[2 * j] = h[2 * i];
        sxy[2 * j + 1] = h[2 * i + 1];
    }
    if ((e = upload(I.pt_leaves, leaves, st)) != cudaSuccess || (e = upload(I.pt_start, start, st)) != cudaSuccess ||
        (e = upload(I.pt_count, cnt, st)) != cudaSuccess || (e = upload(I.pt_perm, perm, st)) != cudaSuccess ||
        (e = upload(I.pt_xy, sxy, st)) != cudaSuccess || (e = I.pt_out.ensure(3 * size_t(n))) != cudaSuccess) {
        err = cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? DC_ERR_OOM : DC_ERR_CUDA;
    }
    if (I.fp32) {
        std::vector<Tile> items;
        std::vector<float2> q32(n);
        for (int c : leaves) {
            double cx = T.cx(c), cy = T.cy(c);
            for (int j = start[c]; j < start[c] + cnt[c]; ++j)
                q32[j] = make_float2((float)(sxy[2 * j] - cx), (float)(sxy[2 * j + 1] - cy));
            for (int j = 0; j < cnt[c]; j += 64) items.push_back({c, start[c] + j, 0, std::min(64, cnt[c] - j), 0, 0});
        }
        if ((e = upload(I.pt_items, items, st)) != cudaSuccess || (e = upload(I.pt_q32, q32, st)) != cudaSuccess ||
            (e = I.eval_points32(int(items.size()), I.pt_out.ptr, sbar, mbar, st)) != cudaSuccess) {
            err = cudaGetErrorString(e);
            return DC_ERR_CUDA;
        }
    } else {
        std::vector<int4> items4;
        for (int c : leaves)
            for (int j = 0; j < cnt[c]; j += evalnodes::kNodeItem)
                items4.push_back(make_int4(c, start[c] + j, std::min(evalnodes::kNodeItem, cnt[c] - j), 0));
        if ((e = upload(I.pt_items4, items4, st)) != cudaSuccess ||
            (e = I.eval_list64(I.pt_items4.ptr, int(items4.size()), I.pt_xy.ptr, nullptr, nullptr,
                               I.pt_perm.ptr, sbar, mbar, 1, 1, I.pt_out.ptr, st)) != cudaSuccess) {
            err = cudaGetErrorString(e);
            return DC_ERR_CUDA;
        }
    }
    if ((e = launch_write_outputs(I.pt_out.ptr, n, out, out_dtype, nullptr, st)) != cudaSuccess) {
        err = cudaGetErrorString(e);
        return DC_ERR_CUDA;
    }
    return DC_OK;
}

dc_status Fmm::eval_points_dev(const double *xy, int n, const double *sbar, const double *mbar, double *out,
                               cudaStream_t st, std::string &err) {
    Impl &I = *impl_;
    if (n <= 0) return DC_OK;
    const Tree &T = I.tree;
    int n_items = 0;
    bool outside = false;
    const int item = I.fp32 ? 64 : evalnodes::kNodeItem;
    cudaError_t e = I.psort.run(xy, n, I.child0.ptr, I.cc.ptr, T.n_cells(), T.x0, T.y0, T.w0, item, I.fp32, st,
                                n_items, outside);
    if (e == cudaSuccess && outside) {
        err = "eval_points: point outside the quadtree root; widen options.domain";
        return DC_ERR_ARG;
    }
    if (e == cudaSuccess)
        e = I.fp32 ? I.eval_points32_at(I.psort.items32.ptr, n_items, I.psort.sxy.ptr, I.psort.perm.ptr, out, sbar,
                                        mbar, st)
                   : I.eval_list64(I.psort.items64.ptr, n_items, I.psort.sxy.ptr, nullptr, nullptr,
                                   I.psort.perm.ptr, sbar, mbar, 1, 1, out, st);
    if (e != cudaSuccess) {
        err = cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? DC_ERR_OOM : DC_ERR_CUDA;
    }
    return DC_OK;
}

void Fmm::fill_sizes(dc_sizes *out) const {
    const Tree &T = impl_->tree;
    out->n_pieces = int(T.pc_seg.size());
    out->n_cells = T.n_cells();
    out->n_leaves = T.n_leaves();
    out->depth = T.depth;
    out->root[0] = T.x0 + 0.5 * T.w0;
    out->root[1] = T.y0 + 0.5 * T.w0;
    out->root[2] = 0.5 * T.w0;
}

long long Fmm::p2p_pairs_nodes() const { return impl_->p2p_nodes; }
void Fmm::precond_info(double out[5]) const { impl_->coarse.info(out); }
long long Fmm::m2l_pairs() const { return impl_->m2l_cnt; }
long long Fmm::last_render_p2p_pairs() const { return impl_->render_pairs; }
long long Fmm::last_render_m2p_pairs() const { return impl_->render_m2p; }
double Fmm::last_render_eval_flops() const { return impl_->render_flops; }
void Fmm::set_eval_timing(bool on) { impl_->eval_timing = on; }
double Fmm::last_render_eval_ms() const { return impl_->render_eval_ms; }

}  // namespace dc
