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
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "fmm_impl.h"
#include "segint.cuh"

namespace dc {

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



// ---------------------------------------------------------------- P2M --
__global__ void p2m_kernel(DevTree t, const int *__restrict__ leaves, const double *__restrict__ sbar,
                           const double *__restrict__ mbar, int use_s, int use_m, int P1,
                           double2 *__restrict__ M) {
    int cell = leaves[blockIdx.x];
    int k = threadIdx.x;
    if (k >= P1) return;
    double cx = t.cc[2 * cell], cy = t.cc[2 * cell + 1], r = t.cw[cell], ir = 1.0 / r;
    double2 acc[3] = {{0, 0}, {0, 0}, {0, 0}};
    int p0 = t.pstart[cell], pn = t.pcount[cell];
    for (int i = p0; i < p0 + pn; ++i) {
        const double *q = t.pc + 4 * (size_t)i;
        double2 a = make_double2((q[0] - cx) * ir, (q[1] - cy) * ir);
        double2 b = make_double2((q[2] - cx) * ir, (q[3] - cy) * ir);
        double dx = q[2] - q[0], dy = q[3] - q[1];
        double len = sqrt(dx * dx + dy * dy);
        double om = t.pw[i] * len;
        // S_k, S_{k-1}
        double2 S = make_double2(1.0, 0.0), Sp = make_double2(0.0, 0.0), ap = make_double2(1.0, 0.0);
        for (int m = 1; m <= k; ++m) {
            ap = cmul(ap, a);
            Sp = S;
            S = cadd(cmul(b, S), ap);
        }
        double2 cg = cscale(S, om / (k + 1));
        // -i (w / r) S_{k-1} * om,  w = (dx, dy)/len
        double2 wr = make_double2(dx / len * ir, dy / len * ir);
        double2 t1 = cmul(wr, Sp);
        double2 cf = make_double2(t1.y * om, -t1.x * om);
        int seg = t.pseg[i];
        for (int c = 0; c < 3; ++c) {
            if (use_s) {
                double s = sbar[3 * (size_t)seg + c];
                acc[c].x += s * cg.x;
                acc[c].y += s * cg.y;
            }
            if (use_m) {
                double mu = mbar[3 * (size_t)seg + c];
                acc[c].x += mu * cf.x;
                acc[c].y += mu * cf.y;
            }
        }
    }
    for (int c = 0; c < 3; ++c) M[((size_t)cell * 3 + c) * P1 + k] = acc[c];
}

// ---------------------------------------------------------------- M2M --
// Parent (cells [c_lo, c_hi) of one level) from its 4 children.
__global__ void m2m_kernel(DevTree t, int c_lo, int P1, const double2 *__restrict__ tab,
                           double2 *__restrict__ M) {
    int cell = c_lo + blockIdx.x;
    int k = threadIdx.x;
    int ch0 = t.child0[cell];
    if (k >= P1 || ch0 < 0) return;
    double2 acc[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int q = 0; q < 4; ++q) {
        const double2 *T = tab + ((size_t)q * P1 + k) * P1;
        const double2 *src = M + (size_t)(ch0 + q) * 3 * P1;
        for (int j = 0; j <= k; ++j) {
            double2 tq = T[j];
            for (int c = 0; c < 3; ++c) cfma(acc[c], tq, src[c * P1 + j]);
        }
    }
    for (int c = 0; c < 3; ++c) M[((size_t)cell * 3 + c) * P1 + k] = acc[c];
}

// ------------------------------------------------ L2L + M2L + P2L -------
__global__ void down_kernel(DevTree t, int c_lo, int level, int P1, const double2 *__restrict__ l2l,
                            const double2 *__restrict__ m2l, const double2 *__restrict__ M,
                            const double *__restrict__ sbar, const double *__restrict__ mbar,
                            int use_s, int use_m, double2 *__restrict__ L) {
    int cell = c_lo + blockIdx.x;
    int l = threadIdx.x;
    if (l >= P1) return;
    double2 acc[3] = {{0, 0}, {0, 0}, {0, 0}};
    double w = t.cw[cell];
    if (level >= 3) {   // Eq. 73 from the parent
        int par = t.parent[cell], q = t.quad[cell];
        const double2 *T = l2l + ((size_t)q * P1 + l) * P1;
        const double2 *src = L + (size_t)par * 3 * P1;
        for (int k = l; k < P1; ++k) {
            double2 tq = T[k];
            for (int c = 0; c < 3; ++c) cfma(acc[c], tq, src[c * P1 + k]);
        }
    }
    // Eq. 69 over list 2
    double mlogw = -log(w);
    for (int e = t.v_ptr[cell]; e < t.v_ptr[cell + 1]; ++e) {
        int src = t.v_idx[e];
        const double2 *T = m2l + ((size_t)t.v_off[e] * P1 + l) * P1;
        const double2 *ms = M + (size_t)src * 3 * P1;
        for (int k = 0; k < P1; ++k) {
            double2 tq = T[k];
            for (int c = 0; c < 3; ++c) cfma(acc[c], tq, ms[c * P1 + k]);
        }
        if (l == 0)
            for (int c = 0; c < 3; ++c) cfma(acc[c], make_double2(mlogw, 0.0), ms[c * P1]);
    }
    // Eq. 62 / 78 / 79 over list 4 (segments of bigger separated leaves)
    double cx = t.cc[2 * cell], cy = t.cc[2 * cell + 1], ir = 1.0 / w;
    for (int e = t.x_ptr[cell]; e < t.x_ptr[cell + 1]; ++e) {
        int src = t.x_idx[e];
        int p0 = t.pstart[src], pn = t.pcount[src];
        for (int i = p0; i < p0 + pn; ++i) {
            const double *q = t.pc + 4 * (size_t)i;
            double2 a = make_double2(q[0] - cx, q[1] - cy);
            double2 b = make_double2(q[2] - cx, q[3] - cy);
            double dx = q[2] - q[0], dy = q[3] - q[1];
            double len = sqrt(dx * dx + dy * dy);
            double om = t.pw[i];
            double2 wv = make_double2(dx / len, dy / len);
            double2 cg, cf;   // coefficient of sigma and of mu
            double2 lba = clog(cmul(b, cinv(a)));   // log(b / a), |arg| < pi
            if (l == 0) {
                double2 la = clog(a);
                double2 wb = cmul(make_double2(wv.x, -wv.y), b);
                double2 t2 = cmul(wb, lba);
                cg = make_double2(om * (len * (1.0 - la.x) - t2.x), om * (-len * la.y - t2.y));
                cf = make_double2(-om * lba.y, om * lba.x);   // i log(b/a)
            } else if (l == 1) {
                double2 t2 = cmul(make_double2(wv.x, -wv.y), lba);
                cg = cscale(t2, om * w);
                double2 al = cinv(make_double2(a.x * ir, a.y * ir));
                double2 be = cinv(make_double2(b.x * ir, b.y * ir));
                double2 ab = cmul(al, be);                      // T_0 = 1
                double2 iw = make_double2(-wv.y, wv.x);         // i w
                cf = cscale(cmul(iw, ab), om * len * ir);
            } else {
                double2 al = cinv(make_double2(a.x * ir, a.y * ir));
                double2 be = cinv(make_double2(b.x * ir, b.y * ir));
                double2 T = make_double2(1.0, 0.0), Tp = T, bp = make_double2(1.0, 0.0);
                for (int m = 1; m <= l - 1; ++m) {   // T_{l-1}, Tp = T_{l-2}
                    bp = cmul(bp, be);
                    Tp = T;
                    T = cadd(cmul(al, T), bp);
                }
                double2 ab = cmul(al, be);
                cg = cscale(cmul(ab, Tp), om * len / (double(l) * (l - 1)));
                double2 iw = make_double2(-wv.y, wv.x);
                cf = cscale(cmul(cmul(iw, ab), T), om * len * ir / l);
            }
            int seg = t.pseg[i];
            for (int c = 0; c < 3; ++c) {
                if (use_s) {
                    double s = sbar[3 * (size_t)seg + c];
                    acc[c].x += s * cg.x;
                    acc[c].y += s * cg.y;
                }
                if (use_m) {
                    double mu = mbar[3 * (size_t)seg + c];
                    acc[c].x += mu * cf.x;
                    acc[c].y += mu * cf.y;
                }
            }
        }
    }
    for (int c = 0; c < 3; ++c) L[((size_t)cell * 3 + c) * P1 + l] = acc[c];
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

__global__ void eval_tiles_kernel(DevTree t, const Tile *__restrict__ tiles, VpDev vp, int P1,
                                  const double2 *__restrict__ M, const double2 *__restrict__ L,
                                  const double *__restrict__ sbar, const double *__restrict__ mbar,
                                  void *rgb, int rgb_dtype, unsigned char *rgb8) {
    Tile tl = tiles[blockIdx.x];
    int npx = tl.nr * tl.nc;
    for (int j = threadIdx.x; j < npx; j += blockDim.x) {
        int r = tl.r0 + j / tl.nc, c = tl.c0 + j % tl.nc;
        double qx = vp.x0 + (c + 0.5) * vp.dx, qy = vp.y0 + (r + 0.5) * vp.dy;
        Acc3 u;
        long long pairs = 0;
        eval_point(t, tl.leaf, qx, qy, -1, -1, P1, M, L, sbar, mbar, 1, 1, u, pairs);
        size_t o = 3 * ((size_t)r * vp.width + c);
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

template <typename T>
cudaError_t upload(DevBuf<T> &buf, const std::vector<T> &v, cudaStream_t st) {
    cudaError_t e = buf.alloc(std::max<size_t>(v.size(), 1));
    if (e != cudaSuccess) return e;
    if (v.empty()) return cudaSuccess;
    return cudaMemcpyAsync(buf.ptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st);
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

// Up and down passes for segment densities (sbar / mbar), FP64.
cudaError_t Fmm::Impl::passes(const double *sb, const double *mb, int use_s, int use_m,
                              cudaStream_t st) {
    const int nC = tree.n_cells();
    size_t ebytes = (size_t)nC * 3 * P1 * sizeof(double2);
    cudaError_t e;
    if ((e = cudaMemsetAsync(M.ptr, 0, ebytes, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(L.ptr, 0, ebytes, st)) != cudaSuccess) return e;
    DevTree t = dt();
    int th = ((P1 + 31) / 32) * 32;
    if (n_p2m > 0)
        p2m_kernel<<<n_p2m, th, 0, st>>>(t, p2m_leaves.ptr, sb, mb, use_s, use_m, P1, M.ptr); note_launch();
    for (int l = tree.depth - 1; l >= 2; --l) {
        int lo = tree.level_start[l], hi = tree.level_start[l + 1];
        if (hi > lo) m2m_kernel<<<hi - lo, th, 0, st>>>(t, lo, P1, m2m.ptr, M.ptr); note_launch();
    }
    for (int l = 2; l <= tree.depth; ++l) {
        int lo = tree.level_start[l], hi = tree.level_start[l + 1];
        if (hi > lo)
            down_kernel<<<hi - lo, th, 0, st>>>(t, lo, l, P1, l2l.ptr, m2l.ptr, M.ptr, sb, mb,
                                                 use_s, use_m, L.ptr); note_launch();
    }
    return cudaGetLastError();
}

cudaError_t Fmm::Impl::apply_nodes(const double *x, double *y, bool single, cudaStream_t st) {
    cudaError_t e = launch_interp(*D, x, single ? sbar.ptr : mbar.ptr, st);
    if (e != cudaSuccess) return e;
    int us = single ? 1 : 0, um = single ? 0 : 1;
    if ((e = passes(sbar.ptr, mbar.ptr, us, um, st)) != cudaSuccess) return e;
    if (n_nt_leaves > 0)
        eval_targets_kernel<<<n_nt_leaves, 64, 0, st>>>(
            dt(), nt_leaves.ptr, nt_start.ptr, nt_count.ptr, nt_xy.ptr, nt_own1.ptr, nt_own2.ptr,
            nt_perm.ptr, P1, M.ptr, L.ptr, sbar.ptr, mbar.ptr, us, um, y); note_launch();
    return cudaGetLastError();
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
    if (!build_quadtree(G.seg_xy, opt.domain, opt.leaf_size, opt.max_depth, I.tree, err))
        return DC_ERR_GEOMETRY;
    const Tree &T = I.tree;
    const int nC = T.n_cells();
    std::vector<double> cc(2 * nC), cw(nC);
    std::vector<int> quad(nC, 0);
    for (int c = 0; c < nC; ++c) {
        cc[2 * c] = T.cx(c);
        cc[2 * c + 1] = T.cy(c);
        cw[c] = T.width(c);
        if (T.parent[c] >= 0) quad[c] = c - T.child0[T.parent[c]];
    }
    std::vector<double> pw(T.pc_seg.size());
    for (size_t i = 0; i < pw.size(); ++i) pw[i] = G.seg_w[T.pc_seg[i]];
    std::vector<int> voff(T.v_idx.size());
    long long m2l_cnt = 0;
    for (int c = 0; c < nC; ++c)
        for (int e = T.v_ptr[c]; e < T.v_ptr[c + 1]; ++e) {
            int s = T.v_idx[e];
            int dx = int(T.ix[c] - T.ix[s]), dy = int(T.iy[c] - T.iy[s]);
            if (std::abs(dx) > 3 || std::abs(dy) > 3 || std::max(std::abs(dx), std::abs(dy)) < 2) {
                err = "internal error: interaction-list offset out of range";
                return DC_ERR_GEOMETRY;
            }
            voff[e] = offset_code(dx, dy);
            ++m2l_cnt;
        }
    I.m2l_cnt = m2l_cnt;
    std::vector<int> p2m;
    for (int c = 0; c < nC; ++c)
        if (T.is_leaf(c) && T.piece_count[c] > 0) p2m.push_back(c);
    I.n_p2m = int(p2m.size());
    // node targets sorted by leaf
    const int N = G.n_nodes();
    std::vector<int> leaf_of(N), cnt(nC, 0);
    for (int i = 0; i < N; ++i) {
        int lf = T.locate(G.node_xy[2 * i], G.node_xy[2 * i + 1]);
        if (lf < 0) {
            err = "internal error: node outside the quadtree root";
            return DC_ERR_GEOMETRY;
        }
        leaf_of[i] = lf;
        cnt[lf]++;
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
    std::vector<cd> m2m, l2l, m2l;
    build_tables(I.p, m2m, l2l, m2l);
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
#undef UP
    if ((e = upload_cd(I.m2m, m2m, st)) != cudaSuccess || (e = upload_cd(I.l2l, l2l, st)) != cudaSuccess ||
        (e = upload_cd(I.m2l, m2l, st)) != cudaSuccess || (e = I.M.alloc((size_t)nC * 3 * I.P1)) != cudaSuccess ||
        (e = I.L.alloc((size_t)nC * 3 * I.P1)) != cudaSuccess ||
        (e = I.sbar.alloc((size_t)3 * D.S)) != cudaSuccess ||
        (e = I.mbar.alloc((size_t)3 * D.S)) != cudaSuccess) {
        err = std::string("fmm allocation: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? DC_ERR_OOM : DC_ERR_CUDA;
    }
    // the other channel of interp output must be defined (zero) for passes
    cudaMemsetAsync(I.sbar.ptr, 0, I.sbar.bytes(), st);
    cudaMemsetAsync(I.mbar.ptr, 0, I.mbar.bytes(), st);
    // block-Jacobi preconditioner over panels and refinement buffers
    if ((e = I.pinv.alloc((size_t)D.n_panels * D.g * D.g)) != cudaSuccess ||
        (e = I.pinfo.alloc((size_t)D.n_panels)) != cudaSuccess ||
        (e = I.ir_r.alloc((size_t)3 * D.N)) != cudaSuccess ||
        (e = I.ir_d.alloc((size_t)3 * D.N)) != cudaSuccess ||
        (e = I.ir_t.alloc((size_t)3 * D.N)) != cudaSuccess ||
        (e = launch_panel_block_inverse(D, I.pinv.ptr, I.pinfo.ptr, st)) != cudaSuccess) {
        err = std::string("fmm preconditioner: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? DC_ERR_OOM : DC_ERR_CUDA;
    }
    {
        std::vector<int> info(D.n_panels);
        e = cudaMemcpyAsync(info.data(), I.pinfo.ptr, info.size() * sizeof(int),
                            cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
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
    if (I.fp32) return I.build32(G, st, err);
    return DC_OK;
}

cudaError_t Fmm::prepare_eval(const double *sbar, const double *mbar, cudaStream_t st) {
    Impl &I = *impl_;
    I.render_pairs = 0;
    I.render_m2p = 0;
    I.render_flops = 0.0;
    I.render_eval_ms = 0.0;
    if (I.fp32) {
        cudaError_t e = I.to_f32_density(sbar, mbar, st);
        if (e != cudaSuccess) return e;
        return I.passes32(I.sbar32.ptr, I.mbar32.ptr, 1, 1, st);
    }
    return I.passes(sbar, mbar, 1, 1, st);
}

cudaError_t Fmm::apply_single_layer(const double *x, double *y, cudaStream_t st) {
    return impl_->apply_nodes(x, y, true, st);
}

cudaError_t Fmm::apply_double_layer(const double *x, double *y, cudaStream_t st) {
    return impl_->apply_nodes(x, y, false, st);
}

namespace {
// v -> A M^-1 v with M the panel-block preconditioner (right preconditioning).
struct PrecOp : Operator {
    Fmm::Impl *f;
    bool fp32 = false;
    cudaError_t apply(const double *v, double *y, cudaStream_t st) override {
        cudaError_t e = launch_block_apply(f->pinv.ptr, f->D->n_panels, f->D->g, v, f->ir_t.ptr, st);
        if (e != cudaSuccess) return e;
        return fp32 ? f->apply_nodes32(f->ir_t.ptr, y, true, st)
                    : f->apply_nodes(f->ir_t.ptr, y, true, st);
    }
};
}  // namespace

cudaError_t Fmm::solve(GmresWork *w, const double *b, double *x, const dc_options &opt,
                       cudaStream_t st, GmresResult &res, std::string &err) {
    // Iterative refinement around right-preconditioned GMRES:
    //   r = b - A x            (FP64 FMM operator)
    //   z = GMRES(A' M^-1, 0, r, tol')   A' = FP64 or FP32 FMM operator,
    //                                    M = block diagonal of G_H (panels)
    //   x += M^-1 z
    // until ||r|| <= tol ||b|| per channel.  The preconditioner changes the
    // iteration, not the discrete solution of Eq. 27.
    Impl &I = *impl_;
    const int N = I.D->N;
    PrecOp op;
    op.f = &I;
    res = GmresResult();
    double bn[3], rn[3];
    cudaError_t e = vec_norms3(w, b, N, bn, st);
    if (e != cudaSuccess) return e;
    const int max_outer = I.fp32 ? 12 : 4;
    int used = 0;
    for (int outer = 0; outer <= max_outer; ++outer) {
        if ((e = I.apply_nodes(x, I.ir_t.ptr, true, st)) != cudaSuccess) return e;
        res.n_matvec++;
        if ((e = vec_residual(b, I.ir_t.ptr, I.ir_r.ptr, 3 * N, st)) != cudaSuccess) return e;
        if ((e = vec_norms3(w, I.ir_r.ptr, N, rn, st)) != cudaSuccess) return e;
        int mask[3], any = 0;
        double need = 1.0;
        for (int c = 0; c < 3; ++c) {
            res.rel_resid[c] = bn[c] > 0 ? rn[c] / bn[c] : 0.0;
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
        double inner_tol = I.fp32 ? std::max(1e-5, need) : std::max(0.5 * need, 1e-15);
        GmresResult inner;
        op.fp32 = I.fp32;
        e = gmres_solve(w, op, N, I.ir_r.ptr, I.ir_d.ptr, inner_tol, opt.gmres_restart,
                        opt.gmres_max_iter - used, st, inner, err);
        if (e != cudaSuccess) return e;
        int mx = 0;
        for (int c = 0; c < 3; ++c) {
            res.iters[c] += inner.iters[c];
            mx = std::max(mx, inner.iters[c]);
        }
        used += std::max(mx, 1);
        res.n_matvec += inner.n_matvec;
        if ((e = launch_block_apply(I.pinv.ptr, I.D->n_panels, I.D->g, I.ir_d.ptr, I.ir_t.ptr, st)) !=
            cudaSuccess)
            return e;
        if ((e = vec_axpy(x, I.ir_t.ptr, 3 * N, st)) != cudaSuccess) return e;
    }
    return cudaGetLastError();
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

dc_status Fmm::render_grid(const VpDev &vp, const double *sbar, const double *mbar, void *rgb,
                           int rgb_dtype, unsigned char *rgb8, cudaStream_t st, std::string &err) {
    Impl &I = *impl_;
    const Tree &T = I.tree;
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
    cudaError_t e = cudaStreamSynchronize(st);   // the host tile list is rebuilt per call
    if (e != cudaSuccess) {
        err = cudaGetErrorString(e);
        return DC_ERR_CUDA;
    }
    std::vector<Tile> tiles;
    const int TS = 16;   // 16 x 16 pixels per block
    long long pairs = 0;
    for (int c = 0; c < T.n_cells(); ++c) {
        if (!T.is_leaf(c)) continue;
        double w = T.width(c);
        double bx0 = T.x0 + double(T.ix[c]) * w, by0 = T.y0 + double(T.iy[c]) * w;
        int c0, c1, r0, r1;
        pixel_range(vp.x0, vp.dx, vp.width, bx0, bx0 + w, c0, c1);
        pixel_range(vp.y0, vp.dy, vp.height, by0, by0 + w, r0, r1);
        if (c1 <= c0 || r1 <= r0) continue;
        long long up = 0, npx = (long long)(c1 - c0) * (r1 - r0);
        for (int e2 = T.u_ptr[c]; e2 < T.u_ptr[c + 1]; ++e2) up += T.piece_count[T.u_idx[e2]];
        pairs += up * npx;
        long long wn = T.w_ptr[c + 1] - T.w_ptr[c];
        I.render_m2p += wn * npx;
        I.render_flops += 45.0 * double(up * npx) + 24.0 * I.P1 * double((1 + wn) * npx);
        for (int r = r0; r < r1; r += TS)
            for (int cc = c0; cc < c1; cc += TS)
                tiles.push_back({c, r, cc, std::min(TS, r1 - r), std::min(TS, c1 - cc)});
    }
    I.render_pairs += pairs;
    if (tiles.empty()) return DC_OK;
    if ((e = upload(I.tiles, tiles, st)) != cudaSuccess) {
        err = cudaGetErrorString(e);
        return DC_ERR_CUDA;
    }
    if (I.eval_timing) {
        if (!I.ev0 && (e = cudaEventCreate(&I.ev0)) != cudaSuccess) return DC_ERR_CUDA;
        if (!I.ev1 && (e = cudaEventCreate(&I.ev1)) != cudaSuccess) return DC_ERR_CUDA;
        cudaEventRecord(I.ev0, st);
    }
    if (I.fp32)
        e = I.render_tiles32(vp, int(tiles.size()), rgb, rgb_dtype, rgb8, st);
    else
        eval_tiles_kernel<<<int(tiles.size()), 128, 0, st>>>(I.dt(), I.tiles.ptr, vp, I.P1, I.M.ptr,
                                                              I.L.ptr, sbar, mbar, rgb, rgb_dtype,
                                                              rgb8); note_launch();
    if (I.eval_timing) {
        cudaEventRecord(I.ev1, st);
        cudaEventSynchronize(I.ev1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, I.ev0, I.ev1);
        I.render_eval_ms += ms;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        err = cudaGetErrorString(e);
        return DC_ERR_CUDA;
    }
    return DC_OK;
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
            for (int j = 0; j < cnt[c]; j += 64) items.push_back({c, start[c] + j, 0, std::min(64, cnt[c] - j), 0});
        }
        if ((e = upload(I.pt_items, items, st)) != cudaSuccess || (e = upload(I.pt_q32, q32, st)) != cudaSuccess ||
            (e = I.eval_points32(int(items.size()), I.pt_out.ptr, st)) != cudaSuccess) {
            err = cudaGetErrorString(e);
            return DC_ERR_CUDA;
        }
    } else {
        eval_targets_kernel<<<int(leaves.size()), 64, 0, st>>>(
            I.dt(), I.pt_leaves.ptr, I.pt_start.ptr, I.pt_count.ptr, I.pt_xy.ptr, nullptr, nullptr,
            I.pt_perm.ptr, I.P1, I.M.ptr, I.L.ptr, sbar, mbar, 1, 1, I.pt_out.ptr); note_launch();
    }
    if ((e = launch_write_outputs(I.pt_out.ptr, n, out, out_dtype, nullptr, st)) != cudaSuccess) {
        err = cudaGetErrorString(e);
        return DC_ERR_CUDA;
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
long long Fmm::m2l_pairs() const { return impl_->m2l_cnt; }
long long Fmm::last_render_p2p_pairs() const { return impl_->render_pairs; }
long long Fmm::last_render_m2p_pairs() const { return impl_->render_m2p; }
double Fmm::last_render_eval_flops() const { return impl_->render_flops; }
void Fmm::set_eval_timing(bool on) { impl_->eval_timing = on; }
double Fmm::last_render_eval_ms() const { return impl_->render_eval_ms; }

}  // namespace dc
