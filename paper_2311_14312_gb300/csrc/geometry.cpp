// Host discretisation of a diffusion-curve drawing (setup, once per drawing).
//
// Sec. 4.2: densities live at g Gauss-Legendre nodes per panel and are
// interpolated (Eq. 10-11, written here in barycentric Lagrange form, which
// is the same map as Pbar Pring^-1) to the midpoints of s straight segments
// of equal arc length.  App. B: arc-length parametrisation of each cubic by
// Newton's method on L(t) = T, with L from Gauss-Legendre quadrature (here a
// per-curve table of cumulative lengths on 64 equal t-intervals plus a
// 16-point rule on the last partial interval).  App. A: every segment is
// weighted by (arc length) / (chord length).  A node's collocation point is
// the point of the solve polyline at the node's arc length; the segment that
// holds it is integrated with the singular rules Eq. 52 / Eq. 53 (App. C.1),
// both segments when the node sits on a vertex.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstring>
#include <functional>
#include <string>
#include <thread>
#include <vector>

#include "dc_internal.h"

namespace dc {

namespace {

constexpr double kPi = 3.14159265358979323846;

struct Cubic {
    double c[8];
    void point(double t, double &x, double &y) const {
        // de Casteljau
        double s = 1.0 - t;
        double ax = s * c[0] + t * c[2], ay = s * c[1] + t * c[3];
        double bx = s * c[2] + t * c[4], by = s * c[3] + t * c[5];
        double ex = s * c[4] + t * c[6], ey = s * c[5] + t * c[7];
        double fx = s * ax + t * bx, fy = s * ay + t * by;
        double gx = s * bx + t * ex, gy = s * by + t * ey;
        x = s * fx + t * gx;
        y = s * fy + t * gy;
    }
    double speed(double t) const {
        // B'(t) = 3 [ (1-t)^2 (C1-C0) + 2 t (1-t) (C2-C1) + t^2 (C3-C2) ]
        double s = 1.0 - t;
        double d0x = c[2] - c[0], d0y = c[3] - c[1];
        double d1x = c[4] - c[2], d1y = c[5] - c[3];
        double d2x = c[6] - c[4], d2y = c[7] - c[5];
        double x = 3.0 * (s * s * d0x + 2.0 * s * t * d1x + t * t * d2x);
        double y = 3.0 * (s * s * d0y + 2.0 * s * t * d1y + t * t * d2y);
        return std::sqrt(x * x + y * y);   // |B'| of a drawing's curves: far from overflow
    }
};

constexpr int kTab = 64;   // cumulative-length table intervals per curve
constexpr int kRule = 16;  // quadrature points per (partial) interval

struct ArcLength {
    const Cubic *cu;
    double cum[kTab + 1];
    double rx[kRule], rw[kRule], r8x[8], r8w[8];

    explicit ArcLength(const Cubic *c) : cu(c) {
        gauss_legendre_rule(kRule, rx, rw);
        gauss_legendre_rule(8, r8x, r8w);
        cum[0] = 0.0;
        for (int j = 0; j < kTab; ++j)
            cum[j + 1] = cum[j] + piece(double(j) / kTab, double(j + 1) / kTab);
    }
    double piece(double a, double b) const {
        double h = 0.5 * (b - a), m = 0.5 * (a + b), acc = 0.0;
        for (int i = 0; i < kRule; ++i) acc += rw[i] * cu->speed(m + h * rx[i]);
        return acc * h;
    }
    double total() const { return cum[kTab]; }
    double at(double t) const {
        if (t <= 0.0) return 0.0;
        if (t >= 1.0) return cum[kTab];
        int j = std::min(kTab - 1, int(t * kTab));
        return cum[j] + piece(double(j) / kTab, t);
    }
    // int_a^b |B'| by an 8-point Gauss-Legendre rule (for short intervals:
    // between neighbouring points of a panel)
    double short_piece(double a, double b) const {
        double h = 0.5 * (b - a), m = 0.5 * (a + b), acc = 0.0;
        for (int i = 0; i < 8; ++i) acc += r8w[i] * cu->speed(m + h * r8x[i]);
        return acc * h;
    }
    // t with L(t) = T from a nearby point t0 with L(t0) = T0 <= T (T - T0 a
    // small part of the curve): Newton on T0 + int_t0^t |B'| - T, started one
    // Newton step from t0, inside the bracket [t0, 1].
    double invert_from(double t0, double T0, double T) const {
        const double L = cum[kTab];
        if (T >= L) return 1.0;
        if (T <= T0) return t0;   // a node on its segment's start (T0 - T a rounding)
        double lo = t0, hi = 1.0;
        double t = std::min(1.0, t0 + (T - T0) / cu->speed(t0));
        for (int it = 0; it < 60; ++it) {
            const double f = T0 + short_piece(t0, t) - T;
            if (std::fabs(f) <= 4e-16 * L) break;
            if (f > 0) hi = t; else lo = t;
            double tn = t - f / cu->speed(t);
            if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
            if (tn == t) break;
            t = tn;
        }
        return t;
    }
    // t with L(t) = T: Newton t <- t - (L(t) - T) / |B'(t)| inside a bracket.
    double invert(double T) const {
        double L = cum[kTab];
        if (T <= 0.0) return 0.0;
        if (T >= L) return 1.0;
        int j = int(std::upper_bound(cum, cum + kTab + 1, T) - cum) - 1;
        j = std::max(0, std::min(kTab - 1, j));
        double lo = double(j) / kTab, hi = double(j + 1) / kTab;
        double t = lo + (hi - lo) * (T - cum[j]) / (cum[j + 1] - cum[j]);
        for (int it = 0; it < 60; ++it) {
            double f = cum[j] + piece(double(j) / kTab, t) - T;
            if (std::fabs(f) <= 4e-16 * L) break;
            if (f > 0) hi = t; else lo = t;
            double tn = t - f / cu->speed(t);
            if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
            if (tn == t) break;
            t = tn;
        }
        return t;
    }
};

bool finite_all(const double *v, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

}  // namespace

void gauss_legendre_rule(int n, double *x, double *w) {
    // Roots of P_n by Newton from x ~ cos(pi (4i + 3) / (4n + 2)), using
    // P_n' = n (P_{n-1} - x P_n) / (1 - x^2).
    auto eval = [n](double z, double &pn, double &pm1) {
        pm1 = 1.0;
        pn = z;
        for (int k = 2; k <= n; ++k) {
            double pk = ((2.0 * k - 1.0) * z * pn - (k - 1.0) * pm1) / k;
            pm1 = pn;
            pn = pk;
        }
    };
    for (int i = 0; i < n; ++i) {
        double z = std::cos(kPi * (4.0 * i + 3.0) / (4.0 * n + 2.0));
        double pn, pm1;
        for (int it = 0; it < 80; ++it) {
            eval(z, pn, pm1);
            double step = pn / (n * (pm1 - z * pn) / (1.0 - z * z));
            z -= step;
            if (std::fabs(step) <= 1e-16) break;
        }
        eval(z, pn, pm1);
        double pd = n * (pm1 - z * pn) / (1.0 - z * z);
        x[n - 1 - i] = z;
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * pd * pd);
    }
}

dc_status discretise(int n_curves, const double *ctrl, const int *panel_ptr,
                     const double *panel_start, const double *colours, int g,
                     int s, Geometry &out, std::string &err) {
    if (n_curves <= 0 || !ctrl || !panel_ptr || !panel_start || !colours) {
        err = "build_tree: n_curves must be positive and all arrays non-NULL";
        return DC_ERR_ARG;
    }
    if (g < 1 || g > kMaxG || s < g || s > 4096) {
        err = "build_tree: need 1 <= g <= 32 and g <= s_per_panel <= 4096";
        return DC_ERR_ARG;
    }
    if (panel_ptr[0] != 0) {
        err = "build_tree: panel_ptr[0] must be 0";
        return DC_ERR_ARG;
    }
    for (int i = 0; i < n_curves; ++i) {
        if (panel_ptr[i + 1] <= panel_ptr[i]) {
            err = "build_tree: every curve needs at least one panel";
            return DC_ERR_ARG;
        }
    }
    const int P = panel_ptr[n_curves];
    if ((long long)P * s > (1LL << 30)) {
        err = "build_tree: too many segments";
        return DC_ERR_ARG;
    }
    if (!finite_all(ctrl, size_t(8) * n_curves) || !finite_all(panel_start, size_t(P)) ||
        !finite_all(colours, size_t(12) * n_curves)) {
        err = "build_tree: non-finite input value";
        return DC_ERR_ARG;
    }
    for (int i = 0; i < n_curves; ++i) {
        if (panel_start[panel_ptr[i]] != 0.0) {
            err = "build_tree: the first panel of each curve must start at 0";
            return DC_ERR_ARG;
        }
        for (int j = panel_ptr[i] + 1; j < panel_ptr[i + 1]; ++j) {
            if (!(panel_start[j] > panel_start[j - 1]) || panel_start[j] >= 1.0) {
                err = "build_tree: panel starts must increase strictly within [0, 1)";
                return DC_ERR_ARG;
            }
        }
    }

    // the vectors keep their storage from the previous drawing (every entry
    // is written below): no fresh pages to fault in on a rebuild
    out.n_curves = n_curves;
    out.n_panels = P;
    out.g = g;
    out.s = s;
    const int N = P * g, S = P * s;
    out.node_xy.resize(size_t(2) * N);
    out.node_t.resize(N);
    out.node_seg.resize(N);
    out.node_seg2.resize(N);
    out.node_curve.resize(N);
    out.seg_xy.resize(size_t(4) * S);
    out.seg_w.resize(S);
    out.u_plus.resize(size_t(3) * N);
    out.u_minus.resize(size_t(3) * N);
    out.curve_len.resize(n_curves);

    std::vector<double> gx(g), gw(g);
    gauss_legendre_rule(g, gx.data(), gw.data());

    // Barycentric Lagrange interpolation at the segment midpoints (Eq. 10-11).
    std::vector<double> bw(g);
    for (int m = 0; m < g; ++m) {
        double prod = 1.0;
        for (int o = 0; o < g; ++o)
            if (o != m) prod *= (gx[m] - gx[o]);
        bw[m] = 1.0 / prod;
    }
    out.lambda.assign(size_t(s) * g, 0.0);
    for (int k = 0; k < s; ++k) {
        double xb = -1.0 + (2.0 * k + 1.0) / s;
        int hit = -1;
        for (int m = 0; m < g; ++m)
            if (xb == gx[m]) hit = m;
        if (hit >= 0) {
            out.lambda[size_t(k) * g + hit] = 1.0;
            continue;
        }
        double den = 0.0;
        for (int m = 0; m < g; ++m) den += bw[m] / (xb - gx[m]);
        for (int m = 0; m < g; ++m) out.lambda[size_t(k) * g + m] = (bw[m] / (xb - gx[m])) / den;
    }

    // curves are independent: host threads take them one at a time from a
    // shared counter (each writes only its curves' nodes and segments), then
    // the bounding boxes and the error of the first failing curve are merged
    struct Part {
        double bb[4] = {1e300, 1e300, -1e300, -1e300};
        dc_status st = DC_OK;
        int err_curve = INT_MAX;
        std::string err;
    };
    std::atomic<int> next_curve(0);
    auto work = [&](Part &pt) {
        std::vector<double> vx(s + 1), vy(s + 1), vt(s + 1);
        double *bb = pt.bb;
        for (int ci = next_curve.fetch_add(1); ci < n_curves; ci = next_curve.fetch_add(1)) {
            // a failing curve records its error and skips its other panels;
            // the smallest failing curve over all threads is reported
            auto fail = [&](const std::string &msg) {
                if (ci < pt.err_curve) {
                    pt.err_curve = ci;
                    pt.err = msg;
                    pt.st = DC_ERR_GEOMETRY;
                }
            };
            Cubic cu;
            std::memcpy(cu.c, ctrl + 8 * size_t(ci), sizeof(cu.c));
            ArcLength al(&cu);
            double L = al.total();
            out.curve_len[ci] = L;
            if (!(L > 0.0)) {
                fail("build_tree: curve " + std::to_string(ci) + " has zero length");
                continue;
            }
            bool bad = false;
            const double *col = colours + 12 * size_t(ci);
            for (int pj = panel_ptr[ci]; pj < panel_ptr[ci + 1] && !bad; ++pj) {
                double fa = panel_start[pj];
                double fb = (pj + 1 < panel_ptr[ci + 1]) ? panel_start[pj + 1] : 1.0;
                double sa = fa * L, sb = fb * L, h = (sb - sa) / s;
                // panel ends from the table (neighbouring panels share them
                // bit for bit), interior points each from the one before
                for (int k = 0; k <= s; ++k) {
                    double t;
                    if (k == 0) t = (fa == 0.0) ? 0.0 : al.invert(sa);
                    else if (k == s) t = (fb == 1.0) ? 1.0 : al.invert(sb);
                    else t = al.invert_from(vt[k - 1], sa + (k - 1) * h, sa + k * h);
                    vt[k] = t;
                    cu.point(t, vx[k], vy[k]);
                }
                for (int k = 0; k < s; ++k) {
                    size_t sid = size_t(pj) * s + k;
                    double *q = &out.seg_xy[4 * sid];
                    q[0] = vx[k];
                    q[1] = vy[k];
                    q[2] = vx[k + 1];
                    q[3] = vy[k + 1];
                    double chord = std::hypot(vx[k + 1] - vx[k], vy[k + 1] - vy[k]);
                    if (!(chord > 0.0)) {
                        fail("build_tree: zero-length segment on curve " + std::to_string(ci));
                        bad = true;
                        break;
                    }
                    out.seg_w[sid] = h / chord;
                    bb[0] = std::min(bb[0], std::min(q[0], q[2]));
                    bb[1] = std::min(bb[1], std::min(q[1], q[3]));
                    bb[2] = std::max(bb[2], std::max(q[0], q[2]));
                    bb[3] = std::max(bb[3], std::max(q[1], q[3]));
                }
                for (int m = 0; m < g && !bad; ++m) {
                    size_t nid = size_t(pj) * g + m;
                    double pos = 0.5 * (gx[m] + 1.0) * s;   // in segment units
                    int k = std::min(s - 1, int(std::floor(pos)));
                    double tau = pos - k;
                    int alt = -1;
                    if (tau < 1e-12 && k > 0) alt = pj * s + k - 1;
                    if (tau > 1.0 - 1e-12 && k + 1 < s) alt = pj * s + k + 1;
                    out.node_xy[2 * nid] = vx[k] + tau * (vx[k + 1] - vx[k]);
                    out.node_xy[2 * nid + 1] = vy[k] + tau * (vy[k + 1] - vy[k]);
                    out.node_seg[nid] = pj * s + k;
                    out.node_seg2[nid] = alt;
                    out.node_curve[nid] = ci;
                    double tn = al.invert(sa + 0.5 * (gx[m] + 1.0) * (sb - sa));
                    out.node_t[nid] = tn;
                    for (int c = 0; c < 3; ++c) {
                        // colours[ci][side][end][rgb], linear in t
                        double p0 = col[0 * 6 + 0 * 3 + c], p1 = col[0 * 6 + 1 * 3 + c];
                        double m0 = col[1 * 6 + 0 * 3 + c], m1 = col[1 * 6 + 1 * 3 + c];
                        out.u_plus[3 * nid + c] = (1.0 - tn) * p0 + tn * p1;
                        out.u_minus[3 * nid + c] = (1.0 - tn) * m0 + tn * m1;
                    }
                }
            }
        }
    };
    const int hw = int(std::max(1u, std::thread::hardware_concurrency()));
    const int nt = std::max(1, std::min({hw, 16, n_curves / 4}));
    std::vector<Part> parts(nt);
    {
        std::vector<std::thread> pool;
        for (int t = 1; t < nt; ++t) pool.emplace_back(work, std::ref(parts[t]));
        work(parts[0]);
        for (auto &th : pool) th.join();
    }
    const Part *first_bad = nullptr;
    for (const Part &pt : parts)
        if (pt.st != DC_OK && (!first_bad || pt.err_curve < first_bad->err_curve)) first_bad = &pt;
    if (first_bad) {
        err = first_bad->err;
        return first_bad->st;
    }
    double bb[4] = {1e300, 1e300, -1e300, -1e300};
    for (const Part &pt : parts) {
        bb[0] = std::min(bb[0], pt.bb[0]);
        bb[1] = std::min(bb[1], pt.bb[1]);
        bb[2] = std::max(bb[2], pt.bb[2]);
        bb[3] = std::max(bb[3], pt.bb[3]);
    }
    std::memcpy(out.bbox, bb, sizeof(bb));
    return DC_OK;
}

}  // namespace dc
