// Adaptive panel split of a drawing (host, setup): each curve starts as one
// panel and a panel is bisected in arc-length fraction while it is longer
// than ratio x its distance to the nearest other curve (the rule the
// 200-curve workload is built with; the paper subdivides adaptively as well,
// Sec. 6.1, there by the density instead of the geometry), or longer than
// max_len, or while the curve has fewer than min_panels panels of equal
// fraction, for at most max_level bisections.  Lengths and distances are
// measured on a polyline of kSamples points per curve at uniform Bezier
// parameter (within one sample spacing); break points are dyadic fractions.
#include <algorithm>
#include <cmath>
#include <unordered_map>
#include <vector>

#include "dc_internal.h"

namespace dc {

namespace {

constexpr int kSamples = 256;

struct Grid {
    double x0, y0, h;
    std::unordered_map<long long, std::vector<int>> cells;
    long long key(long long i, long long j) const { return (i << 32) ^ (j & 0xffffffffLL); }
    long long ix(double x) const { return (long long)std::floor((x - x0) / h); }
    long long iy(double y) const { return (long long)std::floor((y - y0) / h); }
};

}  // namespace

dc_status adaptive_panels(int n_curves, const double *ctrl, double ratio, int max_level, int min_panels,
                          double max_len, std::vector<int> &ptr, std::vector<double> &start, std::string &err) {
    const int S = kSamples;
    std::vector<double> P((size_t)n_curves * S * 2);
    for (int c = 0; c < n_curves; ++c) {
        const double *C = ctrl + 8 * (size_t)c;
        for (int k = 0; k < S; ++k) {
            const double t = (k == S - 1) ? 1.0 : k * (1.0 / (S - 1)), u = 1.0 - t;   // uniform in t
            const double b0 = u * u * u, b1 = 3 * t * u * u, b2 = 3 * t * t * u, b3 = t * t * t;
            P[2 * ((size_t)c * S + k)] = b0 * C[0] + b1 * C[2] + b2 * C[4] + b3 * C[6];
            P[2 * ((size_t)c * S + k) + 1] = b0 * C[1] + b1 * C[3] + b2 * C[5] + b3 * C[7];
        }
    }
    // distance from every sample to the nearest sample of another curve:
    // a uniform grid with cell h, searched ring by ring until the ring's
    // nearest possible point is farther than the best found
    std::vector<double> dist((size_t)n_curves * S, INFINITY);
    if (n_curves > 1) {
        double lo[2] = {INFINITY, INFINITY}, hi[2] = {-INFINITY, -INFINITY};
        for (size_t i = 0; i < (size_t)n_curves * S; ++i)
            for (int d = 0; d < 2; ++d) {
                lo[d] = std::min(lo[d], P[2 * i + d]);
                hi[d] = std::max(hi[d], P[2 * i + d]);
            }
        const double ext = std::max(hi[0] - lo[0], hi[1] - lo[1]);
        Grid G{lo[0], lo[1], std::max(ext / std::sqrt((double)n_curves * S / 8.0), 1e-12), {}};
        for (int i = 0; i < n_curves * S; ++i) G.cells[G.key(G.ix(P[2 * i]), G.iy(P[2 * i + 1]))].push_back(i);
        const long long nmax = (long long)std::ceil(ext / G.h) + 2;
        for (int i = 0; i < n_curves * S; ++i) {
            const int own = i / S;
            const double x = P[2 * i], y = P[2 * i + 1];
            const long long ci = G.ix(x), cj = G.iy(y);
            double best2 = INFINITY;
            for (long long r = 0; r <= nmax; ++r) {
                // every point in ring r lies at least (r - 1) h away
                if (r >= 1 && (double)(r - 1) * G.h * (double)(r - 1) * G.h > best2) break;
                for (long long a = ci - r; a <= ci + r; ++a)
                    for (long long b = cj - r; b <= cj + r; ++b) {
                        if (std::max(std::llabs(a - ci), std::llabs(b - cj)) != r) continue;
                        auto it = G.cells.find(G.key(a, b));
                        if (it == G.cells.end()) continue;
                        for (int j : it->second) {
                            if (j / S == own) continue;
                            const double dx = P[2 * j] - x, dy = P[2 * j + 1] - y;
                            best2 = std::min(best2, dx * dx + dy * dy);
                        }
                    }
            }
            dist[i] = std::sqrt(best2);
        }
    }
    ptr.assign(1, 0);
    start.clear();
    std::vector<double> cum(S), frac(S);
    for (int c = 0; c < n_curves; ++c) {
        const double *p = &P[(size_t)c * S * 2];
        cum[0] = 0.0;
        for (int k = 1; k < S; ++k) cum[k] = cum[k - 1] + std::hypot(p[2 * k] - p[2 * k - 2], p[2 * k + 1] - p[2 * k - 1]);
        const double L = cum[S - 1];
        if (!(L > 0.0)) {
            err = "build_tree: zero-length curve " + std::to_string(c);
            return DC_ERR_GEOMETRY;
        }
        for (int k = 0; k < S; ++k) frac[k] = cum[k] / L;
        const double *d = &dist[(size_t)c * S];
        std::vector<double> out;
        struct Item { double a, b; int lev; };
        std::vector<Item> stack{{0.0, 1.0, 0}};
        while (!stack.empty()) {
            const Item it = stack.back();
            stack.pop_back();
            // samples from just before a to just after b
            const int ia = int(std::lower_bound(frac.begin(), frac.end(), it.a) - frac.begin());
            const int ib = int(std::upper_bound(frac.begin(), frac.end(), it.b) - frac.begin());
            const int lo_i = std::max(ia - 1, 0), hi_i = std::min(ib + 1, S);
            double dmin = INFINITY;
            for (int k = lo_i; k < hi_i; ++k) dmin = std::min(dmin, d[k]);
            const double length = (it.b - it.a) * L;
            const bool need = it.lev < max_level &&
                              ((it.b - it.a) > 1.0 / min_panels + 1e-15 || length > max_len || length > ratio * dmin);
            if (need) {
                const double mid = 0.5 * (it.a + it.b);
                stack.push_back({mid, it.b, it.lev + 1});
                stack.push_back({it.a, mid, it.lev + 1});
            } else {
                out.push_back(it.a);
            }
        }
        std::sort(out.begin(), out.end());
        start.insert(start.end(), out.begin(), out.end());
        ptr.push_back(int(start.size()));
    }
    return DC_OK;
}

}  // namespace dc
