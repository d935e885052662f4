// Per-panel features of the learned warm start (see mlp.cu) and the map
// from predicted scaled densities back to the node densities.
//
// A row is one (panel j, colour channel c).  In the panel's frame (origin at
// the centroid of its nodes, x along the chord from first to last node,
// lengths divided by the panel's arc length l_j):
//   [0, 4g)        own nodes: x, y, normal x, normal y
//   [4g, 6g)       own boundary colours u+, u- of channel c
//   [6g, 22g)      the 8 nearest other panels (by centroid): u+, u- of c
//   [22g, 22g+32)  the 8 neighbours: centroid offset (2), chord direction (2)
// The target of a row is l_j sigma at the panel's g nodes (scale-free).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "dc_internal.h"

namespace dc {

namespace {

constexpr int kNbr = 8;

struct FeatArgs {
    int P, g, F;
    const double *node_xy;    // [N][2]
    const double *node_n;     // [N][2] unit normals (own segment)
    const double *pc;         // [P][2] centroids
    const double *pt;         // [P][2] chord directions
    const double *plen;       // [P] arc lengths
    const int *nbr;           // [P][8] (-1 = none)
    const double *up, *um;    // [N][3]
    const double *sigma;      // [N][3] or null
    float *feat;              // [P*3][F]
    float *target;            // [P*3][g] or null
};

__global__ void features_kernel(FeatArgs a) {
    const int row = blockIdx.x, j = row / 3, c = row % 3;
    const int g = a.g;
    const double cx = a.pc[2 * j], cy = a.pc[2 * j + 1];
    const double tx = a.pt[2 * j], ty = a.pt[2 * j + 1], il = 1.0 / a.plen[j];
    float *out = a.feat + (size_t)row * a.F;
    for (int f = threadIdx.x; f < a.F; f += blockDim.x) {
        double v = 0.0;
        if (f < 4 * g) {
            int m = f / 4, comp = f % 4, i = j * g + m;
            double vx, vy;
            if (comp < 2) {
                vx = (a.node_xy[2 * i] - cx) * il;
                vy = (a.node_xy[2 * i + 1] - cy) * il;
            } else {
                vx = a.node_n[2 * i];
                vy = a.node_n[2 * i + 1];
            }
            v = (comp % 2 == 0) ? vx * tx + vy * ty : -vx * ty + vy * tx;
        } else if (f < 6 * g) {
            int q = f - 4 * g, m = q % g, i = j * g + m;
            v = (q < g) ? a.up[3 * i + c] : a.um[3 * i + c];
        } else if (f < 22 * g) {
            int q = f - 6 * g, k = q / (2 * g), r = q % (2 * g), m = r % g;
            int nb = a.nbr[kNbr * j + k];
            if (nb >= 0) {
                int i = nb * g + m;
                v = (r < g) ? a.up[3 * i + c] : a.um[3 * i + c];
            }
        } else {
            int q = f - 22 * g, k = q / 4, comp = q % 4;
            int nb = a.nbr[kNbr * j + k];
            if (nb >= 0) {
                double vx, vy;
                if (comp < 2) {
                    vx = (a.pc[2 * nb] - cx) * il;
                    vy = (a.pc[2 * nb + 1] - cy) * il;
                } else {
                    vx = a.pt[2 * nb];
                    vy = a.pt[2 * nb + 1];
                }
                v = (comp % 2 == 0) ? vx * tx + vy * ty : -vx * ty + vy * tx;
            }
        }
        out[f] = (float)v;
    }
    if (a.target && a.sigma)
        for (int m = threadIdx.x; m < g; m += blockDim.x)
            a.target[(size_t)row * g + m] = (float)(a.sigma[3 * (j * g + m) + c] * a.plen[j]);
}

// sigma[j g + m][c] = pred[(3 j + c) g + m] / l_j
__global__ void apply_pred_kernel(const float *__restrict__ pred, const double *__restrict__ plen, int P,
                                  int g, double *__restrict__ sigma) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P * 3 * g) return;
    int row = t / g, m = t % g, j = row / 3, c = row % 3;
    sigma[3 * (size_t)(j * g + m) + c] = (double)pred[t] / plen[j];
}

}  // namespace

// Panel frames and nearest panels on the host (grid search), uploaded once.
cudaError_t PanelFeatures::build(const Geometry &G, cudaStream_t st) {
    const int P = G.n_panels, g = G.g, s = G.s;
    std::vector<double> pc(2 * P), pt(2 * P), pl(P), nn(2 * (size_t)G.n_nodes());
    for (int j = 0; j < P; ++j) {
        double sx = 0, sy = 0;
        for (int m = 0; m < g; ++m) {
            sx += G.node_xy[2 * (j * g + m)];
            sy += G.node_xy[2 * (j * g + m) + 1];
        }
        pc[2 * j] = sx / g;
        pc[2 * j + 1] = sy / g;
        const double *a = &G.node_xy[2 * (j * g)], *b = &G.node_xy[2 * (j * g + g - 1)];
        double dx = b[0] - a[0], dy = b[1] - a[1], d = std::hypot(dx, dy);
        if (!(d > 0)) {  // g == 1: use the panel's own segments
            const double *q0 = &G.seg_xy[4 * (size_t)(j * s)], *q1 = &G.seg_xy[4 * (size_t)(j * s + s - 1)];
            dx = q1[2] - q0[0];
            dy = q1[3] - q0[1];
            d = std::hypot(dx, dy);
        }
        pt[2 * j] = dx / d;
        pt[2 * j + 1] = dy / d;
        double L = 0.0;
        for (int k = 0; k < s; ++k) {
            const double *q = &G.seg_xy[4 * (size_t)(j * s + k)];
            L += G.seg_w[j * s + k] * std::hypot(q[2] - q[0], q[3] - q[1]);
        }
        pl[j] = L;
    }
    for (int i = 0; i < G.n_nodes(); ++i) {
        const double *q = &G.seg_xy[4 * (size_t)G.node_seg[i]];
        double dx = q[2] - q[0], dy = q[3] - q[1], d = std::hypot(dx, dy);
        nn[2 * i] = dy / d;
        nn[2 * i + 1] = -dx / d;
    }
    // 8 nearest other panels by centroid: uniform grid, growing rings
    double lo[2] = {1e300, 1e300}, hi[2] = {-1e300, -1e300};
    for (int j = 0; j < P; ++j)
        for (int d = 0; d < 2; ++d) {
            lo[d] = std::min(lo[d], pc[2 * j + d]);
            hi[d] = std::max(hi[d], pc[2 * j + d]);
        }
    int R = std::max(1, int(std::sqrt(double(P) / 2.0)));
    double cw = std::max(hi[0] - lo[0], hi[1] - lo[1]) / R + 1e-300;
    std::vector<std::vector<int>> cells((size_t)R * R);
    auto cell_of = [&](double v, int d) { return std::min(R - 1, std::max(0, int((v - lo[d]) / cw))); };
    for (int j = 0; j < P; ++j) cells[(size_t)cell_of(pc[2 * j + 1], 1) * R + cell_of(pc[2 * j], 0)].push_back(j);
    std::vector<int> nbr((size_t)kNbr * P, -1);
    for (int j = 0; j < P; ++j) {
        int gx = cell_of(pc[2 * j], 0), gy = cell_of(pc[2 * j + 1], 1);
        std::vector<std::pair<double, int>> best;
        for (int ring = 0; ring <= R; ++ring) {
            for (int yy = gy - ring; yy <= gy + ring; ++yy)
                for (int xx = gx - ring; xx <= gx + ring; ++xx) {
                    if (std::max(std::abs(xx - gx), std::abs(yy - gy)) != ring) continue;
                    if (xx < 0 || yy < 0 || xx >= R || yy >= R) continue;
                    for (int k : cells[(size_t)yy * R + xx]) {
                        if (k == j) continue;
                        double d2 = std::pow(pc[2 * k] - pc[2 * j], 2) + std::pow(pc[2 * k + 1] - pc[2 * j + 1], 2);
                        best.push_back({d2, k});
                    }
                }
            std::sort(best.begin(), best.end());
            if ((int)best.size() > kNbr) best.resize(kNbr);
            // every unseen panel is at least ring * cw away
            if ((int)best.size() == kNbr && best.back().first <= std::pow(ring * cw, 2)) break;
        }
        for (int k = 0; k < (int)best.size(); ++k) nbr[(size_t)kNbr * j + k] = best[k].second;
    }
    P_ = P;
    g_ = g;
    cudaError_t e;
    auto up = [&](auto &buf, const auto &v) -> cudaError_t {
        cudaError_t r = buf.alloc(v.size());
        if (r != cudaSuccess) return r;
        return cudaMemcpyAsync(buf.ptr, v.data(), v.size() * sizeof(v[0]), cudaMemcpyHostToDevice, st);
    };
    if ((e = up(pc_, pc)) != cudaSuccess || (e = up(pt_, pt)) != cudaSuccess || (e = up(plen_, pl)) != cudaSuccess ||
        (e = up(nn_, nn)) != cudaSuccess || (e = up(nbr_, nbr)) != cudaSuccess)
        return e;
    return cudaStreamSynchronize(st);
}

cudaError_t PanelFeatures::compute(const DevGeom &D, const double *sigma, float *feat, float *target,
                                   cudaStream_t st) const {
    FeatArgs a;
    a.P = P_;
    a.g = g_;
    a.F = n_features(g_);
    a.node_xy = D.node_xy.ptr;
    a.node_n = nn_.ptr;
    a.pc = pc_.ptr;
    a.pt = pt_.ptr;
    a.plen = plen_.ptr;
    a.nbr = nbr_.ptr;
    a.up = D.u_plus.ptr;
    a.um = D.u_minus.ptr;
    a.sigma = sigma;
    a.feat = feat;
    a.target = target;
    features_kernel<<<P_ * 3, 128, 0, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

cudaError_t PanelFeatures::apply(const float *pred, double *sigma, cudaStream_t st) const {
    int n = P_ * 3 * g_, th = 256;
    apply_pred_kernel<<<(n + th - 1) / th, th, 0, st>>>(pred, plen_.ptr, P_, g_, sigma);
    note_launch();
    return cudaGetLastError();
}

}  // namespace dc
