// Non-uniform quadtree with segment clipping and the four interaction lists.
//
// Sec. 5.1 / App. E.5: cells split into 4 equal children while they hold more
// than b degrees of freedom.  Sec. 5.2: every segment is clipped at cell
// boundaries so that each piece lies in exactly one leaf; here a segment is
// carried as parameter intervals [ta, tb] that are cut where the segment
// crosses a splitting midline, each sub-interval going to the child that
// holds its midpoint -- the pieces partition the segment exactly.
// Lists (App. E.3, E.5, Alg. 8): list 1 = adjacent leaves (self included),
// list 2 = same-level cells whose parents are adjacent but which are not,
// list 3 = descendants of a leaf's colleagues that are not adjacent to it but
// whose parent is, list 4 = the dual of list 3.  Cells "touch" when their
// closed boxes share at least a point (corners included).
#include "tree.h"

#include <atomic>
#include <thread>

#include <algorithm>
#include <cmath>
#include <unordered_set>

namespace dc {

double Tree::width(int c) const { return std::ldexp(w0, -level[c]); }
double Tree::cx(int c) const { return x0 + (double(ix[c]) + 0.5) * width(c); }
double Tree::cy(int c) const { return y0 + (double(iy[c]) + 0.5) * width(c); }

int Tree::n_leaves() const {
    int n = 0;
    for (int c = 0; c < n_cells(); ++c) n += is_leaf(c);
    return n;
}

int Tree::locate(double x, double y) const {
    if (!(x >= x0 && x < x0 + w0 && y >= y0 && y < y0 + w0)) return -1;
    int c = 0;
    while (child0[c] >= 0) {
        double xm = cx(c), ym = cy(c);
        c = child0[c] + (x >= xm ? 1 : 0) + (y >= ym ? 2 : 0);
    }
    return c;
}

namespace {

struct Piece {
    int seg;
    double ta, tb;
};

bool touches(const Tree &t, int a, int b) {
    if (t.level[a] > t.level[b]) std::swap(a, b);
    int d = t.level[b] - t.level[a];
    long long ax0 = t.ix[a] << d, ax1 = (t.ix[a] + 1) << d;
    long long ay0 = t.iy[a] << d, ay1 = (t.iy[a] + 1) << d;
    long long bx0 = t.ix[b], bx1 = t.ix[b] + 1, by0 = t.iy[b], by1 = t.iy[b] + 1;
    return bx1 >= ax0 && bx0 <= ax1 && by1 >= ay0 && by0 <= ay1;
}

void to_csr(const std::vector<std::vector<int>> &lists, std::vector<int> &ptr,
            std::vector<int> &idx) {
    ptr.assign(lists.size() + 1, 0);
    for (size_t i = 0; i < lists.size(); ++i) ptr[i + 1] = ptr[i] + int(lists[i].size());
    idx.resize(ptr.back());
    for (size_t i = 0; i < lists.size(); ++i)
        std::copy(lists[i].begin(), lists[i].end(), idx.begin() + ptr[i]);
}

}  // namespace

bool quadtree_root(const std::vector<double> &seg_xy, const double domain[4], Tree &t, std::string &err) {
    const int S = int(seg_xy.size() / 4);
    double lo[2] = {domain[0], domain[1]}, hi[2] = {domain[2], domain[3]};
    for (int k = 0; k < S; ++k) {
        const double *q = &seg_xy[4 * size_t(k)];
        lo[0] = std::min(lo[0], std::min(q[0], q[2]));
        lo[1] = std::min(lo[1], std::min(q[1], q[3]));
        hi[0] = std::max(hi[0], std::max(q[0], q[2]));
        hi[1] = std::max(hi[1], std::max(q[1], q[3]));
    }
    double ext = std::max(hi[0] - lo[0], hi[1] - lo[1]);
    if (!(ext > 0.0)) ext = 1.0;
    if (!std::isfinite(ext)) {
        err = "build_tree: non-finite extent";
        return false;
    }
    t.w0 = std::ldexp(1.0, int(std::ceil(std::log2(ext * (1.0 + 1.0 / 256)))));
    double grid = t.w0 / 1024.0, small = ext * 1e-6;
    t.x0 = std::floor((lo[0] - small) / grid) * grid;
    t.y0 = std::floor((lo[1] - small) / grid) * grid;
    if (!(t.x0 + t.w0 > hi[0] && t.y0 + t.w0 > hi[1])) {
        err = "build_tree: internal error choosing the root box";
        return false;
    }
    return true;
}

bool build_quadtree(const std::vector<double> &seg_xy, const double domain[4], int leaf_size,
                    int max_depth, Tree &t, std::string &err) {
    t = Tree();
    const int S = int(seg_xy.size() / 4);
    if (!quadtree_root(seg_xy, domain, t, err)) return false;

    // breadth-first construction
    std::vector<std::vector<Piece>> cur(1);
    cur[0].reserve(S);
    for (int k = 0; k < S; ++k) cur[0].push_back({k, 0.0, 1.0});
    t.level.push_back(0);
    t.parent.push_back(-1);
    t.child0.push_back(-1);
    t.ix.push_back(0);
    t.iy.push_back(0);
    t.level_start.push_back(0);
    std::vector<std::vector<Piece>> leaf_pieces;   // indexed by cell
    leaf_pieces.resize(1);
    int lev = 0;
    int first = 0;   // first cell of the current level
    while (true) {
        const int n_level = int(cur.size());
        const int next_first = t.n_cells();
        // which cells of this level split (their children are numbered in
        // cell order), then the pieces of each splitting cell are cut at its
        // midlines into the children's lists, cells in parallel
        std::vector<int> split(n_level, -1);
        int n_split = 0;
        for (int j = 0; j < n_level; ++j) {
            const int c = first + j;
            if (int(cur[j].size()) > leaf_size && lev < max_depth) {
                split[j] = n_split++;
                t.child0[c] = t.n_cells();
                for (int q = 0; q < 4; ++q) {
                    t.level.push_back(lev + 1);
                    t.parent.push_back(c);
                    t.child0.push_back(-1);
                    t.ix.push_back(2 * t.ix[c] + (q & 1));
                    t.iy.push_back(2 * t.iy[c] + (q >> 1));
                }
            } else {
                leaf_pieces[c].swap(cur[j]);
            }
        }
        leaf_pieces.resize(t.n_cells());
        std::vector<std::vector<Piece>> nxt(4 * (size_t)n_split);
        // work items: pieces [a, b) of splitting cell j (large cells are
        // cut in chunks); each item fills its own four lists, which are
        // concatenated per cell in item order (deterministic)
        struct Item {
            int j, a, b;
            std::vector<Piece> kids[4];
        };
        constexpr int kChunkPieces = 8192;
        std::vector<Item> items;
        for (int j = 0; j < n_level; ++j) {
            if (split[j] < 0) continue;
            const int n = int(cur[j].size());
            for (int a0 = 0; a0 < n; a0 += kChunkPieces) items.push_back({j, a0, std::min(n, a0 + kChunkPieces), {}});
        }
        auto cut = [&](Item &it) {
            const int c = first + it.j;
            const std::vector<Piece> &pcs = cur[it.j];
            for (int q = 0; q < 4; ++q) it.kids[q].reserve((it.b - it.a) / 2 + 4);
            const double xm = t.cx(c), ym = t.cy(c);
            for (int pi = it.a; pi < it.b; ++pi) {
                const Piece &p = pcs[pi];
                const double *q = &seg_xy[4 * size_t(p.seg)];
                double dx = q[2] - q[0], dy = q[3] - q[1];
                double cuts[4];
                int nc = 0;
                cuts[nc++] = p.ta;
                if (dx != 0.0) {
                    double tx = (xm - q[0]) / dx;
                    if (tx > p.ta && tx < p.tb) cuts[nc++] = tx;
                }
                if (dy != 0.0) {
                    double ty = (ym - q[1]) / dy;
                    if (ty > p.ta && ty < p.tb) cuts[nc++] = ty;
                }
                cuts[nc++] = p.tb;
                for (int i = 1; i < nc; ++i)   // at most four values: insertion sort
                    for (int k = i; k > 0 && cuts[k] < cuts[k - 1]; --k) std::swap(cuts[k], cuts[k - 1]);
                for (int i = 0; i + 1 < nc; ++i) {
                    double u = cuts[i], v = cuts[i + 1];
                    if (!(v > u)) continue;
                    double tm = 0.5 * (u + v);
                    double px = q[0] + tm * dx, py = q[1] + tm * dy;
                    int qd = (px >= xm ? 1 : 0) + (py >= ym ? 2 : 0);
                    it.kids[qd].push_back({p.seg, u, v});
                }
            }
        };
        const int hw = int(std::max(1u, std::thread::hardware_concurrency()));
        const int nt = std::max(1, std::min({hw, 16, int(items.size())}));
        if (nt <= 1 || items.size() < 4) {
            for (Item &it : items) cut(it);
        } else {
            std::atomic<int> next{0};
            auto run = [&]() {
                for (int i = next++; i < int(items.size()); i = next++) cut(items[i]);
            };
            std::vector<std::thread> pool;
            for (int k = 1; k < nt; ++k) pool.emplace_back(run);
            run();
            for (auto &th : pool) th.join();
        }
        for (Item &it : items) {
            std::vector<Piece> *kids = &nxt[4 * (size_t)split[it.j]];
            for (int q = 0; q < 4; ++q) {
                if (kids[q].empty()) kids[q].swap(it.kids[q]);
                else kids[q].insert(kids[q].end(), it.kids[q].begin(), it.kids[q].end());
            }
        }
        for (int j = 0; j < n_level; ++j)
            if (split[j] >= 0) std::vector<Piece>().swap(cur[j]);
        if (nxt.empty()) break;
        ++lev;
        t.level_start.push_back(next_first);
        first = next_first;
        cur.swap(nxt);
    }
    t.depth = lev;
    t.level_start.push_back(t.n_cells());

    // pieces grouped by leaf (cell order); drop pieces shorter than 1e-12 of
    // their segment (their integrals are below rounding of the whole)
    const int nC = t.n_cells();
    t.piece_start.assign(nC, 0);
    t.piece_count.assign(nC, 0);
    for (int c = 0; c < nC; ++c) {
        if (!t.is_leaf(c)) continue;
        t.piece_start[c] = int(t.pc_seg.size());
        for (const Piece &p : leaf_pieces[c]) {
            if (!(p.tb - p.ta > 1e-12)) continue;
            const double *q = &seg_xy[4 * size_t(p.seg)];
            double dx = q[2] - q[0], dy = q[3] - q[1];
            double ax = (p.ta == 0.0) ? q[0] : q[0] + p.ta * dx;
            double ay = (p.ta == 0.0) ? q[1] : q[1] + p.ta * dy;
            double bx = (p.tb == 1.0) ? q[2] : q[0] + p.tb * dx;
            double by = (p.tb == 1.0) ? q[3] : q[1] + p.tb * dy;
            t.pc_xy.push_back(ax);
            t.pc_xy.push_back(ay);
            t.pc_xy.push_back(bx);
            t.pc_xy.push_back(by);
            t.pc_seg.push_back(p.seg);
        }
        t.piece_count[c] = int(t.pc_seg.size()) - t.piece_start[c];
    }

    quadtree_lists(t);
    return true;
}

void quadtree_lists(Tree &t) {
    const int nC = t.n_cells();
    // colleagues (same level, touching, not self), top-down
    std::vector<std::vector<int>> coll(nC);
    for (int c = 1; c < nC; ++c) {
        int P = t.parent[c];
        auto consider = [&](int Q) {
            if (t.child0[Q] < 0) return;
            for (int q = 0; q < 4; ++q) {
                int D = t.child0[Q] + q;
                if (D != c && touches(t, c, D)) coll[c].push_back(D);
            }
        };
        consider(P);
        for (int Q : coll[P]) consider(Q);
    }

    // list 2
    std::vector<std::vector<int>> V(nC), U(nC), W(nC), X(nC);
    for (int c = 0; c < nC; ++c) {
        if (t.level[c] < 2) continue;
        int P = t.parent[c];
        for (int Q : coll[P]) {
            if (t.child0[Q] < 0) continue;
            for (int q = 0; q < 4; ++q) {
                int D = t.child0[Q] + q;
                if (!touches(t, c, D)) V[c].push_back(D);
            }
        }
    }
    // lists 1 and 3 by descent through the colleagues of each leaf
    for (int b = 0; b < nC; ++b) {
        if (!t.is_leaf(b)) continue;
        U[b].push_back(b);
        std::vector<int> stack(coll[b].begin(), coll[b].end());
        while (!stack.empty()) {
            int C = stack.back();
            stack.pop_back();
            if (t.is_leaf(C)) {
                U[b].push_back(C);
                continue;
            }
            for (int q = 0; q < 4; ++q) {
                int D = t.child0[C] + q;
                if (touches(t, b, D)) stack.push_back(D);
                else W[b].push_back(D);
            }
        }
    }
    // coarser adjacent leaves by symmetry; list 4 as the dual of list 3
    for (int b = 0; b < nC; ++b) {
        if (!t.is_leaf(b)) continue;
        size_t n0 = U[b].size();
        for (size_t i = 0; i < n0; ++i) {
            int d = U[b][i];
            if (t.level[d] > t.level[b]) U[d].push_back(b);
        }
        for (int d : W[b]) X[d].push_back(b);
    }
    for (auto &l : U) std::sort(l.begin(), l.end());
    for (auto &l : X) std::sort(l.begin(), l.end());
    to_csr(U, t.u_ptr, t.u_idx);
    to_csr(V, t.v_ptr, t.v_idx);
    to_csr(W, t.w_ptr, t.w_idx);
    to_csr(X, t.x_ptr, t.x_idx);
}

long long check_quadtree_routes(const Tree &t) {
    const int nC = t.n_cells();
    auto key = [](int a, int b) { return (long long)a * 0x100000000LL + b; };
    std::unordered_set<long long> Us, Vs, Ws, Xs;
    for (int c = 0; c < nC; ++c) {
        for (int i = t.u_ptr[c]; i < t.u_ptr[c + 1]; ++i) Us.insert(key(c, t.u_idx[i]));
        for (int i = t.v_ptr[c]; i < t.v_ptr[c + 1]; ++i) Vs.insert(key(c, t.v_idx[i]));
        for (int i = t.w_ptr[c]; i < t.w_ptr[c + 1]; ++i) Ws.insert(key(c, t.w_idx[i]));
        for (int i = t.x_ptr[c]; i < t.x_ptr[c + 1]; ++i) Xs.insert(key(c, t.x_idx[i]));
    }
    auto chain = [&](int c) {
        std::vector<int> v;
        for (; c >= 0; c = t.parent[c]) v.push_back(c);
        return v;
    };
    long long bad = 0;
    for (int a = 0; a < nC; ++a) {
        if (!t.is_leaf(a)) continue;
        std::vector<int> ca = chain(a);
        for (int b = 0; b < nC; ++b) {
            if (!t.is_leaf(b)) continue;
            std::vector<int> cb = chain(b);
            int cnt = Us.count(key(a, b)) ? 1 : 0;
            for (int A : ca)
                for (int C : cb) cnt += Vs.count(key(A, C)) ? 1 : 0;
            for (int C : cb) cnt += Ws.count(key(a, C)) ? 1 : 0;
            for (int A : ca) cnt += Xs.count(key(A, b)) ? 1 : 0;
            if (cnt != 1) ++bad;
        }
    }
    return bad;
}

}  // namespace dc
