// Non-uniform quadtree over clipped segments (Sec. 5.1-5.2, App. E.3-E.5).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace dc {

struct Tree {
    // Root: lower-left corner (x0, y0) and width w0.  w0 is a power of two
    // and x0, y0 are multiples of w0 / 1024, so every cell boundary
    // x0 + i w0 / 2^l is an exact double (no ambiguity for points on edges).
    double x0 = 0, y0 = 0, w0 = 1;
    int depth = 0;                      // deepest level present
    std::vector<int> level_start;       // cells of level l: [level_start[l], level_start[l+1])
    std::vector<int> level;             // [cells]
    std::vector<int> parent;            // [cells], -1 for the root
    std::vector<int> child0;            // [cells], first of 4 contiguous children or -1 (leaf)
    std::vector<long long> ix, iy;      // integer position on the level's grid
    std::vector<int> piece_start;       // [cells] (leaves own pieces; others 0 / 0)
    std::vector<int> piece_count;
    // Clipped segment pieces, grouped by leaf (Sec. 5.2).
    std::vector<double> pc_xy;          // [pieces][4]
    std::vector<int> pc_seg;            // owning segment
    // Interaction lists (CSR over cells):
    std::vector<int> u_ptr, u_idx;      // list 1 (leaves): adjacent leaves, self included
    std::vector<int> v_ptr, v_idx;      // list 2 (all cells): interaction list
    std::vector<int> w_ptr, w_idx;      // list 3 (leaves): smaller separated list
    std::vector<int> x_ptr, x_idx;      // list 4 (all cells): bigger separated list

    double ms_cut = 0.0, ms_lists = 0.0;   // wall time of the last build's clipping and lists
    int n_cells() const { return int(level.size()); }
    bool is_leaf(int c) const { return child0[c] < 0; }
    double width(int c) const;
    double cx(int c) const;
    double cy(int c) const;
    // Leaf containing (x, y) with half-open cell boxes; -1 outside the root.
    int locate(double x, double y) const;
    int n_leaves() const;
};

// Builds the tree over the segments seg_xy[S][4]; the root covers the
// segments and the rectangle domain[4] = (x0, y0, x1, y1).  A cell splits
// while it holds more than leaf_size pieces and is above max_depth.
bool build_quadtree(const std::vector<double> &seg_xy, const double domain[4], int leaf_size,
                    int max_depth, Tree &t, std::string &err);

// The root box alone (x0, y0, w0 of t), as build_quadtree chooses it.
bool quadtree_root(const std::vector<double> &seg_xy, const double domain[4], Tree &t, std::string &err);

// Lists 1-4 of a tree whose cells and pieces are set.
void quadtree_lists(Tree &t);

// build_quadtree with the clipping of segments into pieces on the device
// (tree_gpu.cu): the same cells, pieces (in the same order, with the same
// IEEE operations) and lists.  seg_dev: the segments [S][4] on the device.
bool build_quadtree_device(const double *seg_dev, const std::vector<double> &seg_xy, const double domain[4],
                           int leaf_size, int max_depth, Tree &t, void *stream, std::string &err);

// Exhaustive check that every (target leaf, source leaf) pair is covered by
// exactly one of the four routes of Alg. 8.  Returns the number of pairs
// covered 0 or >1 times (0 = complete and disjoint).  O(leaves^2 depth^2).
long long check_quadtree_routes(const Tree &t);

}  // namespace dc
