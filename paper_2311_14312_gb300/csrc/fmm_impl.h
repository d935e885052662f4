// Internal state of the FMM forms, shared by the FP64 (fmm.cu) and FP32
// (fmm32.cu) translation units.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "dc_internal.h"
#include "evalnodes.cuh"
#include "fmm.h"
#include "passes.cuh"
#include "tree.h"

namespace dc {

// FP64 view of the tree: absolute coordinates.
struct DevTree {
    const double *cc;       // [nC][2] centres
    const double *cw;       // [nC] widths
    const int *parent, *child0, *quad;
    const int *pstart, *pcount;
    const double *pc;       // [np][4]
    const double *pw;       // [np] arc weight
    const int *pseg;        // [np]
    const int *u_ptr, *u_idx, *v_ptr, *v_idx, *v_off, *w_ptr, *w_idx, *x_ptr, *x_idx;
};

// FP32 view: every coordinate is relative to a cell centre, so FP32 keeps
// the relative accuracy of the local geometry at any zoom of the canvas.
struct DevTree32 {
    const float *iw;        // [nC] 1 / width
    const float *logw;      // [nC] log(width)
    const int *parent, *child0, *quad;
    const int *pstart, *pcount;
    const float4 *pc;       // [np] endpoints minus the own leaf's centre
    const float *pw;        // [np] arc weight
    const float *plen;      // [np] chord length
    const int *pseg;
    const int *u_ptr, *u_idx, *v_ptr, *v_idx, *v_off, *w_ptr, *w_idx, *x_ptr, *x_idx;
    const float2 *u_off;    // per list-1 entry: centre(source) - centre(target)
    const float2 *w_off;    // per list-3 entry
    const float2 *x_off;    // per list-4 entry
    const int *uf_ptr, *uf_idx;   // list-1 pieces of each leaf, flattened (list order)
    const float4 *pch, *pcl;      // [np] endpoints (x1, y1, x2, y2) as FP32 (hi, lo) pairs
};

// A unit of evaluation work inside one leaf: a pixel rectangle (r0, c0,
// nr x nc) or, for target lists, targets [r0, r0 + nr) with nc = 0.
struct Tile {
    int leaf, r0, c0, nr, nc, vp;   // vp: viewport index (pixel tiles)
};

// Pixel tiles of the render: kEvalTile x kEvalTile pixels of one leaf per
// block of the evaluation kernel, one thread per pixel.
#ifndef DC_EVAL_TILE
#define DC_EVAL_TILE 8
#endif
constexpr int kEvalTile = DC_EVAL_TILE;
// pixel tile width x height of the FP32 evaluation kernel for options.eval_tile
inline void tile_shape(int eval_tile, int &w, int &h) {
    static const int W[4] = {8, 16, 16, 32}, H[4] = {8, 8, 16, 8};
    const int k = (eval_tile >= 0 && eval_tile < 4) ? eval_tile : 0;
    w = W[k];
    h = H[k];
}

// Cells that need incoming expansions for one set of targets (all cells for
// pixels; the cells above the nodes for the matvec), by pass.
struct Schedule {
    DevBuf<int> m2l, p2l, l2l;        // cells with list 2 / list 4; cells per level
    std::vector<int> l2l_ptr;         // [depth + 2] offsets into l2l by level
    DevBuf<int> walk;                 // leaves whose incoming expansion is needed
    DevBuf<int> chains;               // per walk leaf: length, then itself and its ancestors to level 2
    int n_m2l = 0, n_p2l = 0, n_walk = 0;
};

// Arbitrary points sorted into the leaves that hold them, on the device
// (aa.cu): leaf of each point by descent from the root, counting sort by
// leaf, work items of at most `item` points of one leaf (Tile for the FP32
// kernel, int4 (leaf, first, count, 0) for the FP64 one).  perm maps sorted
// positions to the caller's order; sxy holds the sorted points.
struct PointSort {
    DevBuf<int> leaf_of, cnt, start, ioff, perm, flag;
    DevBuf<double> sxy;
    DevBuf<Tile> items32;
    DevBuf<int4> items64;
    ScanWork scan;
    cudaError_t run(const double *xy, int n, const int *child0, const double *cc, int n_cells, double x0,
                    double y0, double w0, int item, bool f32, cudaStream_t st, int &n_items, bool &outside);
};

struct Fmm::Impl {
    dc_options opt{};
    int p = 0, P1 = 0;
    bool fp32 = false;
    Tree tree;
    const DevGeom *D = nullptr;
    // FP64 tree
    DevBuf<double> cc, cw, pc, pw;
    DevBuf<int> parent, child0, quad, pstart, pcount, pseg;
    DevBuf<int> u_ptr, u_idx, v_ptr, v_idx, v_off, w_ptr, w_idx, x_ptr, x_idx;
    DevBuf<int> p2m_leaves;
    int n_p2m = 0;
    // node targets sorted by leaf
    DevBuf<int> nt_leaves, nt_start, nt_count, nt_perm, nt_own1, nt_own2;
    DevBuf<double> nt_xy;
    int n_nt_leaves = 0;
    // point targets (eval_points)
    DevBuf<int> pt_leaves, pt_start, pt_count, pt_perm;
    DevBuf<double> pt_xy, pt_out;
    DevBuf<float2> pt_q32;
    DevBuf<Tile> pt_items;
    DevBuf<int4> nt_items4, pt_items4;   // (leaf, first target, count, list-1 pieces) work items
    int n_nt_items4 = 0;
    // near-field coefficients of the node operator (formed once per drawing):
    // single and double layer in FP64, single layer in FP32
    DevBuf<long long> near_off;
    long long near_total = 0;
    bool near_ready = false;
    DevBuf<double> near_g64, near_f64;   // while they are built (near and far both stored: float-float)
    DevBuf<float2> near_gff, near_fff, dens_ff;
    DevBuf<float4> farff, Lff, Mff;
    DevBuf<float> near_g32;
    cudaError_t build_near(cudaStream_t st);
    // far-field coefficients of the node targets: (1 + list-3 length) blocks
    // of P1 (FP64) / P1i (FP32) complex values per target from block far_off[item]
    DevBuf<long long> far_off;
    long long far_blocks = 0;
    bool far_ready = false;
    DevBuf<double2> far64;
    DevBuf<float2> far32;
    void far_coef_launch(cudaStream_t st);
    // stored P2M rows [pieces][P1] and P2L rows [p2l_rows][P1] (G and F parts,
    // FP64; P2M G part at order p_inner in FP32), p2l_off[cell] = first row
    bool rows_ready = false;
    long long p2l_rows = 0;
    DevBuf<long long> p2l_off;
    DevBuf<int> p2l_cnt;          // [cells] rows of the cell's list 4
    DevBuf<int2> p2l_item;        // [p2l_rows] (piece, list-4 entry), row order
    DevBuf<double2> p2m_g64, p2m_f64, p2l_g64, p2l_f64;   // FP64 rows while they are built
    DevBuf<float4> p2m_gff, p2m_fff, p2l_gff, p2l_fff;    // the same rows in float-float
    DevBuf<float2> p2m_g32;
    cudaError_t build_rows(cudaStream_t st);
    // FP64 tables and expansions
    DevBuf<double2> m2m, l2l, m2l, M, L;
    DevBuf<double> sbar, mbar;
    DevBuf<Tile> tiles;               // the render's tiles, by decreasing estimated cost
    DevBuf<int> render_queue;         // the persistent render's tile counter
    DevBuf<VpDev> vps;
    // FP32 form
    DevBuf<float> iw32, logw32, pw32, plen32;
    DevBuf<float4> pc32;
    DevBuf<float4> pch32, pcl32;  // piece endpoints as (hi, lo) float pairs
    DevBuf<float2> uoff32, woff32, xoff32;
    DevBuf<float2> m2m32, l2l32, m2l32, M32, L32;
    DevBuf<float> sbar32, mbar32;
    DevBuf<float2> nt_q32;        // node targets minus their leaf centre
    DevBuf<Tile> nt_items;        // node work items (<= 64 targets each)
    int n_nt_items = 0;
    DevBuf<double> ir_r, ir_d, ir_t;   // refinement residual, correction, scratch
    DevBuf<double> pinv;          // [panels][g][g] inverse self-interaction blocks
    TwoLevel coarse;              // coarse space of panel constants
    cudaError_t precond(const double *v, double *w, cudaStream_t st);
    DevBuf<int> pinfo;
    // pass schedules and tables of the templated passes
    Schedule sched_all, sched_nodes;
    DevBuf<int> m2m_cells, v_code;
    DevBuf<int> uf_ptr, uf_idx, uf_seg;   // list-1 pieces per leaf, flattened, and their segments
    std::vector<int> m2m_ptr;         // [depth + 2]: inner cells with pieces, by level
    // one-launch upward pass of the FP32 operator: chunks (ancestor, first
    // pair, pairs, slot), reductions (cell, first slot, slots), leaves of the
    // pairs, C(k, j)
    DevBuf<int4> mchunks, mred;
    DevBuf<int> pair_leaf;
    DevBuf<float4> pair_geo;          // per pair: shift d (x, y), scale rho
    DevBuf<float> binom32;
    DevBuf<float2> mpart32;
    int n_mchunks = 0, n_mred = 0, n_mslots = 0;
    DevBuf<int> level_d;              // cell levels
    int walk_nmax = 1;                // longest walk chain (levels 2 .. depth)
    DevBuf<double2> base64, Lm2l;
    DevBuf<float4> baseff;            // base M2L tables in float-float
    DevBuf<float4> m2mff, l2lff;      // M2M / L2L tables in float-float
    DevBuf<float2> base32, Lm2l32;
    // the FP32 operator inside GMRES runs at a lower order p_inner (its
    // accuracy only has to beat the inner tolerance; the FP64 residual at
    // order p decides convergence): own tables and expansions
    int P1i = 0;
    DevBuf<float2> m2m32i, l2l32i, base32i, M32i, L32i, Lm2l32i;
    DevBuf<float2> m2lfull32i;        // [56][P1i][P1i] full M2L variants
    // tensor-core M2L of the inner operator (passes_tc.cuh): G_v tiles, the
    // node schedule's list-2 entries grouped by variant, the tiles, the
    // per-entry rows Y and the wait-limit flag
    DevBuf<float> tc_tab, tc_y;
    DevBuf<int> tc_entries, tc_err;
    DevBuf<int4> tc_tiles;
    int n_tc_tiles = 0;
    long long m2l_pairs_nodes = 0;    // list-2 pairs of the node schedule
    DevBuf<float2> lam_ff;            // Lambda [s][g] as (hi, lo) floats
    DevBuf<double> iw64, logw64, plen64;
    DevBuf<unsigned char> heavy;      // per piece: near field evaluated in FP64
    DevBuf<unsigned char> heavyL, heavyM;   // per cell: L2P / M2P evaluated in FP64
    int n_sms = 152;
    passes::TreeView<double> view64() const;
    passes::TreeView<float> view32() const;
    long long p2p_nodes = 0, m2l_cnt = 0, render_pairs = 0, render_m2p = 0;
    double render_flops = 0.0, render_eval_ms = 0.0;
    bool eval_timing = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // the FP32 preconditioned matvec v -> A32 M^-1 v captured as one CUDA
    // graph that reads g_in and writes g_out
    cudaStream_t cap_stream = nullptr;
    // side stream and events of the captured graph's parallel branch (the
    // list-4 P2L beside the M2M / M2L chain)
    cudaStream_t side = nullptr;
    cudaEvent_t fork_ev[2] = {nullptr, nullptr};
    // stream of the preconditioner's build, beside the schedules, and the
    // event it starts from
    cudaStream_t pre_stream = nullptr;
    cudaEvent_t pre_ev = nullptr;
    // stream of the tree build (highest priority)
    cudaStream_t tree_stream = nullptr;
    bool graph_split = true;   // capture the branches in parallel
    bool render_only = false;  // no preconditioner, no node near-field coefficients
    cudaGraph_t g32 = nullptr;
    cudaGraphExec_t g32_exec = nullptr;
    int g32_kernels = 0;
    DevBuf<double> g_in, g_out;
    DevBuf<double> agg_py, agg_gpy;   // the aggregated coarse level's P y and G_H P y
    double build_ms[6] = {0, 0, 0, 0, 0, 0};   // wall time of the build phases
    // the render's tile plan (tiles, vps) for the viewports plan_vps
    bool plan_valid = false;
    std::vector<VpDev> plan_vps;
    int plan_tiles = 0, plan_tile = 0;
    long long plan_pairs = 0, plan_m2p = 0;
    double plan_flops = 0.0;
    cudaError_t graph_matvec32(const double *x, double *y, cudaStream_t st);
    cudaError_t graph_ensure();
    cudaError_t graph_launch(cudaStream_t st);
    ~Impl() {
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        if (g32_exec) cudaGraphExecDestroy(g32_exec);
        if (g32) cudaGraphDestroy(g32);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        if (side) cudaStreamDestroy(side);
        if (pre_stream) cudaStreamDestroy(pre_stream);
        if (tree_stream) cudaStreamDestroy(tree_stream);
        if (pre_ev) cudaEventDestroy(pre_ev);
        for (auto &ev : fork_ev)
            if (ev) cudaEventDestroy(ev);
    }

    DevTree dt() const;
    DevTree32 dt32() const;
    // FP64 passes / node operator (fmm.cu)
    cudaError_t passes(const double *sb, const double *mb, int use_s, int use_m, cudaStream_t st,
                       const Schedule &sc);
    cudaError_t apply_nodes(const double *x, double *y, bool single, cudaStream_t st);
    // FP32 (fmm32.cu)
    // host arrays of the FP32 form that depend on the (pruned) tree and the
    // discretisation alone: built on a helper thread during the schedules
    struct Prep32 {
        std::vector<float> iw, logw;
        std::vector<double> ccx, ccy;
        std::vector<float4> pcf, pch, pcl;
        std::vector<float> pwf, plf;
        std::vector<float2> uo, wo, xo;
    };
    static void prep32(const Tree &T, const Geometry &G, Prep32 &out);
    // txy, start, cnt: the node targets sorted by leaf and each leaf's range
    dc_status build32(const Geometry &G, const Prep32 &pr, const std::vector<double> &txy,
                      const std::vector<int> &start, const std::vector<int> &cnt, cudaStream_t st,
                      std::string &err);
    cudaError_t passes32(const float *sb, const float *mb, int use_s, int use_m, cudaStream_t st,
                         const Schedule &sc);
    // render preparation of the FP32 form: FP64 passes, FP32 copies of the
    // expansions, heavy-piece flags from the FP64 segment densities
    cudaError_t prepare_render32(const double *sb, const double *mb, cudaStream_t st);
    cudaError_t check_tc_wait(cudaStream_t st, std::string &err);
    cudaError_t launch_m2l32(const Schedule &sc, int part, cudaStream_t st);
    cudaError_t time_inner_m2l(int reps, cudaStream_t st, double out[6]);
    cudaError_t apply_nodes32(const double *x, double *y, bool single, cudaStream_t st);
    cudaError_t interp32(const double *node_vals, float *seg_vals, cudaStream_t st);
    // the FP32 operator at the nodes from segment values already in
    // sbar32 (single) or mbar32
    cudaError_t nodes32_from_segments(double *y, bool single, cudaStream_t st);
    // the single layer of the inner operator with the list-4 P2L as a branch
    // beside P2M -> M2M -> M2L; fork: the branch on side (while capturing
    // the graph), else everything on st in the same order
    bool split_ok() const;
    cudaError_t nodes32_split(double *y, cudaStream_t st, bool fork);
    evalnodes::NodeArgs<float> node_args32(double *y, bool single) const;
    cudaError_t render_tiles32(int n_tiles, void *rgb, int rgb_dtype,
                               unsigned char *rgb8, const double *sb64, const double *mb64,
                               cudaStream_t st);
    cudaError_t eval_points32(int n_items, double *out, const double *sb64, const double *mb64,
                              cudaStream_t st);
    cudaError_t eval_points32_at(const Tile *items, int n_items, const double *q64, const int *perm,
                                 double *out, const double *sb64, const double *mb64, cudaStream_t st);
    PointSort psort;
    evalnodes::NodeArgs<double> node_args64(const int4 *items, const double *q64, const int *own1,
                                            const int *own2, const int *perm, const double *sb,
                                            const double *mb, int use_s, int use_m, double *out) const;
    cudaError_t eval_list64(const int4 *items, int n_items, const double *q64, const int *own1,
                            const int *own2, const int *perm, const double *sb, const double *mb,
                            int use_s, int use_m, double *out, cudaStream_t st);
    cudaError_t to_f32_density(const double *sb, const double *mb, cudaStream_t st);
};

}  // namespace dc
