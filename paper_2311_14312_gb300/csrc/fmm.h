// FMM forms of the layer-potential operator (App. E, Alg. 8) on a
// non-uniform quadtree with clipped segments (Sec. 5.2).
#pragma once

#include <memory>
#include <string>

#include "dc_internal.h"

namespace dc {

class Fmm {
public:
    Fmm();
    ~Fmm();
    // quadtree(S) and pre_FMM(S, q, Q) (Alg. 3).
    dc_status build(const dc_options &opt, const Geometry &G, const DevGeom &D,
                    cudaStream_t st, std::string &err);
    // y = G_H x at the nodes (single layer of the interpolated density).
    cudaError_t apply_single_layer(const double *x, double *y, cudaStream_t st);
    // y = F_H x at the nodes (double layer), for the right-hand side.
    cudaError_t apply_double_layer(const double *x, double *y, cudaStream_t st);
    // The FP32 inner operator of the iterative refinement: y = G_H M x
    // (order p_inner, two-level preconditioner M), through the captured
    // graph.  cudaErrorNotSupported for the FP64 form.
    cudaError_t apply_inner(const double *x, double *y, cudaStream_t st);
    // The preconditioner alone, y = M x.
    cudaError_t apply_precond(const double *x, double *y, cudaStream_t st);
    // The FP32 operator without the preconditioner, y = G_H x.
    cudaError_t apply_inner_raw(const double *x, double *y, cudaStream_t st);
    // Test hook of the tensor-core M2L: the CTA that takes `tile` issues no
    // MMA for it, so its bounded wait runs out (-1 = off).
    cudaError_t set_mma_skip_tile(int tile, cudaStream_t st);
    void set_eval_tile(int t);   // pixel tile shape of the FP32 render (options.eval_tile)
    // A render-only build (a viewport's evaluation polyline) skips the
    // solve's structures: the two-level preconditioner and the node
    // near-field coefficients.  Set before build().
    void set_render_only(bool on);
    // The tree built on the device against build_quadtree on the host over
    // the same segments: out[0] 1 when cells, piece counts, piece segments
    // and lists 1-4 are identical, out[1] the largest piece-endpoint difference, out[2]
    // cells, out[3] pieces, out[4] / out[5] wall ms of the device build's
    // clipping and lists.
    void compare_host_tree(const Geometry &G, double out[6]) const;
    // y = B x with B the panels' inverse self-interaction blocks of G_H (the
    // first level of the two-level preconditioner alone).
    cudaError_t apply_block_jacobi(const double *x, double *y, cudaStream_t st);
    // Device time of the inner operator's M2L kernels (fmm32.cu).
    cudaError_t time_inner_m2l(int reps, cudaStream_t st, double out[6]);
    // GMRES with this operator (Alg. 3); x holds x0 on entry.
    // n_refine: outer refinement steps taken.  Ax0: G_H x0 when the caller
    // has it (the first residual then needs no operator application), else
    // nullptr.
    cudaError_t solve(GmresWork *w, const double *b, double *x, const dc_options &opt,
                      cudaStream_t st, GmresResult &res, std::string &err, int *n_refine = nullptr,
                      const double *Ax0 = nullptr);
    // Forms the expansions of segment densities sbar and mbar (Alg. 8 up and
    // down passes); render_grid / eval_points then evaluate them.
    cudaError_t prepare_eval(const double *sbar, const double *mbar, cudaStream_t st);
    // Single + double layer of segment densities at the pixels of n
    // viewports in one launch; rgb / rgb8 are the outputs of the whole call
    // and each viewport writes from its VpDev::offset.
    dc_status render_viewports(const VpDev *vps, int n, const double *sbar, const double *mbar,
                               void *rgb, int rgb_dtype, unsigned char *rgb8, cudaStream_t st,
                               std::string &err);
    dc_status eval_points(const double *xy, int n, const double *sbar, const double *mbar,
                          void *out, int out_dtype, cudaStream_t st, std::string &err);
    // The same at device points xy [n][2], FP64 output out [n][3], with the
    // points located and sorted by leaf on the device (no host round trip);
    // after prepare_eval.
    dc_status eval_points_dev(const double *xy, int n, const double *sbar, const double *mbar, double *out,
                              cudaStream_t st, std::string &err);
    void fill_sizes(dc_sizes *out) const;
    // wall ms of the build phases: tree and lists, schedules and uploads,
    // preconditioner, stored P2M / P2L rows, near / far coefficients, FP32 form
    void build_timings(double out[6]) const;
    // two-level preconditioner: ready, panels, near pairs, inverse check
    void precond_info(double out[5]) const;
    long long p2p_pairs_nodes() const;
    long long m2l_pairs() const;
    long long last_render_p2p_pairs() const;
    long long last_render_m2p_pairs() const;
    double last_render_eval_flops() const;
    // When on, render_viewports times its evaluation kernel with CUDA events on
    // the launching stream (synchronising after each launch).
    void set_eval_timing(bool on);
    double last_render_eval_ms() const;

    struct Impl;

private:
    std::unique_ptr<Impl> impl_;
};

}  // namespace dc
