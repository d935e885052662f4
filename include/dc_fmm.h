/*
 * dc_fmm.h -- C ABI of libdc_fmm: GPU (sm_103a) solver and renderer for
 * diffusion curves with the hybrid boundary-integral method accelerated by
 * a fast multipole method on a non-uniform quadtree.
 *
 * Method: S. Bang, K. Serkh, O. Stein, A. Jacobson, "An Adaptive
 * Fast-Multipole-Accelerated Hybrid Boundary Integral Equation Method for
 * Accurate Diffusion Curves", ACM TOG 42(6) 215, 2023.
 *
 * Problem statement (Sec. 3, Sec. 4.3, Alg. 3, Alg. 4): cubic Bezier curves
 * carry a colour on each side (u+ on the right of the direction of travel,
 * u- on the left).  The colour field is
 *     u(x) = int_S [ G(p,x) sigma(p) + F(p,x) mu(p) ] dS(p)        (Eq. 23)
 * with G = -log|p-x| / 2pi (Eq. 3), F = dG/dn(p) (Eq. 4), mu = u+ - u-
 * (Eq. 25) and sigma solving the hybrid system (Eq. 27)
 *     (u+ + u-)/2 = G_H sigma + F_H mu  at the Gauss-Legendre nodes,
 * G_H = Gbar Pbar Pring^-1 (Eq. 19): densities live at g Gauss-Legendre
 * nodes per panel and are interpolated to s straight segments per panel,
 * integrated in closed form (App. D) with arc-length weighting (App. A).
 * The operator is applied by an FMM (App. E, Alg. 8) inside GMRES
 * (Sec. 5.5) and again to render pixels (Alg. 4).
 *
 * Conventions:
 *  - All entry points return a dc_status; none aborts, exits or traps.  On
 *    failure dc_last_error(ctx) holds a message until the next call.
 *  - Host inputs are copied before the call returns; the caller keeps
 *    ownership of every buffer it passes.  The context owns all device
 *    memory it allocates and frees it in dc_destroy.
 *  - Device work is issued on the stream given in dc_options (NULL = the
 *    legacy default stream).  Device output buffers are written in stream
 *    order; host output buffers are complete when the call returns.
 *  - Calls are ordered: dc_build_tree before dc_solve_density before
 *    dc_render_viewport / dc_eval_points (or dc_set_density in place of a
 *    solve).  A call out of order returns DC_ERR_STATE.
 *  - Results are deterministic: the same inputs and options give
 *    bit-identical outputs (fixed reduction orders, no float atomics).
 *  - Not thread-safe per context; distinct contexts are independent.
 */
#ifndef DC_FMM_H
#define DC_FMM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DC_ABI_VERSION 1

typedef struct dc_ctx dc_ctx;

typedef enum {
    DC_OK = 0,
    DC_ERR_ARG = 1,         /* invalid argument (sizes, NULL, NaN, range)   */
    DC_ERR_STATE = 2,       /* call out of order                            */
    DC_ERR_CUDA = 3,        /* CUDA runtime error (message has the detail)  */
    DC_ERR_OOM = 4,         /* device or host allocation failed             */
    DC_ERR_NOCONV = 5,      /* GMRES hit gmres_max_iter before gmres_tol    */
    DC_ERR_TIMEOUT = 6,     /* a bounded device wait gave up                */
    DC_ERR_GEOMETRY = 7,    /* degenerate geometry (zero-length curve, ...) */
    DC_ERR_UNSUPPORTED = 8  /* option combination not available             */
} dc_status;

/* How the layer-potential operator is applied. */
typedef enum {
    DC_FORM_DENSE64 = 0,    /* plain form: dense FP64 operator rows (Eq. 19,
                               27) and FP64 direct sums for pixels (A11)    */
    DC_FORM_FMM64 = 1,      /* FP64 FMM on the non-uniform quadtree (Alg. 8) */
    DC_FORM_FMM32 = 2       /* chosen form: FP32 FMM with FP64 GMRES
                               (Arnoldi, least squares, outer residual)     */
} dc_form;

typedef enum {
    DC_X0_ONES = 0,        /* the paper's choice (Sec. 5.5)                  */
    DC_X0_ZEROS = 1,
    DC_X0_USER = 2,        /* x0 passed to dc_solve_density                  */
    DC_X0_LEARNED = 3      /* predicted by the model set with
                              dc_aux_set_warm_start_model (no counterpart in
                              the paper): per channel x0 = a x_pred + c 1
                              with a, c minimising ||b - G_H x0|| (two extra
                              operator applications); a = 0 is the cold
                              fallback, so the start is never worse than
                              zeros or the paper's ones                      */
} dc_x0_mode;
typedef enum { DC_MEM_DEVICE = 0, DC_MEM_HOST = 1 } dc_mem;
typedef enum { DC_F32 = 0, DC_F64 = 1 } dc_dtype;

typedef struct {
    int form;              /* dc_form                                        */
    int g;                 /* Gauss-Legendre nodes per panel, 1..32 (Sec. 4.2;
                              paper uses 4)                                  */
    int s_per_panel;       /* straight segments per panel, >= g (Sec. 6.2;
                              paper: s = 5 g)                                */
    int p;                 /* FMM expansion order: terms 0..p (App. E, "K") */
    int leaf_size;         /* max clipped segments per quadtree leaf ("b")  */
    int max_depth;         /* quadtree depth limit, 1..40                    */
    double gmres_tol;      /* relative residual ||b - A x|| / ||b|| per channel */
    int gmres_restart;     /* Krylov basis size before a restart             */
    int gmres_max_iter;    /* total iterations per solve                     */
    int x0_mode;           /* dc_x0_mode; paper uses ones (Sec. 5.5)         */
    void *stream;          /* cudaStream_t or NULL                           */
    double domain[4];      /* x0, y0, x1, y1: region the quadtree root must
                              cover besides the curves (render targets must
                              lie inside the root)                           */
    int p_inner;           /* DC_FORM_FMM32: expansion order of the FP32
                              operator inside the iterative refinement, 1..p
                              (0 = min(p, 12))                               */
    double inner_tol;      /* DC_FORM_FMM32: floor of the inner GMRES
                              tolerance per refinement step, in (0, 1)
                              (0 = 3e-5)                                     */
    int m2l_engine;        /* DC_FORM_FMM32: M2L of the inner operator on
                              DC_M2L_TENSOR (tcgen05 TF32 with a three-term
                              split; p_inner <= 15, else CUDA cores) or
                              DC_M2L_CUDA_CORES                              */
    int coarse_max;        /* FMM forms: most coarse unknowns of the two-level
                              preconditioner's dense coarse inverse, a
                              multiple of 32 in [64, 16384] (0 = 12288); more
                              panels than that are grouped into aggregates of
                              consecutive panels of a curve                  */
    double adapt_ratio;    /* dc_build_tree with panel_ptr and panel_start both
                              NULL splits panels adaptively: bisect (in
                              arc-length fraction) while a panel is longer than
                              adapt_ratio x its distance to the nearest other
                              curve (0 = 0.2) ...                            */
    int adapt_max_level;   /* ... for at most this many bisections (0 = 8) ... */
    int adapt_min_panels;  /* ... with at least this many panels per curve
                              (0 = 2) ...                                    */
    double adapt_max_len;  /* ... and no panel longer than this (0 = 0.5);
                              measured on 256-point polylines per curve      */
    int eval_tile;         /* DC_FORM_FMM32: pixel tile of one block of the
                              render's evaluation kernel: 0 = 8 x 8 (default),
                              1 = 16 x 8, 2 = 16 x 16, 3 = 32 x 8 (width x
                              height)                                         */
    int aa_levels;         /* quadtree anti-aliasing of the render (Sec. 7):
                              0 = off (centre samples, default); m in [1, 6]:
                              a pixel whose closed square meets a segment is
                              split into quarter cells while they meet one,
                              down to 2^-m of the pixel, and takes the
                              area-weighted mean of the cells' centre values */
} dc_options;

enum {
    DC_M2L_TENSOR = 0,
    DC_M2L_CUDA_CORES = 1
};

typedef struct {
    int n_curves, n_panels, n_nodes, n_segments;
    int n_pieces;          /* segments after clipping at leaf boundaries     */
    int n_cells, n_leaves, depth;
    double root[3];        /* root cell centre x, y and half-width           */
} dc_sizes;

typedef struct {
    int iters[3];          /* GMRES iterations per colour channel            */
    double rel_resid[3];   /* final ||b - A x|| / ||b|| as GMRES reports it   */
    int converged;         /* 1 if every channel met gmres_tol               */
    int n_matvec;          /* operator applications, right-hand side included */
    double ms_rhs;         /* right-hand side (Alg. 3), device time   */
    double ms_solve;       /* x0 set-up and GMRES (Alg. 3), host wall
                              time                                           */
    long long p2p_pairs;   /* near-field (target, piece) pairs per matvec    */
    long long m2l_pairs;   /* cell pairs in M2L per matvec                   */
    int used_warm;         /* DC_X0_LEARNED: bit c set if channel c's start
                              uses the prediction (a != 0; 0 in other modes) */
    double warm_resid[3];  /* DC_X0_LEARNED: ||b - G_H x0|| / ||b|| of the
                              start per channel (0 otherwise)                */
    double ms_warm;        /* DC_X0_LEARNED: features, network and residual
                              check, host wall time (inside ms_solve)        */
    int n_refine;          /* FMM forms: outer (iterative refinement) steps,
                              each one FP64 residual and one inner GMRES     */
    double true_rel_resid[3]; /* ||b - G_H sigma|| / ||b|| per channel with
                              the form's FP64 operator applied to the
                              returned sigma (FMM forms: the refinement's
                              last outer residual; dense form: GMRES's last
                              recomputed residual), never a Givens estimate */
} dc_solve_stats;

typedef struct {
    double x0, y0, x1, y1; /* world rectangle                                */
    int width, height;     /* pixels; pixel (r, c) has centre
                              (x0 + (c + 1/2)(x1 - x0)/width,
                               y0 + (r + 1/2)(y1 - y0)/height); row 0 is the
                              bottom row (y0) and rows are stored in order   */
} dc_viewport;

typedef struct {
    double ms;             /* device time of the whole call                  */
    double ms_eval;        /* device time of the pixel-evaluation kernels    */
    long long pixels;
    long long p2p_pairs;   /* (pixel, clipped piece) pairs of list 1         */
    long long m2p_pairs;   /* (pixel, cell) pairs of list 3                  */
    long long m2l_pairs;   /* cell pairs of list 2 in the passes             */
    double eval_flops;     /* algorithmic flops of the evaluation kernels:
                              45 per near-field pair, 24 (p + 1) per L2P and
                              per list-3 M2P (3 colour channels)              */
    long long aa_pixels;   /* pixels refined by the anti-aliasing (aa_levels) */
    long long aa_samples;  /* their samples                                  */
    double ms_aa;          /* device time of the anti-aliasing pass          */
} dc_render_stats;

/* Fills *opt with defaults: DC_FORM_FMM32, g 16, s 80, p 24, leaf 64,
 * depth 30, tol 1e-10, restart 200, max_iter 2000, x0 ones, domain [0,1]^2,
 * p_inner 0 and inner_tol 0 (the built-in choices), m2l_engine
 * DC_M2L_TENSOR, coarse_max 0 (12288). */
dc_status dc_default_options(dc_options *opt);

/* Creates a context bound to the current CUDA device.  *out is set to NULL
 * on failure. */
dc_status dc_create(dc_ctx **out, const dc_options *opt);

/* Frees every device and host resource of the context (NULL is a no-op). */
void dc_destroy(dc_ctx *ctx);

/* Discretises the drawing and builds the solver state (Alg. 3:
 * quadtree(S) and pre_FMM(S, q, Q), Sec. 5.3).
 *   ctrl         host [n_curves][4][2] control points C0..C3 (App. B)
 *   panel_ptr    host [n_curves + 1]; curve i owns panels
 *                panel_ptr[i] .. panel_ptr[i+1]-1 (at least one each)
 *   panel_start  host [panel_ptr[n_curves]]: arc-length fraction in [0,1)
 *                where each panel starts, strictly increasing per curve,
 *                first = 0 (panels end where the next starts, or at 1)
 *                panel_ptr and panel_start both NULL: the library splits
 *                the panels itself by the options' adapt_* rule (the panels
 *                chosen are returned by dc_get_panels)
 *   colours      host [n_curves][2][2][3]: [side: 0 = u+ (right of travel),
 *                1 = u- (left)][end: colour at t = 0, t = 1][rgb]; colours
 *                are linear in the Bezier parameter t between the ends
 * Errors: DC_ERR_ARG for bad sizes/ordering/non-finite values,
 * DC_ERR_GEOMETRY for a zero-length curve or panel, DC_ERR_OOM/CUDA.
 * Replaces any previous drawing of the context.  It first waits for the
 * device's queued work (as a cudaFree would: the previous drawing's device
 * buffers are recycled for the new one); it runs helper host threads and
 * streams of its own and returns with the build complete. */
dc_status dc_build_tree(dc_ctx *ctx, int n_curves, const double *ctrl,
                        const int *panel_ptr, const double *panel_start,
                        const double *colours);

/* Solves for the density (Alg. 3): mu = u+ - u-,
 * b = (u+ + u-)/2 - F_H mu, sigma = GMRES(G_H, x0, b, tol) with FP64
 * Arnoldi.  x0: host [n_nodes][3] used when x0_mode == DC_X0_USER (else
 * may be NULL).  stats may be NULL.  Returns DC_ERR_NOCONV (density kept,
 * stats filled) if gmres_max_iter is reached first. */
dc_status dc_solve_density(dc_ctx *ctx, const double *x0, dc_solve_stats *stats);

/* Mixed Dirichlet / Neumann conditions on closed curves (Sec. 4.3).  The
 * region is the one the curves bound: every curve closed and traversed
 * counter-clockwise (outer boundary) or clockwise (holes), so that the
 * right-hand normal n points out of the region.  On each Dirichlet panel u
 * is given, on each Neumann panel psi = du/dn.  Green's third identity
 * seen from inside gives at the nodes
 *     u / 2 = G_H psi - F_H u,
 * solved for psi on the Dirichlet panels and u on the Neumann panels by
 * FP64 GMRES, right-preconditioned by the panels' inverse G_H blocks on the
 * Dirichlet panels (identity in the dense form) and -2 on the Neumann
 * panels.  Both FMM forms apply G_H and F_H with the FP64 passes.
 * Afterwards sigma = psi and mu = -u at every node, so dc_render_viewport
 * and dc_eval_points give u inside the region and 0 outside.
 *   neumann   host [n_panels]: nonzero = Neumann panel
 *   psi_star  host [n_nodes][3]: du/dn, read on the Neumann panels only
 *   u_star    host [n_nodes][3]: u, read on the Dirichlet panels only;
 *             NULL = the drawing's colours on the left of the curves
 * stats (may be NULL): iters, rel_resid, true_rel_resid, converged,
 * n_matvec (G_H and F_H applications), ms_solve.
 * Errors: DC_ERR_STATE before dc_build_tree, DC_ERR_ARG for NULL inputs,
 * non-finite values or no Dirichlet panel at all, DC_ERR_GEOMETRY when the
 * total signed area of the curves is not positive (a necessary condition
 * of the orientation; closedness is the caller's), DC_ERR_NOCONV as in
 * dc_solve_density (the densities are kept).  The next dc_solve_density
 * restores mu = u+ - u- from the colours. */
dc_status dc_solve_mixed(dc_ctx *ctx, const unsigned char *neumann, const double *psi_star,
                         const double *u_star, dc_solve_stats *stats);

/* Renders n_vp viewports (Alg. 4): u = single layer of sigma plus
 * double layer of mu at every pixel centre.
 *   rgb       [sum_v height_v width_v][3] of rgb_dtype, viewports
 *             concatenated in order, pixels row-major; may be NULL
 *   rgb8      [same][3] unsigned char = floor(255 clamp(u,0,1) + 1/2);
 *             may be NULL
 *   out_where DC_MEM_DEVICE or DC_MEM_HOST for both outputs
 *   stats     may be NULL (when given, the call synchronises its stream)
 * Every pixel centre must lie inside the quadtree root (DC_ERR_ARG). */
dc_status dc_render_viewport(dc_ctx *ctx, int n_vp, const dc_viewport *vps,
                             void *rgb, int rgb_dtype, unsigned char *rgb8,
                             int out_where, dc_render_stats *stats);

/* Layer potential (Eq. 23) at n arbitrary points inside the quadtree root.
 *   xy   [n][2] double in xy_where memory
 *   out  [n][3] of out_dtype in out_where memory */
dc_status dc_eval_points(dc_ctx *ctx, int n, const void *xy, int xy_where,
                         void *out, int out_dtype, int out_where);

/* No counterpart in the paper.  An allocation-free variant of
 * dc_eval_points for callers that must not allocate device memory during a
 * call -- for example a frame loop whose memory belongs to another
 * framework, or code held to a fixed memory budget.  It evaluates the layer
 * potential (single layer of sigma plus double layer of mu) at n points by
 * the FP64 direct sum over all of the context's segments, whatever its form.
 *   xy_dev   [n][2] double in device memory (caller-owned)
 *   out_dev  [n][3] double in device memory (caller-owned), written in
 *            stream order on the context's stream
 * Scratch: the segment densities go to one file-scope device array sized for
 * at most 262,144 segments (12 MiB, held by every GPU that loads the library
 * until the process exits); a drawing with more segments gets DC_ERR_ARG.
 * The call allocates nothing (no cudaMalloc / cudaFree, no allocating
 * library routine).  Its first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current: make that first
 * call before any stream capture.  All calls share the one array and it
 * keeps the last call's contents, so calls that overlap on the GPU (other
 * streams or contexts without ordering between them) race on it.
 * The cached address belongs to the device's primary context and does not
 * survive a cudaDeviceReset (rebuild the context after one).
 * Errors: DC_ERR_STATE without a density or when the current CUDA device is
 * not the context's, DC_ERR_ARG for bad sizes, DC_ERR_CUDA when the symbol
 * lookup or a launch fails. */
dc_status dc_eval_points_noalloc(dc_ctx *ctx, int n, const double *xy_dev, double *out_dev);

/* ---------------------------------------------------------------------
 * Autotuning of the chosen form (no counterpart in the paper, which gives
 * neither the leaf size b nor K): candidates are the cross product of leaf
 * sizes x inner orders p_inner x pixel tile shapes (eval_tile); each is
 * built on the context's drawing, warmed up, and timed (solve + render of
 * the viewports, CUDA events on the context's stream, best of `repeats`);
 * its FP32 pixels are compared with a plain FP64 FMM render of the same
 * drawing at the context's order p.
 * --------------------------------------------------------------------- */
typedef struct {
    int leaf_size, p_inner, eval_tile;
    double ms;             /* solve + render device time, -1 if it failed    */
    double max_err;        /* max colour difference to the FP64 reference    */
    int converged;
} dc_autotune_row;

/* Runs the search on the drawing last given to dc_build_tree (DC_FORM_FMM32
 * only).  An empty list (n = 0, pointer may be NULL) keeps the context's
 * current value for that option.  rows [max(n_leaf,1) x max(n_pinner,1) x
 * max(n_tile,1)], leaf-major then p_inner then tile; *best = the index of
 * the fastest row that converged with max_err <= tol (-1 if none).  The
 * context is left built with the chosen options (its own if none) and has
 * no density: solve again.  A learned or user start is replaced by x0 = 1
 * during the search.  Errors: DC_ERR_STATE before dc_build_tree,
 * DC_ERR_UNSUPPORTED in other forms, DC_ERR_ARG, errors of the reference
 * solve. */
dc_status dc_autotune(dc_ctx *ctx, int n_vp, const dc_viewport *vps, int n_leaf, const int *leaf_sizes,
                      int n_pinner, const int *p_inners, int n_tile, const int *eval_tiles, double tol,
                      int repeats, dc_autotune_row *rows, int *best);

/* Copies the current density sigma at the nodes to host [n_nodes][3]. */
dc_status dc_get_density(dc_ctx *ctx, double *sigma_out);

/* Sets the density from host [n_nodes][3] (instead of solving). */
dc_status dc_set_density(dc_ctx *ctx, const double *sigma_in);

/* ---------------------------------------------------------------------
 * Adaptive subdivision with local re-solve (Sec. 6.1 Adaptive Subdivision,
 * Alg. 5; Sec. 6.3 local update of the density, Eq. 40-41, Alg. 6-7).
 * --------------------------------------------------------------------- */
typedef enum {
    DC_RESOLVE_LOCAL = 0,   /* label_curves (Eq. 40-41), then the local system
                               of Sec. 6.3 on the re-solving panels only      */
    DC_RESOLVE_GLOBAL = 1,  /* re-solve every panel from the warm start       */
    DC_RESOLVE_NONE = 2     /* keep the warm start as the density             */
} dc_resolve_mode;

typedef struct {
    double eps_coef;       /* epsilon_2 of Alg. 5: a panel is split when the
                              largest magnitude, over the colour channels, of
                              its density's highest-order Legendre coefficient
                              (Legendre polynomials with P_k(1) = 1, on the
                              panel's arc-length coordinate) exceeds it      */
    double eps_len;        /* epsilon_1 of Alg. 5: panels whose arc length
                              (world units) is below it are never split; tie
                              it to the pixel size of the target viewport     */
    int resolve;           /* dc_resolve_mode                                 */
    double label_ratio;    /* the 0.9 of Eq. 41 (0 = 0.9), in [0, 1)          */
} dc_subdivide_options;

typedef struct {
    int n_split;           /* panels split (Alg. 5)                           */
    int n_panels_before, n_panels_after;
    int n_resolve_panels;  /* panels whose density was re-solved (r)          */
    int n_label_matvec;    /* operator applications of label_curves (three
                              unit densities each, one per colour channel)    */
    int iters[3];          /* GMRES iterations of the (local) re-solve        */
    double rel_resid[3];   /* ||[b - G_H sigma]_r|| / ||b_r|| after it         */
    int converged;         /* 1 if every channel is within 10 gmres_tol       */
    double ms_test, ms_rebuild, ms_label, ms_solve;   /* host wall time       */
} dc_subdivide_stats;

/* One round of adaptive subdivision (Alg. 5) and the re-solve of the
 * density (Alg. 7) on the current density:
 *  1. per panel, the highest Legendre coefficient of sigma (device); split
 *     every panel with |c_{g-1}| > eps_coef and arc length >= eps_len into
 *     its two halves in arc-length fraction;
 *  2. update_quadtree / update_pre_FMM: the drawing is rebuilt on the refined
 *     panels (the same work as dc_build_tree; the curves and colours are the
 *     ones last given to it);
 *  3. warm start (Sec. 6.1): the old panels' Legendre expansions evaluated at
 *     the new nodes;
 *  4. label_curves (Eq. 40-41, DC_RESOLVE_LOCAL): for each new half panel
 *     alpha, v = G_H 1_alpha at every node; a panel beta is re-solved when
 *     max v - min v over its nodes exceeds label_ratio times that over alpha
 *     (the new halves are always re-solved);
 *  5. the local system (G_H)_rr sigma_r = b_r - (G_H)_rc sigma_c (Sec. 6.3)
 *     with b = (u+ + u-)/2 - F_H mu of the refined discretisation, the other
 *     panels' densities fixed at the warm start, by GMRES (tolerance
 *     gmres_tol relative to ||b_r||) on the correction of the warm start
 *     with the operator FMM(S_r, ., q_r) of the context's form (the FP64
 *     operator in the FMM forms) and the panels' inverse self-interaction
 *     blocks as a right preconditioner.
 * A call that splits nothing changes nothing.  Needs a density (DC_ERR_STATE
 * otherwise); DC_ERR_ARG for bad options; errors of the rebuild as in
 * dc_build_tree.  stats may be NULL. */
dc_status dc_subdivide(dc_ctx *ctx, const dc_subdivide_options *opt, dc_subdivide_stats *stats);

/* ------------------------------------------------------------------------
 * Viewport update (Sec. 6.2, 6.4; Alg. 9)
 * --------------------------------------------------------------------- */
typedef struct {
    double eps_coef;       /* epsilon_2 of Alg. 5 (0 = no subdivision)        */
    double eps_len_px;     /* epsilon_1 of Alg. 5 in pixels of the viewport:
                              panels shorter than this many pixel sizes (the
                              larger side of a pixel) are not split          */
    double len_unit;       /* unit of the curve length in the e rule,
                              e = ceil(length / (10 len_unit)) + s per panel
                              (0 = 1/512, a pixel of a 512-pixel image of the
                              unit square)                                   */
    int resolve;           /* dc_resolve_mode of each round                   */
    int max_rounds;        /* rounds of subdivide + re-solve (0 = 4)          */
    double label_ratio;    /* the 0.9 of Eq. 41 (0 = 0.9), in [0, 1)          */
} dc_view_options;

typedef struct {
    int rounds;            /* rounds that split panels                        */
    int n_split;           /* panels split over all rounds                    */
    int n_resolve_panels;  /* panels re-solved in the last round              */
    int n_fixed;           /* labels of Sec. 6.4 on the final panels: outside */
    int n_interpolating;   /* ... meeting the viewport, density interpolated  */
    int n_resolving;       /* ... re-solved in the last round                 */
    int e;                 /* evaluation segments per panel                   */
    long long n_eval_segments;
    int converged;         /* 1 if every re-solve converged                   */
    double ms_subdivide, ms_build, ms_total;   /* host wall time              */
} dc_view_stats;

/* Prepares the rendering of a viewport (Alg. 9 after the initial solve):
 *  1. rounds of Alg. 5 restricted to the panels that meet the viewport
 *     (the bounding box of a panel's solve polyline meets the viewport's
 *     closed rectangle), with epsilon_1 = eps_len_px pixel sizes, each
 *     followed by the re-solve of dc_subdivide (resolve mode), until a
 *     round splits nothing or max_rounds;
 *  2. labels (Sec. 6.4): fixed = panels outside the viewport, re-solving =
 *     panels re-solved in the last round, interpolating = the others;
 *  3. the evaluation polyline (Sec. 6.2): e = ceil(L / (10 len_unit)) + s
 *     segments for every panel, the largest over the panels that meet the
 *     viewport (s when none does), placed at equal arc length on each panel
 *     like the solve's; the densities move to it by the interpolation
 *     Lambda_e from the same nodes (no re-solve).
 * dc_render_viewport then renders on that polyline (any viewport) until the
 * panels or densities change (dc_build_tree, dc_solve_density,
 * dc_solve_mixed, dc_set_density, dc_subdivide) or dc_view_reset;
 * dc_eval_points stays on the solve polyline.  Needs a density
 * (DC_ERR_STATE); DC_ERR_ARG for bad options or when e would exceed 4096;
 * errors of dc_subdivide and dc_build_tree.  stats may be NULL. */
dc_status dc_view_update(dc_ctx *ctx, const dc_viewport *vp, const dc_view_options *opt, dc_view_stats *stats);

/* Auxiliary: the quadtree of the context (its segments clipped into pieces
 * and its lists 1-4 built on the device) against the host construction over
 * the same segments.  out[0] = 1 when cells, piece counts, piece segments
 * and lists 1-4 (entry for entry, in order) are identical, out[1] = the largest difference of piece endpoints, out[2] =
 * cells, out[3] = pieces, out[4] and out[5] = wall ms of the last build's
 * clipping (device) and lists (host).  FMM forms after dc_build_tree
 * (DC_ERR_STATE). */
dc_status dc_aux_tree_compare(dc_ctx *ctx, double *out);

/* Renders on the solve polyline again (drops the view of dc_view_update). */
dc_status dc_view_reset(dc_ctx *ctx);

/* The current panels (after dc_subdivide, the refined ones), host outputs
 * in dc_build_tree's format: panel_ptr [n_curves + 1], panel_start
 * [panel_ptr[n_curves]] (either may be NULL; sizes from dc_get_sizes). */
dc_status dc_get_panels(dc_ctx *ctx, int *panel_ptr, double *panel_start);

/* Auxiliary: per-panel results of the last dc_subdivide, host outputs (any
 * may be NULL): top_old [panels before] the test value of step 1,
 * split_old [panels before] 1 where split, resolve_new [panels after] 1
 * where the density was re-solved.  Errors: DC_ERR_STATE before a call. */
dc_status dc_aux_subdivision_info(dc_ctx *ctx, double *top_old, unsigned char *split_old,
                                  unsigned char *resolve_new);

/* Node data after dc_build_tree, host outputs (any may be NULL):
 *   xy [n_nodes][2] collocation points on the solve polyline,
 *   t  [n_nodes] Bezier parameter of each node,
 *   u_plus, u_minus [n_nodes][3] boundary colours at the nodes. */
dc_status dc_get_nodes(dc_ctx *ctx, double *xy, double *t, double *u_plus,
                       double *u_minus);

dc_status dc_get_sizes(dc_ctx *ctx, dc_sizes *out);

/* Message of the last failed call on ctx ("" if none).  With ctx == NULL:
 * the message of the last failed dc_create in this process. */
const char *dc_last_error(dc_ctx *ctx);

const char *dc_status_string(dc_status st);

/* Auxiliary, host only (no GPU): builds the quadtree of Sec. 5.1-5.2 over
 * n_seg segments seg_xy[n_seg][4] (x1, y1, x2, y2, host) with a root that
 * also covers domain[4], and checks it:
 *   out[0] cells, out[1] leaves, out[2] depth, out[3] clipped pieces,
 *   out[4] number of (target leaf, source leaf) pairs that the four routes
 *          of Alg. 8 (list 1 direct, list 2 M2L, list 3 M2P, list 4 P2L,
 *          through all ancestors) cover zero or several times (0 = correct;
 *          O(leaves^2 depth^2) work, so keep inputs small),
 *   out[5] max over segments of |sum of piece lengths - segment length| /
 *          segment length (clipping partitions each segment).
 * Errors: DC_ERR_ARG for bad sizes or non-finite input. */
dc_status dc_aux_tree_check(int n_seg, const double *seg_xy, const double *domain,
                            int leaf_size, int max_depth, double *out);

/* Auxiliary, host only (no GPU): the adaptive panel rule dc_build_tree
 * applies when given no panels (see adapt_ratio in dc_options), with
 * explicit parameters (ratio > 0, max_level in [0, 30], min_panels >= 1,
 * max_len > 0).  ctrl host [n_curves][4][2]; outputs panel_ptr
 * [n_curves + 1] and *n_panels always, panel_start [*n_panels] when it fits
 * in capacity (else DC_ERR_ARG with *n_panels set, so a second call can size
 * the array).  Errors: DC_ERR_ARG, DC_ERR_GEOMETRY for a zero-length curve. */
dc_status dc_aux_adaptive_panels(int n_curves, const double *ctrl, double ratio, int max_level,
                                 int min_panels, double max_len, int capacity, int *panel_ptr,
                                 double *panel_start, int *n_panels);

/* Auxiliary, host only (no GPU): the discretisation dc_build_tree starts
 * from (Sec. 4.2, App. A-B), with the inputs of dc_build_tree (explicit
 * panels) and g, s as in dc_options.  With P = panel_ptr[n_curves],
 * N = P g nodes and S = P s segments it writes, each when not NULL:
 * node_xy host [N][2] collocation points, node_t [N] their Bezier
 * parameters, seg_xy [S][4] segment end points (x1 y1 x2 y2), seg_w [S]
 * arc length / chord length, u_plus and u_minus [N][3] boundary colours.
 * Errors as dc_build_tree's: DC_ERR_ARG, DC_ERR_GEOMETRY. */
dc_status dc_aux_discretise(int n_curves, const double *ctrl, const int *panel_ptr, const double *panel_start,
                            const double *colours, int g, int s, double *node_xy, double *node_t,
                            double *seg_xy, double *seg_w, double *u_plus, double *u_minus);

/* ---------------------------------------------------------------------
 * Learned warm start (no counterpart in the paper: its warm start, Sec. 6.1,
 * re-uses an earlier solution).  A 4-layer perceptron
 *     n_in -> hidden -> hidden -> hidden -> n_out,  GELU between layers,
 * predicts one panel's g node densities times the panel's arc length for one
 * colour channel from n_in = 22 g + 32 local features: the panel's own nodes
 * (position and normal in the panel frame, scaled by its arc length), its
 * boundary colours u+ and u-, the boundary colours of the 8 nearest other
 * panels by node centroid and those panels' centroid offsets and chord
 * directions.  Parameters are FP32, packed layer by layer as W_l [out][in]
 * row-major then b_l [out]; the network reads them rounded to BF16 and
 * accumulates in FP32.  All device pointers below are caller-owned; work is
 * issued on `stream` (cudaStream_t, NULL = legacy default stream).
 * --------------------------------------------------------------------- */

/* Parameter count and workspace size (floats) for a batch of `batch` rows. */
size_t dc_aux_mlp_param_count(int n_in, int hidden, int n_out);
size_t dc_aux_mlp_workspace_floats(int n_in, int hidden, int n_out, int batch);

/* y [batch][n_out] = net(x [batch][n_in]); params, x, y, work on the device.
 * Errors: DC_ERR_ARG for bad sizes or NULL pointers, DC_ERR_CUDA. */
dc_status dc_aux_mlp_forward(int n_in, int hidden, int n_out, const float *params, int batch,
                             const float *x, float *y, float *work, void *stream);

/* Mean squared error of net(x) against target [batch][n_out] into *loss
 * (device float) and its gradient with respect to the parameters into
 * grad [param_count] (device).  The gradient is that of the network as it
 * computes (BF16-rounded weights, exact GELU), with the bias and weight
 * reductions over the batch in a fixed order (deterministic). */
dc_status dc_aux_mlp_loss_grad(int n_in, int hidden, int n_out, const float *params, int batch,
                               const float *x, const float *target, float *grad, float *loss,
                               float *work, void *stream);

/* One Adam step (Kingma and Ba 2015) on n parameters: m, v are the moment
 * buffers (zero before step 1), step counts from 1. */
dc_status dc_aux_mlp_adam(size_t n, float *params, const float *grad, float *m, float *v, float lr,
                          float beta1, float beta2, float eps, int step, void *stream);

/* Sizes of the context's feature rows (one per panel and colour channel):
 * *rows = 3 n_panels, *n_features = 22 g + 32, *n_out = g.
 * Errors: DC_ERR_STATE before dc_build_tree. */
dc_status dc_aux_feature_dims(dc_ctx *ctx, int *rows, int *n_features, int *n_out);

/* Writes the features of every (panel, channel) row to feat_dev
 * [rows][n_features] (device, float) and, if target_dev is not NULL, the
 * current density as targets [rows][n_out] (sigma times panel arc length;
 * needs a density: DC_ERR_STATE otherwise).  Row 3 j + c is panel j,
 * channel c; nodes are in panel order. */
dc_status dc_aux_panel_features(dc_ctx *ctx, float *feat_dev, float *target_dev);

/* Sets the network that DC_X0_LEARNED uses: params [dc_aux_mlp_param_count(
 * 22 g + 32, hidden, g)] floats in `where` memory (DC_MEM_HOST or
 * DC_MEM_DEVICE), copied into the context.  hidden = 0 removes the model.
 * Errors: DC_ERR_ARG for bad sizes or non-finite parameters. */
dc_status dc_aux_set_warm_start_model(dc_ctx *ctx, int hidden, const float *params, int where);

/* Auxiliary: one application of the operator at the nodes, the call
 * FMM(S, sigma, q) of Sec. 5.5 (the matvec of GMRES):
 *   op 0: y = G_H x (single layer, Eq. 19), op 1: y = F_H x (double layer)
 * in the context's form.  With DC_FORM_FMM32 (op 0 only), inner = 1 applies
 * the FP32 operator of the inner GMRES instead, y = G_H M x with M the
 * two-level preconditioner (panel blocks of G_H inverted and a coarse space
 * of panel constants; order p_inner), inner = 2 the same FP32 operator
 * without M, y = G_H x, and (any FMM form) inner = 3 the preconditioner
 * alone, y = M x.
 *   x, y  [n_nodes][3] double, device, caller-owned, distinct
 * Errors: DC_ERR_STATE before dc_build_tree, DC_ERR_ARG for a bad op,
 * inner or pointer, DC_ERR_UNSUPPORTED for inner 1..3 in other forms. */
dc_status dc_aux_apply_operator(dc_ctx *ctx, int op, int inner, const double *x, double *y);

/* Auxiliary: state of the FMM forms' two-level preconditioner (no
 * counterpart in the paper; it changes the iteration count, not the
 * solution), host double[5]: out[0] = 1 if the coarse level is in use (else
 * the panel blocks alone), out[1] = coarse unknowns (panels, or aggregates
 * of out[4] consecutive panels of a curve when the panels outnumber the
 * dense coarse inverse's limit of 12,288; the levels are then combined
 * additively), out[2] = near panel pairs, out[3] = max |(Ac^-1 Ac - I)_ij|
 * over sampled entries of the coarse inverse, out[4] = panels per
 * aggregate (1 = one coarse unknown per panel, multiplicative form).
 * Errors: DC_ERR_STATE before dc_build_tree or in the dense form. */
dc_status dc_aux_precond_info(dc_ctx *ctx, double *out);

/* Auxiliary: wall-clock ms of the last dc_build_tree, by phase (each phase
 * drains the context's stream before it is timed): out[0] discretisation
 * (host), out[1] uploads, out[2..7] the FMM build (quadtree and lists;
 * schedules and uploads; the wait for the two-level preconditioner, whose
 * work runs beside the two phases before it; stored P2M / P2L rows, with
 * the node near / far coefficients built beside them; the wait for those
 * coefficients; FP32 form), out[8] panel features, out[9] G_H 1, out[10]
 * total.  out: host array of 11 doubles (zero where a phase does not
 * apply).  Errors: DC_ERR_STATE before dc_build_tree. */
dc_status dc_aux_build_timings(dc_ctx *ctx, double *out);

/* Auxiliary measurement (no counterpart in the paper): the FP32 vector peak
 * of the current device, timed with CUDA events on `stream` (cudaStream_t,
 * NULL = legacy default stream): 8 independent fused multiply-add chains per
 * thread, 8 blocks of 256 threads per SM, best of three timed launches.
 *   out  host double[2]: out[0] TFLOP/s (2 flops per FMA), out[1] ms of the
 *        best launch
 * Errors: DC_ERR_ARG for NULL out, DC_ERR_CUDA. */
dc_status dc_aux_fp32_peak(void *stream, double *out);

/* Auxiliary measurement: device time of the M2L kernels (Eq. 69 over list
 * 2, Alg. 8) of the FP32 inner operator (DC_FORM_FMM32), `reps` launches
 * each after one warm-up, CUDA events on the context's stream.
 *   out  host double[6]: out[0] ms per launch of the main kernel (tcgen05
 *        tiles, or the CUDA-core kernel), out[1] ms of the tensor path's
 *        per-target reduction (0 on the CUDA cores), out[2] algorithmic
 *        flops per application: 8 (p_i + 1)^2 per list-2 pair and channel,
 *        out[3] flops the tensor pipe executes per application (0 on the
 *        CUDA cores), out[4] engine (DC_M2L_TENSOR / DC_M2L_CUDA_CORES),
 *        out[5] list-2 pairs
 * The kernels read and overwrite the context's inner expansions (the next
 * solve recomputes them).  Errors: DC_ERR_ARG, DC_ERR_STATE before
 * dc_build_tree or in other forms, DC_ERR_UNSUPPORTED without list-2
 * pairs, DC_ERR_TIMEOUT when a bounded wait ran out, DC_ERR_CUDA. */
dc_status dc_aux_time_inner_m2l(dc_ctx *ctx, int reps, double *out);

/* Auxiliary test hook (no counterpart in the paper) for the bounded device
 * waits of DC_FORM_FMM32 with m2l_engine DC_M2L_TENSOR: from the next
 * operator application on, the CTA of the tensor-core M2L that takes tile
 * `tile` (0-based, in the kernel's tile order) issues neither its MMAs nor
 * their commit, so its wait on the commit runs out after about 20 ms; the
 * kernel then sets the context's wait-limit flag, frees its tensor memory
 * and returns.  The running GMRES cycle ends at its next Givens step and
 * dc_solve_density returns DC_ERR_TIMEOUT.  The flag is cleared at the start
 * of every solve; tile = -1 switches the hook off, and the next solve is then
 * clean.  Nothing faults: no MMA is in flight when the memory is freed.
 * Errors: DC_ERR_ARG for tile < -1, DC_ERR_STATE before dc_build_tree or in
 * the dense form, DC_ERR_UNSUPPORTED when the inner operator's M2L does not
 * run on the tensor cores (p_inner > 15 or DC_M2L_CUDA_CORES). */
dc_status dc_aux_test_skip_mma_tile(dc_ctx *ctx, int tile);

int dc_abi_version(void);

/* Auxiliary: number of CUDA kernels this library has launched in this
 * process (all contexts), for launch accounting by benchmarks. */
long long dc_aux_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* DC_FMM_H */
