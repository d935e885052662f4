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

typedef enum { DC_X0_ONES = 0, DC_X0_ZEROS = 1, DC_X0_USER = 2 } dc_x0_mode;
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
} dc_options;

typedef struct {
    int n_curves, n_panels, n_nodes, n_segments;
    int n_pieces;          /* segments after clipping at leaf boundaries     */
    int n_cells, n_leaves, depth;
    double root[3];        /* root cell centre x, y and half-width           */
} dc_sizes;

typedef struct {
    int iters[3];          /* GMRES iterations per colour channel            */
    double rel_resid[3];   /* final ||b - A x|| / ||b|| (GMRES estimate)     */
    int converged;         /* 1 if every channel met gmres_tol               */
    int n_matvec;          /* operator applications, right-hand side included */
    double ms_rhs;         /* right-hand side (Alg. 3 line 4), device time   */
    double ms_solve;       /* GMRES (Alg. 3 line 5), host wall time          */
    long long p2p_pairs;   /* near-field (target, piece) pairs per matvec    */
    long long m2l_pairs;   /* cell pairs in M2L per matvec                   */
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
} dc_render_stats;

/* Fills *opt with defaults: DC_FORM_FMM32, g 16, s 80, p 24, leaf 64,
 * depth 30, tol 1e-10, restart 200, max_iter 2000, x0 ones, domain [0,1]^2. */
dc_status dc_default_options(dc_options *opt);

/* Creates a context bound to the current CUDA device.  *out is set to NULL
 * on failure. */
dc_status dc_create(dc_ctx **out, const dc_options *opt);

/* Frees every device and host resource of the context (NULL is a no-op). */
void dc_destroy(dc_ctx *ctx);

/* Discretises the drawing and builds the solver state (Alg. 3 lines 1-2:
 * quadtree(S) and pre_FMM(S, q, Q), Sec. 5.3).
 *   ctrl         host [n_curves][4][2] control points C0..C3 (App. B)
 *   panel_ptr    host [n_curves + 1]; curve i owns panels
 *                panel_ptr[i] .. panel_ptr[i+1]-1 (at least one each)
 *   panel_start  host [panel_ptr[n_curves]]: arc-length fraction in [0,1)
 *                where each panel starts, strictly increasing per curve,
 *                first = 0 (panels end where the next starts, or at 1)
 *   colours      host [n_curves][2][2][3]: [side: 0 = u+ (right of travel),
 *                1 = u- (left)][end: colour at t = 0, t = 1][rgb]; colours
 *                are linear in the Bezier parameter t between the ends
 * Errors: DC_ERR_ARG for bad sizes/ordering/non-finite values,
 * DC_ERR_GEOMETRY for a zero-length curve or panel, DC_ERR_OOM/CUDA.
 * Replaces any previous drawing of the context. */
dc_status dc_build_tree(dc_ctx *ctx, int n_curves, const double *ctrl,
                        const int *panel_ptr, const double *panel_start,
                        const double *colours);

/* Solves for the density (Alg. 3 lines 3-5): mu = u+ - u-,
 * b = (u+ + u-)/2 - F_H mu, sigma = GMRES(G_H, x0, b, tol) with FP64
 * Arnoldi.  x0: host [n_nodes][3] used when x0_mode == DC_X0_USER (else
 * may be NULL).  stats may be NULL.  Returns DC_ERR_NOCONV (density kept,
 * stats filled) if gmres_max_iter is reached first. */
dc_status dc_solve_density(dc_ctx *ctx, const double *x0, dc_solve_stats *stats);

/* Renders n_vp viewports (Alg. 4 line 3): u = single layer of sigma plus
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
 * Errors: DC_ERR_STATE without a density, DC_ERR_ARG for bad sizes. */
dc_status dc_eval_points_noalloc(dc_ctx *ctx, int n, const double *xy_dev, double *out_dev);

/* Copies the current density sigma at the nodes to host [n_nodes][3]. */
dc_status dc_get_density(dc_ctx *ctx, double *sigma_out);

/* Sets the density from host [n_nodes][3] (instead of solving). */
dc_status dc_set_density(dc_ctx *ctx, const double *sigma_in);

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

int dc_abi_version(void);

/* Auxiliary: number of CUDA kernels this library has launched in this
 * process (all contexts), for launch accounting by benchmarks. */
long long dc_aux_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* DC_FMM_H */
