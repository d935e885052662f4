// Internal declarations of libdc_fmm (host side).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>
#include <utility>
#include <unordered_map>
#include <mutex>
#include <map>

#include "dc_fmm.h"

namespace dc {

constexpr int kMaxG = 32;        // nodes per panel supported by the kernels
constexpr int kMaxP = 40;        // expansion order supported by the kernels

// ------------------------------------------------------------ geometry --
// Host discretisation of a drawing (Sec. 4.2, App. A, App. B).
struct Geometry {
    int n_curves = 0, n_panels = 0, g = 0, s = 0;
    std::vector<double> node_xy;      // [N][2] collocation points (polyline)
    std::vector<double> node_t;       // [N] Bezier parameter
    std::vector<int> node_seg;        // [N] segment holding the node
    std::vector<int> node_seg2;       // [N] second segment at a vertex or -1
    std::vector<int> node_curve;      // [N]
    std::vector<double> seg_xy;       // [S][4] x1 y1 x2 y2
    std::vector<double> seg_w;        // [S] arc length / chord length
    std::vector<double> lambda;       // [s][g] node -> segment-midpoint map
    std::vector<double> u_plus;       // [N][3]
    std::vector<double> u_minus;      // [N][3]
    std::vector<double> curve_len;    // [n_curves]
    double bbox[4] = {0, 0, 0, 0};    // of all segment endpoints
    int n_nodes() const { return n_panels * g; }
    int n_segments() const { return n_panels * s; }
};

// Returns DC_OK or an error with a message in err.
dc_status discretise(int n_curves, const double *ctrl, const int *panel_ptr,
                     const double *panel_start, const double *colours, int g,
                     int s, Geometry &out, std::string &err);

// Adaptive panel split (panels.cpp): ptr [n_curves + 1], start [panels].
dc_status adaptive_panels(int n_curves, const double *ctrl, double ratio, int max_level, int min_panels,
                          double max_len, std::vector<int> &ptr, std::vector<double> &start, std::string &err);

// Gauss-Legendre nodes on [-1, 1] (ascending) and weights.
void gauss_legendre_rule(int n, double *x, double *w);

// Process-wide count of kernels launched by this library (dc_api.cpp).
void note_launch(int n = 1);
// FP32 FMA-chain peak of the current device in TFLOP/s (peaks.cu)
cudaError_t measure_fp32_peak(cudaStream_t st, double *tflops, double *ms_out);
long long kernel_launches();

// Adaptive subdivision and local re-solve (adaptive.cu; Sec. 6.1, 6.3)
void legendre_top_row(int g, double *q);          // last row of the Legendre transform
void split_matrices(int g, double *E);            // [3][g][g]: keep, left half, right half
cudaError_t launch_legendre_top(const double *sigma, int n_panels, int g, const double *q, double *top,
                                cudaStream_t st);
cudaError_t launch_split_interp(const double *sig_old, const int2 *pmap, const double *E, int g, int n_new,
                                double *sig_new, cudaStream_t st);
cudaError_t launch_unit_density(double *x, int N, int g, const int panels[3], cudaStream_t st);
cudaError_t launch_panel_range(const double *v, int n_panels, int g, double *out, cudaStream_t st);
cudaError_t launch_node_mask(double *v, const unsigned char *pmask, int N, int g, cudaStream_t st);
// out = pmask[panel] ? beta b : alpha a
cudaError_t launch_blend(double *out, const double *a, double alpha, const double *b, double beta,
                         const unsigned char *pmask, int N, int g, cudaStream_t st);
// *out = max |a_i - b_i| (FP32 bits, device)
cudaError_t launch_max_diff(const float *a, const double *b, long long n, unsigned *out, cudaStream_t st);

// ---------------------------------------------------------- device util --
// While a FreeDefer lives on a thread, the frees of device buffers released
// on that thread are held back until flush() or its end: cudaFree waits for
// all of the device's work, including other streams' work that the thread
// means to overlap.
struct FreeDefer {
    std::vector<std::pair<void *, size_t>> ptrs;   // block, bytes
    FreeDefer *prev;
    FreeDefer();
    ~FreeDefer();
    void flush();
    void take(std::vector<std::pair<void *, size_t>> &out);    // hands the held frees to the caller
    void adopt(std::vector<std::pair<void *, size_t>> &in);    // holds another thread's frees too
    FreeDefer(const FreeDefer &) = delete;
    FreeDefer &operator=(const FreeDefer &) = delete;
};

// A cache of idle device blocks, one per context.  While a DevPool is
// installed on a thread (PoolScope), buffers allocated there take a cached
// block that fits before calling cudaMalloc, and buffers freed there (after
// a FreeDefer, if one holds them back) return their block to the cache
// instead of calling cudaFree.  Whoever installs it guarantees that no
// pending device work reads or writes a block that is freed meanwhile.
// Blocks not taken during one rebuild are freed at the end of the next.
class DevPool {
public:
    void *get(size_t bytes);          // nullptr when no cached block fits
    void put(void *p, size_t bytes);
    void next_generation();           // cudaFree blocks cached before the last call and not taken since
    void trim();                      // cudaFree every cached block
    ~DevPool() { trim(); }

private:
    struct Block {
        void *p;
        size_t cap;
        int gen;
    };
    std::mutex mu_;
    std::multimap<size_t, Block> free_;   // by capacity
    std::unordered_map<void *, size_t> cap_;   // capacities of the blocks handed out
    int gen_ = 0;
};
struct PoolScope {
    explicit PoolScope(DevPool *p);
    ~PoolScope();
    DevPool *prev;
    PoolScope(const PoolScope &) = delete;
    PoolScope &operator=(const PoolScope &) = delete;
};
DevPool *current_pool();                        // the pool installed on this thread, or null
cudaError_t dev_alloc(void **p, size_t bytes);  // the thread's pool, else cudaMalloc
void dev_free(void *p, size_t bytes);           // held back, cached, or cudaFree

template <typename T>
struct DevBuf {
    T *ptr = nullptr;
    size_t n = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    cudaError_t alloc(size_t count) {
        release();
        if (count == 0) return cudaSuccess;
        cudaError_t e = dev_alloc(reinterpret_cast<void **>(&ptr), count * sizeof(T));
        if (e == cudaSuccess) n = count; else ptr = nullptr;
        return e;
    }
    cudaError_t ensure(size_t count) {
        if (count <= n) return cudaSuccess;
        return alloc(count);
    }
    void release() {
        if (ptr) dev_free(ptr, n * sizeof(T));
        ptr = nullptr;
        n = 0;
    }
    size_t bytes() const { return n * sizeof(T); }
};

// Device copy of the discretisation.
struct DevGeom {
    int N = 0, S = 0, g = 0, s = 0, n_panels = 0;
    DevBuf<double> seg;       // [S][4]
    DevBuf<double> segw;      // [S]
    DevBuf<double> node_xy;   // [N][2]
    DevBuf<int> node_seg;     // [N]
    DevBuf<int> node_seg2;    // [N]
    DevBuf<double> lambda;    // [s][g]
    DevBuf<double> u_plus;    // [N][3]
    DevBuf<double> u_minus;   // [N][3]
};

// Pixel grid of one viewport on the device.
struct VpDev {
    double x0, y0, dx, dy;
    int width, height;
    long long offset;         // first output pixel of this viewport
};

// Exclusive scan of int counts on the device (aa.cu): out[i] = sum of
// in[0..i); the total lands in total.ptr[0] (device).  in may equal out.
struct ScanWork {
    static constexpr int kLevels = 6;
    DevBuf<long long> lv[kLevels];
    DevBuf<long long> total;
};
cudaError_t scan_exclusive(const int *in, int *out, long long n, ScanWork &w, cudaStream_t st);

// Quadtree anti-aliasing of a render (Sec. 7; aa.cu).  prepare() finds the
// pixels whose closed square meets a segment, splits their cells and lists
// the samples (sxy [n_samples][2], weights sw); the caller evaluates the
// colours at sxy into u [n_samples][3]; finish() writes each refined
// pixel's weighted sum over the render's outputs.  cudaErrorInvalidValue
// with err set for calls beyond the index ranges.
struct AaWork {
    DevBuf<VpDev> vps;
    DevBuf<int> cnt, off, ids, ns, soff;
    DevBuf<long long> edge;
    DevBuf<double> sxy, sw, u;
    ScanWork scan;
    int n_edge = 0, n_samples = 0;
    cudaError_t prepare(const DevGeom &G, const VpDev *vps_host, int n_vp, long long total_px, int levels,
                        cudaStream_t st, std::string &err);
    cudaError_t finish(void *rgb, int rgb_dtype, unsigned char *rgb8, cudaStream_t st);
};

// ------------------------------------------------------- kernel entry --
// K1: values at segments from values at nodes (sigma_bar = Lambda sigma).
cudaError_t launch_interp(const DevGeom &G, const double *node_vals, double *seg_vals,
                          cudaStream_t st);

// K9 (plain dense form): A_G, A_F [N][N] row-major (Eq. 19 / Eq. 27).
cudaError_t launch_dense_assemble(const DevGeom &G, double *AG, double *AF, cudaStream_t st);
// y[N][3] = A[N][N] x[N][3]
cudaError_t launch_dense_gemv(const double *A, int N, const double *x, double *y,
                              cudaStream_t st);
// Direct-sum layer potential at pixel centres of one viewport, FP64.
cudaError_t launch_dense_eval_grid(const DevGeom &G, const double *sbar, const double *mbar,
                                   const VpDev &vp, double *u, cudaStream_t st);
// Direct-sum layer potential at explicit points, FP64.
cudaError_t launch_dense_eval_points(const DevGeom &G, const double *sbar, const double *mbar,
                                     const double *xy, int n, double *u, cudaStream_t st);

// Block-Jacobi preconditioner over panels: inv[j] = (G_H)_{jj}^-1, the
// inverse of panel j's g x g self-interaction block; info[j] = 1 if singular.
cudaError_t launch_panel_block_inverse(const DevGeom &G, double *inv, int *info, cudaStream_t st);
// y = blockdiag(inv) x on [N][3] vectors.
cudaError_t launch_block_apply(const double *inv, int n_panels, int g, const double *x, double *y,
                               cudaStream_t st);

// Output conversion: u[n][3] FP64 -> rgb (f32 or f64) and rgb8 (K12).
cudaError_t launch_write_outputs(const double *u, long long n, void *rgb, int rgb_dtype,
                                 unsigned char *rgb8, cudaStream_t st);
cudaError_t launch_write_outputs_f32(const float *u, long long n, void *rgb, int rgb_dtype,
                                     unsigned char *rgb8, cudaStream_t st);

// b = (u+ + u-)/2 - Fmu ; mu = u+ - u-
cudaError_t launch_mu(const DevGeom &G, double *mu, cudaStream_t st);
cudaError_t launch_rhs(const DevGeom &G, const double *Fmu, double *b, cudaStream_t st);

// Per-panel features of the learned warm start (features.cu): one row per
// (panel, colour channel), n_features(g) floats; targets are the panel's g
// node densities times its arc length.
class PanelFeatures {
public:
    static int n_features(int g) { return 22 * g + 32; }
    cudaError_t build(const Geometry &G, cudaStream_t st);
    bool ready() const { return P_ > 0; }
    int rows() const { return 3 * P_; }
    // feat [rows][n_features]; target [rows][g] (when sigma and target are given)
    cudaError_t compute(const DevGeom &D, const double *sigma, float *feat, float *target,
                        cudaStream_t st) const;
    // sigma [N][3] from predictions pred [rows][g]
    cudaError_t apply(const float *pred, double *sigma, cudaStream_t st) const;

private:
    int P_ = 0, g_ = 0;
    DevBuf<double> pc_, pt_, plen_, nn_;
    DevBuf<int> nbr_;
};

// Two-level preconditioner (coarse.cu): M v = P y + B (v - A~ P y),
// y = Ac^-1 R v, with B the panel blocks' inverses and a coarse space of
// panel-wise constants.  build() forms the near-pair corrections and inverts
// the coarse matrix; ready() is false when that failed (one level then).
class TwoLevel {
public:
    // Built in three steps, so that the caller can overlap them with other
    // work: plan() is host work only (centroids, aggregates, near panel
    // pairs; max_coarse: most coarse unknowns, 0 = the built-in 12288);
    // launch() enqueues the uploads, the coarse matrix, its inversion and the
    // check of the inverse on st and waits for none of them; finish() waits
    // for st and decides from the check whether the coarse level is used.
    void plan(const Geometry &G, int max_coarse);
    cudaError_t launch(const DevGeom &D, cudaStream_t st);
    cudaError_t finish(cudaStream_t st);
    bool ready() const { return ready_; }
    // coarse unknowns (panels, or aggregates of K panels), near panel pairs,
    // max |(Ac^-1 Ac - I)_ij| over 5 sampled rows, K
    void info(double out[5]) const {
        out[0] = ready_ ? 1.0 : 0.0;
        out[1] = nA_;
        out[2] = n_pairs_;
        out[3] = check_;
        out[4] = K_;
    }
    // w = M v on [N][3] vectors (w may be null); inv: the panel blocks'
    // inverses.  With lam (Lambda as hi/lo floats, [s][g]) and sv: also
    // sv = Lambda (M v) per panel, [S][3] FP32.
    cudaError_t apply(const double *inv, const double *v, double *w, cudaStream_t st, const float2 *lam = nullptr,
                      int s = 0, float *sv = nullptr);
    // The aggregated form (aggregated() true) in two stages around the
    // caller's operator application: stage 1 solves the coarse system and
    // spreads py = P y to the nodes; stage 2 takes gpy = G_H py and forms
    // w = P y + B (v - gpy) (and sv as in apply).
    bool aggregated() const { return ready_ && K_ > 1; }
    cudaError_t apply_stage1(const double *v, double *py, cudaStream_t st);
    cudaError_t apply_stage2(const double *inv, const double *v, const double *gpy, double *w, cudaStream_t st,
                             const float2 *lam = nullptr, int s = 0, float *sv = nullptr);

private:
    bool ready_ = false, planned_ = false, launched_ = false;
    int P_ = 0, g_ = 0, s_seg_ = 0, N_ = 0, n_pad_ = 0, n_pairs_ = 0, nA_ = 0, K_ = 1;
    // plan() output, uploaded by launch()
    std::vector<float2> h_c32_, h_q32_;
    std::vector<double> h_pl_;
    std::vector<float> h_pl32_;
    std::vector<int> h_pagg_, h_perm_, h_agg_of_, h_nptr_;
    std::vector<int2> h_pairs_;
    // launch() to finish(): the coarse matrix before inversion, the check's
    // row errors and its bad-pivot flag
    DevBuf<float> Ac_, gj_tmp_;
    DevBuf<double> errs_;
    DevBuf<int> bad_;
    DevBuf<int> pagg_, agg_of_, perm_;   // aggregates: start of each in perm_ (+ end), aggregate of each
                                         // panel, panels in Morton order
    double check_ = -1.0;
    DevBuf<float2> c32_, q32_;
    DevBuf<double> plen_, corr_, y_;
    DevBuf<float> plen32_, pan2_, Ainv_, part_;
    DevBuf<float4> pan_;
    DevBuf<float2> s_;
    DevBuf<int> nptr_;
    DevBuf<int2> pairs_;
};

// --------------------------------------------------------------- GMRES --
// Matrix-free operator y = A x on [N][3] FP64 vectors (all 3 channels).
struct Operator {
    virtual ~Operator() = default;
    virtual cudaError_t apply(const double *x, double *y, cudaStream_t st) = 0;
    // Optional: an operator that reads its input from a buffer of its own
    // and writes its output to another (a captured graph) returns both, and
    // apply_buffers() applies it there without copies.
    virtual double *in_buffer() { return nullptr; }
    virtual double *out_buffer() { return nullptr; }
    virtual cudaError_t apply_buffers(cudaStream_t) { return cudaErrorNotSupported; }
    // Optional: a device int that the operator's kernels set when a bounded
    // wait ran out; GMRES then ends its cycle at the next Givens step.
    virtual const int *fault_flag() { return nullptr; }
};

struct GmresResult {
    int iters[3] = {0, 0, 0};
    double true_rel_resid[3] = {0, 0, 0};   // recomputed b - A x, never an estimate
    double rel_resid[3] = {0, 0, 0};
    int converged = 0;
    int n_matvec = 0;
    int stagnated = 0;   // stopped at the operator's own error level
};

struct GmresWork;   // device workspace (gmres.cu)
GmresWork *gmres_work_create();
void gmres_work_destroy(GmresWork *w);

// Restarted GMRES for the 3 channels at once (Sec. 5.5), FP64 Arnoldi by
// classical Gram-Schmidt with one re-orthogonalisation pass, Givens
// rotations and the least-squares update on the device.  x holds x0 on
// entry and the solution on exit; x0_zero: x is zero on entry (the first
// residual is b, no operator application); trust_estimate: stop as soon as
// a cycle's Givens residual estimate meets tol (the caller checks the true
// residual itself), rel_resid then holds the estimate.
cudaError_t gmres_solve(GmresWork *w, Operator &A, int N, const double *b, double *x, bool x0_zero,
                        bool trust_estimate, double tol, int restart, int max_iter, cudaStream_t st,
                        GmresResult &res, std::string &err);

// Allocation-free FP64 direct sum at points (noalloc.cu): segment densities
// in a static device array of noalloc_max_segments() segments.
int noalloc_max_segments();
cudaError_t eval_points_noalloc(const DevGeom &G, const double *sigma, const double *mu,
                                const double *xy, int n, double *out, cudaStream_t st,
                                std::string &err);

// Small FP64 vector helpers on [N][3] vectors (gmres.cu).
cudaError_t vec_residual(const double *b, const double *Ax, double *r, int n3, cudaStream_t st);
cudaError_t vec_axpy(double *x, const double *d, int n3, cudaStream_t st);
// zero the channels c with keep[c] == 0
cudaError_t vec_mask3(double *v, int N, const int keep[3], cudaStream_t st);
// y[:, c] = a[c] x[:, c] + b[c] z[:, c] (z == nullptr: a vector of ones; a[c] == 0:
// x[:, c] is not read); y may alias x
cudaError_t vec_combine3(const double *x, const double *z, double *y, int N, const double a[3],
                         const double b[3], cudaStream_t st);
// host_out[c] = u[:, c] . v[:, c] (synchronises the stream)
cudaError_t vec_dots3(GmresWork *w, const double *u, const double *v, int N, double host_out[3],
                      cudaStream_t st);
// host_out[c] = || v[:, c] ||_2 (synchronises the stream)
cudaError_t vec_norms3(GmresWork *w, const double *v, int N, double host_out[3], cudaStream_t st);

}  // namespace dc
