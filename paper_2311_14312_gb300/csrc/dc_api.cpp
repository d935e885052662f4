// C ABI of libdc_fmm (declarations and contracts in include/dc_fmm.h).
//
// The entry points follow the paper's problem statement: build the
// discretisation and quadtree (Alg. 3), solve for the density
// (Alg. 3), render viewports (Alg. 4).
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "dc_internal.h"
#include "fmm.h"
#include "tree.h"

using dc::DevBuf;

namespace dc {
static std::atomic<long long> g_launches{0};
void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

namespace {
thread_local FreeDefer *t_defer = nullptr;
thread_local DevPool *t_pool = nullptr;
void free_now(void *p, size_t bytes) {   // to the thread's pool, else cudaFree
    if (t_pool) {
        try {
            t_pool->put(p, bytes);
            return;
        } catch (...) {   // no room to record it: free now
        }
    }
    cudaFree(p);
}
}  // namespace
FreeDefer::FreeDefer() : prev(t_defer) { t_defer = this; }
FreeDefer::~FreeDefer() {
    flush();
    t_defer = prev;
}
void FreeDefer::flush() {
    for (auto &b : ptrs) free_now(b.first, b.second);
    ptrs.clear();
}
void FreeDefer::take(std::vector<std::pair<void *, size_t>> &out) {
    out.insert(out.end(), ptrs.begin(), ptrs.end());
    ptrs.clear();
}
void FreeDefer::adopt(std::vector<std::pair<void *, size_t>> &in) {
    ptrs.insert(ptrs.end(), in.begin(), in.end());
    in.clear();
}
void dev_free(void *p, size_t bytes) {
    if (!p) return;
    if (t_defer) {
        try {
            t_defer->ptrs.emplace_back(p, bytes);
            return;
        } catch (...) {   // no room to hold it back: free now
        }
    }
    free_now(p, bytes);
}
cudaError_t dev_alloc(void **p, size_t bytes) {
    *p = nullptr;
    if (t_pool) {
        try {
            if ((*p = t_pool->get(bytes)) != nullptr) return cudaSuccess;
        } catch (...) {
        }
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) *p = nullptr;
    return e;
}
void *DevPool::get(size_t bytes) {
    std::lock_guard<std::mutex> lock(mu_);
    // the smallest cached block that holds the request without wasting more
    // than about as much again
    auto it = free_.lower_bound(bytes);
    if (it == free_.end() || it->first > 2 * bytes + 4096) return nullptr;
    Block b = it->second;
    free_.erase(it);
    cap_[b.p] = b.cap;
    return b.p;
}
void DevPool::put(void *p, size_t bytes) {
    std::lock_guard<std::mutex> lock(mu_);
    size_t cap = bytes;
    auto it = cap_.find(p);
    if (it != cap_.end()) {
        cap = std::max(cap, it->second);
        cap_.erase(it);
    }
    free_.emplace(cap, Block{p, cap, gen_});
}
void DevPool::next_generation() {
    std::lock_guard<std::mutex> lock(mu_);
    for (auto it = free_.begin(); it != free_.end();) {
        if (it->second.gen < gen_) {
            cudaFree(it->second.p);
            it = free_.erase(it);
        } else {
            ++it;
        }
    }
    ++gen_;
}
void DevPool::trim() {
    std::lock_guard<std::mutex> lock(mu_);
    for (auto &kv : free_) cudaFree(kv.second.p);
    free_.clear();
}
PoolScope::PoolScope(DevPool *p) : prev(t_pool) { t_pool = p; }
PoolScope::~PoolScope() { t_pool = prev; }
DevPool *current_pool() { return t_pool; }
long long kernel_launches() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace dc

struct dc_ctx {
    dc_options opt{};
    std::string err;
    cudaStream_t stream = nullptr;
    int device = 0;
    int state = 0;                 // 0 empty, 1 built, 2 density available
    dc::DevPool pool;              // idle device blocks recycled between rebuilds
    dc::Geometry geo;
    dc::DevGeom dg;
    DevBuf<double> mu, sigma, b, fmu, sbar, mbar, u64, xy;
    DevBuf<float> u32;
    DevBuf<unsigned char> stage8;
    DevBuf<double> stage64;
    DevBuf<double> AG, AF;         // dense form
    bool seg_density_valid = false;
    bool mu_custom = false;
    dc::AaWork aa;                 // anti-aliasing buffers (options.aa_levels)        // mu set by dc_solve_mixed (restored from the colours by the next solve)
    dc::GmresWork *gw = nullptr;
    std::unique_ptr<dc::Fmm> fmm;  // FMM forms
    // learned warm start: network parameters, feature tables, buffers
    int warm_hidden = 0;
    DevBuf<float> warm_params, warm_feat, warm_pred, warm_work;
    DevBuf<double> warm_ax, warm_a1;   // G_H x_pred, G_H 1
    bool warm_a1_valid = false;
    double build_ms[11] = {};   // dc_aux_build_timings
    dc::PanelFeatures pfeat;
    bool feat_built = false;       // pfeat for the current drawing (built on first use)
    // the drawing as given to dc_build_tree (host copies), for dc_subdivide
    int in_ncurves = 0;
    std::vector<double> in_ctrl, in_start, in_col;
    std::vector<int> in_ptr;
    // adaptive subdivision (Alg. 5-7): device scratch and the last call's
    // per-panel results
    DevBuf<double> ad_sig_old, ad_r0, ad_tmp, ad_tmp2, ad_q, ad_E, ad_top, ad_range;
    DevBuf<int2> ad_pmap;
    DevBuf<unsigned char> ad_mask;
    std::vector<double> last_top;
    std::vector<unsigned char> last_split, last_resolve;
    // the viewport's evaluation discretisation (Sec. 6.2, 6.4): a render-only
    // context on the same panels with e segments each, used by
    // dc_render_viewport while view_valid (cleared by every change of the
    // panels or the densities)
    dc_ctx *view = nullptr;
    bool view_valid = false;
    bool render_only = false;      // this context is a view: no solve structures
    ~dc_ctx();
};

dc_ctx::~dc_ctx() {
    if (view) {
        cudaStreamSynchronize(view->stream);
        delete view;
    }
    if (gw) dc::gmres_work_destroy(gw);
}

namespace {

thread_local std::string g_create_error;

dc_status fail(dc_ctx *ctx, dc_status st, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return st;
}

dc_status cuda_fail(dc_ctx *ctx, cudaError_t e, const char *where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return fail(ctx, DC_ERR_OOM, m);
    if (e == cudaErrorTimeout) return fail(ctx, DC_ERR_TIMEOUT, where);   // a bounded device wait gave up
    return fail(ctx, DC_ERR_CUDA, m);
}

#define DC_CK(ctx, expr, where)                        \
    do {                                               \
        cudaError_t e__ = (expr);                      \
        if (e__ != cudaSuccess) return cuda_fail(ctx, e__, where); \
    } while (0)

dc_status check_options(const dc_options &o, std::string &msg) {
    if (o.form < DC_FORM_DENSE64 || o.form > DC_FORM_FMM32) {
        msg = "options: unknown form";
        return DC_ERR_ARG;
    }
    if (o.g < 1 || o.g > dc::kMaxG) {
        msg = "options: g must be in [1, 32]";
        return DC_ERR_ARG;
    }
    if (o.s_per_panel < o.g || o.s_per_panel > 4096) {
        msg = "options: s_per_panel must be in [g, 4096]";
        return DC_ERR_ARG;
    }
    if (o.p < 1 || o.p > dc::kMaxP) {
        msg = "options: p must be in [1, 40]";
        return DC_ERR_ARG;
    }
    if (o.leaf_size < 1 || o.leaf_size > 4096) {
        msg = "options: leaf_size must be in [1, 4096]";
        return DC_ERR_ARG;
    }
    if (o.max_depth < 1 || o.max_depth > 40) {
        msg = "options: max_depth must be in [1, 40]";
        return DC_ERR_ARG;
    }
    if (!(o.gmres_tol > 0.0) || o.gmres_restart < 1 || o.gmres_max_iter < 1 ||
        o.gmres_restart > 4096) {
        msg = "options: need gmres_tol > 0, 1 <= gmres_restart <= 4096, gmres_max_iter >= 1";
        return DC_ERR_ARG;
    }
    if (o.x0_mode < DC_X0_ONES || o.x0_mode > DC_X0_LEARNED) {
        msg = "options: unknown x0_mode";
        return DC_ERR_ARG;
    }
    if (o.p_inner < 0 || o.p_inner > o.p) {
        msg = "options: p_inner must be 0 (default) or in [1, p]";
        return DC_ERR_ARG;
    }
    if (o.m2l_engine != DC_M2L_TENSOR && o.m2l_engine != DC_M2L_CUDA_CORES) {
        msg = "options: m2l_engine must be DC_M2L_TENSOR or DC_M2L_CUDA_CORES";
        return DC_ERR_ARG;
    }
    if (!(o.adapt_ratio >= 0.0) || o.adapt_max_level < 0 || o.adapt_max_level > 30 || o.adapt_min_panels < 0 ||
        o.adapt_min_panels > 1024 || !(o.adapt_max_len >= 0.0)) {
        msg = "options: adapt_ratio, adapt_max_len >= 0, adapt_max_level in [0, 30], adapt_min_panels in [0, 1024]";
        return DC_ERR_ARG;
    }
    if (o.eval_tile < 0 || o.eval_tile > 3) {
        msg = "options: eval_tile must be in [0, 3]";
        return DC_ERR_ARG;
    }
    if (o.aa_levels < 0 || o.aa_levels > 6) {
        msg = "options: aa_levels must be in [0, 6]";
        return DC_ERR_ARG;
    }
    if (o.coarse_max != 0 && (o.coarse_max < 64 || o.coarse_max > 16384 || o.coarse_max % 32 != 0)) {
        msg = "options: coarse_max must be 0 (default) or a multiple of 32 in [64, 16384]";
        return DC_ERR_ARG;
    }
    if (!(o.inner_tol >= 0.0 && o.inner_tol < 1.0)) {
        msg = "options: inner_tol must be 0 (default) or in (0, 1)";
        return DC_ERR_ARG;
    }
    for (double d : o.domain)
        if (!std::isfinite(d)) {
            msg = "options: domain must be finite";
            return DC_ERR_ARG;
        }
    if (!(o.domain[2] >= o.domain[0]) || !(o.domain[3] >= o.domain[1])) {
        msg = "options: domain must have x1 >= x0 and y1 >= y0";
        return DC_ERR_ARG;
    }
    return DC_OK;
}

// Dense operator y = A_G x (plain form).
struct DenseOp : dc::Operator {
    const double *A;
    int N;
    cudaError_t apply(const double *x, double *y, cudaStream_t st) override {
        return dc::launch_dense_gemv(A, N, x, y, st);
    }
};

// FMM operator y = G_H x (Alg. 3, the matvec of GMRES).
struct FmmOp : dc::Operator {
    dc::Fmm *fmm;
    cudaError_t apply(const double *x, double *y, cudaStream_t st) override {
        return fmm->apply_single_layer(x, y, st);
    }
};

// The operator of the local system of Sec. 6.3 (Eq. 27 restricted to the
// re-solving panels r): v -> mask (G_H B (mask v)), with B the panels'
// inverse self-interaction blocks as a right preconditioner in the FMM forms
// (block diagonal, so it keeps the restriction) and none in the dense form.
struct MaskedOp : dc::Operator {
    dc_ctx *ctx = nullptr;
    const unsigned char *pmask = nullptr;
    double *t1 = nullptr, *t2 = nullptr;
    cudaError_t apply(const double *x, double *y, cudaStream_t st) override {
        const int N = ctx->dg.N, g = ctx->dg.g;
        cudaError_t e;
        if ((e = cudaMemcpyAsync(t1, x, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
        if ((e = dc::launch_node_mask(t1, pmask, N, g, st)) != cudaSuccess) return e;
        if (ctx->opt.form == DC_FORM_DENSE64) {
            if ((e = dc::launch_dense_gemv(ctx->AG.ptr, N, t1, y, st)) != cudaSuccess) return e;
        } else {
            if ((e = ctx->fmm->apply_block_jacobi(t1, t2, st)) != cudaSuccess) return e;
            if ((e = ctx->fmm->apply_single_layer(t2, y, st)) != cudaSuccess) return e;
        }
        return dc::launch_node_mask(y, pmask, N, g, st);
    }
};

// The block operator of the mixed problem (Sec. 4.3) with its right
// preconditioner: x holds psi on the Dirichlet panels and u on the Neumann
// panels; y = A M x with
//   M x = B x on Dirichlet panels (the panels' inverse G_H blocks; identity
//         in the dense form), -2 x on Neumann panels,
//   A z = G_H (m_d z) - F_H (m_n z) - (m_n z) / 2.
struct MixedOp : dc::Operator {
    dc_ctx *ctx = nullptr;
    const unsigned char *nmask = nullptr, *dmask = nullptr;   // per panel
    double *t1 = nullptr, *t2 = nullptr, *t3 = nullptr;
    cudaError_t precond(const double *x, double *out, cudaStream_t st) {
        const int N = ctx->dg.N, g = ctx->dg.g;
        cudaError_t e;
        const double *bx = x;
        if (ctx->opt.form != DC_FORM_DENSE64) {
            if ((e = ctx->fmm->apply_block_jacobi(x, t3, st)) != cudaSuccess) return e;
            bx = t3;
        }
        return dc::launch_blend(out, bx, 1.0, x, -2.0, nmask, N, g, st);
    }
    cudaError_t apply_A(const double *z, double *y, cudaStream_t st) {
        const int N = ctx->dg.N, g = ctx->dg.g;
        const bool dense = ctx->opt.form == DC_FORM_DENSE64;
        cudaError_t e;
        if ((e = cudaMemcpyAsync(t2, z, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
            (e = dc::launch_node_mask(t2, dmask, N, g, st)) != cudaSuccess)
            return e;
        e = dense ? dc::launch_dense_gemv(ctx->AG.ptr, N, t2, y, st) : ctx->fmm->apply_single_layer(t2, y, st);
        if (e != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(t2, z, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
            (e = dc::launch_node_mask(t2, nmask, N, g, st)) != cudaSuccess)
            return e;
        e = dense ? dc::launch_dense_gemv(ctx->AF.ptr, N, t2, t3, st) : ctx->fmm->apply_double_layer(t2, t3, st);
        if (e != cudaSuccess) return e;
        const double one[3] = {1, 1, 1}, m1[3] = {-1, -1, -1}, mh[3] = {-0.5, -0.5, -0.5};
        if ((e = dc::vec_combine3(y, t3, y, N, one, m1, st)) != cudaSuccess) return e;
        return dc::vec_combine3(y, t2, y, N, one, mh, st);
    }
    cudaError_t apply(const double *x, double *y, cudaStream_t st) override {
        cudaError_t e = precond(x, t1, st);
        if (e != cudaSuccess) return e;
        return apply_A(t1, y, st);
    }
};

dc_status ensure_segment_density(dc_ctx *ctx) {
    if (ctx->seg_density_valid) return DC_OK;
    DC_CK(ctx, dc::launch_interp(ctx->dg, ctx->sigma.ptr, ctx->sbar.ptr, ctx->stream), "interp");
    DC_CK(ctx, dc::launch_interp(ctx->dg, ctx->mu.ptr, ctx->mbar.ptr, ctx->stream), "interp");
    ctx->seg_density_valid = true;
    return DC_OK;
}

}  // namespace

extern "C" {

int dc_abi_version(void) { return DC_ABI_VERSION; }

long long dc_aux_kernel_launches(void) { return dc::kernel_launches(); }

dc_status dc_aux_tree_check(int n_seg, const double *seg_xy, const double *domain, int leaf_size,
                            int max_depth, double *out) {
    if (n_seg < 0 || (n_seg > 0 && !seg_xy) || !domain || !out || leaf_size < 1 ||
        max_depth < 1 || max_depth > 40)
        return DC_ERR_ARG;
    std::vector<double> seg(seg_xy, seg_xy + 4 * size_t(n_seg));
    for (double v : seg)
        if (!std::isfinite(v)) return DC_ERR_ARG;
    for (int i = 0; i < 4; ++i)
        if (!std::isfinite(domain[i])) return DC_ERR_ARG;
    dc::Tree t;
    std::string msg;
    if (!dc::build_quadtree(seg, domain, leaf_size, max_depth, t, msg)) return DC_ERR_GEOMETRY;
    out[0] = t.n_cells();
    out[1] = t.n_leaves();
    out[2] = t.depth;
    out[3] = double(t.pc_seg.size());
    out[4] = double(dc::check_quadtree_routes(t));
    std::vector<double> sum(n_seg, 0.0);
    for (size_t i = 0; i < t.pc_seg.size(); ++i) {
        const double *q = &t.pc_xy[4 * i];
        sum[t.pc_seg[i]] += std::hypot(q[2] - q[0], q[3] - q[1]);
    }
    double worst = 0.0;
    for (int k = 0; k < n_seg; ++k) {
        const double *q = &seg[4 * size_t(k)];
        double L = std::hypot(q[2] - q[0], q[3] - q[1]);
        if (L > 0) worst = std::max(worst, std::fabs(sum[k] - L) / L);
    }
    out[5] = worst;
    return DC_OK;
}

const char *dc_status_string(dc_status st) {
    switch (st) {
        case DC_OK: return "ok";
        case DC_ERR_ARG: return "invalid argument";
        case DC_ERR_STATE: return "call out of order";
        case DC_ERR_CUDA: return "CUDA error";
        case DC_ERR_OOM: return "out of memory";
        case DC_ERR_NOCONV: return "GMRES did not converge";
        case DC_ERR_TIMEOUT: return "device wait timed out";
        case DC_ERR_GEOMETRY: return "degenerate geometry";
        case DC_ERR_UNSUPPORTED: return "unsupported option combination";
    }
    return "unknown status";
}

const char *dc_last_error(dc_ctx *ctx) {
    if (!ctx) return g_create_error.c_str();
    return ctx->err.c_str();
}

dc_status dc_default_options(dc_options *opt) {
    if (!opt) return DC_ERR_ARG;
    std::memset(opt, 0, sizeof(*opt));
    opt->form = DC_FORM_FMM32;
    opt->g = 16;
    opt->s_per_panel = 80;
    opt->p = 24;
    opt->leaf_size = 64;
    opt->max_depth = 30;
    opt->gmres_tol = 1e-10;
    opt->gmres_restart = 200;
    opt->gmres_max_iter = 2000;
    opt->x0_mode = DC_X0_ONES;
    opt->stream = nullptr;
    opt->domain[0] = 0.0;
    opt->domain[1] = 0.0;
    opt->domain[2] = 1.0;
    opt->domain[3] = 1.0;
    return DC_OK;
}

dc_status dc_create(dc_ctx **out, const dc_options *opt) {
    if (!out) {
        g_create_error = "dc_create: out is NULL";
        return DC_ERR_ARG;
    }
    *out = nullptr;
    dc_options o;
    if (opt) o = *opt;
    else dc_default_options(&o);
    std::string msg;
    dc_status st = check_options(o, msg);
    if (st != DC_OK) {
        g_create_error = msg;
        return st;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        g_create_error = std::string("dc_create: ") + cudaGetErrorString(e);
        return DC_ERR_CUDA;
    }
    dc_ctx *ctx = new (std::nothrow) dc_ctx();
    if (!ctx) {
        g_create_error = "dc_create: host allocation failed";
        return DC_ERR_OOM;
    }
    ctx->opt = o;
    ctx->device = dev;
    ctx->stream = static_cast<cudaStream_t>(o.stream);
    ctx->gw = dc::gmres_work_create();
    *out = ctx;
    return DC_OK;
}

void dc_destroy(dc_ctx *ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    delete ctx;
}

dc_status dc_build_tree(dc_ctx *ctx, int n_curves, const double *ctrl, const int *panel_ptr,
                        const double *panel_start, const double *colours) {
    if (!ctx) return DC_ERR_ARG;
    ctx->err.clear();
    ctx->state = 0;
    ctx->view_valid = false;
    ctx->seg_density_valid = false;
    std::string msg;
    for (double &v : ctx->build_ms) v = 0.0;
    const auto t_start = std::chrono::steady_clock::now();
    // The previous drawing's buffers are recycled through the context's
    // block cache (no cudaFree / cudaMalloc per buffer): nothing of its may
    // still run, so the device is drained first (as cudaFree would).
    DC_CK(ctx, cudaDeviceSynchronize(), "build_tree");
    dc::PoolScope pool_scope(&ctx->pool);
    auto t_prev = t_start;
    auto lap = [&](int i) {   // the stream drained first
        cudaStreamSynchronize(ctx->stream);
        const auto t = std::chrono::steady_clock::now();
        ctx->build_ms[i] = std::chrono::duration<double, std::milli>(t - t_prev).count();
        t_prev = t;
    };
    std::vector<int> auto_ptr;
    std::vector<double> auto_start;
    if (!panel_ptr && !panel_start) {   // the adaptive panel rule of the options
        if (n_curves < 1 || !ctrl) return fail(ctx, DC_ERR_ARG, "build_tree: need curves");
        for (int i = 0; i < 8 * n_curves; ++i)
            if (!std::isfinite(ctrl[i])) return fail(ctx, DC_ERR_ARG, "build_tree: non-finite control point");
        const dc_options &o = ctx->opt;
        dc_status sa = dc::adaptive_panels(n_curves, ctrl, o.adapt_ratio > 0 ? o.adapt_ratio : 0.2,
                                           o.adapt_max_level > 0 ? o.adapt_max_level : 8,
                                           o.adapt_min_panels > 0 ? o.adapt_min_panels : 2,
                                           o.adapt_max_len > 0 ? o.adapt_max_len : 0.5, auto_ptr, auto_start, msg);
        if (sa != DC_OK) return fail(ctx, sa, msg);
        panel_ptr = auto_ptr.data();
        panel_start = auto_start.data();
    }
    dc_status st = dc::discretise(n_curves, ctrl, panel_ptr, panel_start, colours, ctx->opt.g,
                                  ctx->opt.s_per_panel, ctx->geo, msg);
    if (st != DC_OK) return fail(ctx, st, msg);
    {   // keep the inputs for dc_subdivide (copies first: they may alias)
        const int np = panel_ptr[n_curves];
        std::vector<double> c(ctrl, ctrl + 8 * (size_t)n_curves), ps(panel_start, panel_start + np),
            col(colours, colours + 12 * (size_t)n_curves);
        std::vector<int> pp(panel_ptr, panel_ptr + n_curves + 1);
        ctx->in_ncurves = n_curves;
        ctx->in_ctrl.swap(c);
        ctx->in_start.swap(ps);
        ctx->in_col.swap(col);
        ctx->in_ptr.swap(pp);
    }
    lap(0);
    const dc::Geometry &G = ctx->geo;
    dc::DevGeom &D = ctx->dg;
    D.N = G.n_nodes();
    D.S = G.n_segments();
    D.g = G.g;
    D.s = G.s;
    D.n_panels = G.n_panels;
    cudaStream_t s = ctx->stream;
    // buffers of the previous drawing are reused when large enough
    auto up = [&](auto &buf, const auto &vec, const char *what) -> dc_status {
        DC_CK(ctx, buf.ensure(vec.size()), what);
        DC_CK(ctx,
              cudaMemcpyAsync(buf.ptr, vec.data(), vec.size() * sizeof(vec[0]),
                              cudaMemcpyHostToDevice, s),
              what);
        return DC_OK;
    };
    if ((st = up(D.seg, G.seg_xy, "upload segments")) != DC_OK) return st;
    if ((st = up(D.segw, G.seg_w, "upload weights")) != DC_OK) return st;
    if ((st = up(D.node_xy, G.node_xy, "upload nodes")) != DC_OK) return st;
    if ((st = up(D.node_seg, G.node_seg, "upload nodes")) != DC_OK) return st;
    if ((st = up(D.node_seg2, G.node_seg2, "upload nodes")) != DC_OK) return st;
    if ((st = up(D.lambda, G.lambda, "upload interpolation")) != DC_OK) return st;
    if ((st = up(D.u_plus, G.u_plus, "upload colours")) != DC_OK) return st;
    if ((st = up(D.u_minus, G.u_minus, "upload colours")) != DC_OK) return st;
    size_t n3 = size_t(3) * D.N, s3 = size_t(3) * D.S;
    DC_CK(ctx, ctx->mu.ensure(n3), "alloc");
    DC_CK(ctx, ctx->sigma.ensure(n3), "alloc");
    DC_CK(ctx, ctx->b.ensure(n3), "alloc");
    DC_CK(ctx, ctx->fmu.ensure(n3), "alloc");
    DC_CK(ctx, ctx->sbar.ensure(s3), "alloc");
    DC_CK(ctx, ctx->mbar.ensure(s3), "alloc");
    DC_CK(ctx, dc::launch_mu(D, ctx->mu.ptr, s), "mu");
    lap(1);
    ctx->AG.release();
    ctx->AF.release();
    ctx->fmm.reset();
    if (ctx->opt.form == DC_FORM_DENSE64) {
        if (!ctx->render_only) {
            size_t nn = size_t(D.N) * D.N;
            DC_CK(ctx, ctx->AG.alloc(nn), "alloc dense A_G");
            DC_CK(ctx, ctx->AF.alloc(nn), "alloc dense A_F");
            DC_CK(ctx, dc::launch_dense_assemble(D, ctx->AG.ptr, ctx->AF.ptr, s), "dense assembly");
        }
    } else {
        ctx->fmm.reset(new (std::nothrow) dc::Fmm());
        if (!ctx->fmm) return fail(ctx, DC_ERR_OOM, "build_tree: host allocation failed");
        ctx->fmm->set_render_only(ctx->render_only);
        st = ctx->fmm->build(ctx->opt, G, D, s, msg);
        if (st != DC_OK) {
            ctx->fmm.reset();
            return fail(ctx, st, msg);
        }
        ctx->fmm->build_timings(ctx->build_ms + 2);
    }
    t_prev = std::chrono::steady_clock::now();
    if (ctx->render_only) {   // a view renders: no solve structures
        DC_CK(ctx, cudaStreamSynchronize(s), "build_tree");
        ctx->pool.next_generation();
        ctx->state = 1;
        return DC_OK;
    }
    ctx->feat_built = false;   // the warm start's panel geometry: built on first use
    lap(8);
    ctx->warm_a1_valid = false;
    {   // G_H 1, once per drawing: the first residual of the paper's start
        // x0 = 1 and the learned start's least-residual projection use it
        const int N = ctx->dg.N;
        const double zero[3] = {0, 0, 0}, one[3] = {1, 1, 1};
        DC_CK(ctx, ctx->warm_ax.ensure(size_t(3) * N), "alloc G_H 1");
        DC_CK(ctx, ctx->warm_a1.ensure(size_t(3) * N), "alloc G_H 1");
        DC_CK(ctx, dc::vec_combine3(ctx->warm_ax.ptr, nullptr, ctx->warm_ax.ptr, N, zero, one, s), "G_H 1");
        if (ctx->opt.form == DC_FORM_DENSE64)
            DC_CK(ctx, dc::launch_dense_gemv(ctx->AG.ptr, N, ctx->warm_ax.ptr, ctx->warm_a1.ptr, s), "G_H 1");
        else
            DC_CK(ctx, ctx->fmm->apply_single_layer(ctx->warm_ax.ptr, ctx->warm_a1.ptr, s), "G_H 1");
        ctx->warm_a1_valid = true;
    }
    lap(9);
    DC_CK(ctx, cudaStreamSynchronize(s), "build_tree");
    ctx->build_ms[10] = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    ctx->pool.next_generation();   // blocks no longer taken are freed
    ctx->state = 1;
    return DC_OK;
}

// The panel geometry of the warm-start features, once per drawing.
dc_status ensure_features(dc_ctx *ctx) {
    if (ctx->feat_built) return DC_OK;
    DC_CK(ctx, ctx->pfeat.build(ctx->geo, ctx->stream), "panel features");
    ctx->feat_built = true;
    return DC_OK;
}

// Learned warm start: features -> network -> sigma_p, then per channel the
// x0 = alpha sigma_p + beta 1 of least residual ||b - G_H x0|| (two FP64
// operator applications, G_H 1 cached per drawing).  The span holds 0 and the
// paper's start 1, so the start is never worse than either (cold fallback:
// alpha = 0 when the prediction does not help).
dc_status warm_start(dc_ctx *ctx, dc_solve_stats *stats) {
    if (dc_status fs = ensure_features(ctx); fs != DC_OK) return fs;
    cudaStream_t s = ctx->stream;
    const int N = ctx->dg.N, g = ctx->dg.g;
    const int rows = ctx->pfeat.rows(), F = dc::PanelFeatures::n_features(g), H = ctx->warm_hidden;
    DC_CK(ctx, ctx->warm_feat.ensure(size_t(rows) * F), "alloc features");
    DC_CK(ctx, ctx->warm_pred.ensure(size_t(rows) * g), "alloc prediction");
    DC_CK(ctx, ctx->warm_work.ensure(dc_aux_mlp_workspace_floats(F, H, g, rows)), "alloc network");
    DC_CK(ctx, ctx->warm_ax.ensure(size_t(3) * N), "alloc residual");
    DC_CK(ctx, ctx->warm_a1.ensure(size_t(3) * N), "alloc residual");
    DC_CK(ctx, ctx->pfeat.compute(ctx->dg, nullptr, ctx->warm_feat.ptr, nullptr, s), "features");
    dc_status st = dc_aux_mlp_forward(F, H, g, ctx->warm_params.ptr, rows, ctx->warm_feat.ptr,
                                      ctx->warm_pred.ptr, ctx->warm_work.ptr, s);
    if (st != DC_OK) return fail(ctx, st, "solve_density: warm-start network failed");
    DC_CK(ctx, ctx->pfeat.apply(ctx->warm_pred.ptr, ctx->sigma.ptr, s), "warm start");
    auto apply = [&](const double *x, double *y) -> cudaError_t {
        if (ctx->opt.form == DC_FORM_DENSE64) return dc::launch_dense_gemv(ctx->AG.ptr, N, x, y, s);
        return ctx->fmm->apply_single_layer(x, y, s);
    };
    if (!ctx->warm_a1_valid) return fail(ctx, DC_ERR_STATE, "solve_density: G_H 1 missing");
    DC_CK(ctx, apply(ctx->sigma.ptr, ctx->warm_ax.ptr), "warm start");
    double pp[3], p1[3], q1[3], pb[3], qb[3], bb[3];
    const double *Ap = ctx->warm_ax.ptr, *A1 = ctx->warm_a1.ptr, *b = ctx->b.ptr;
    DC_CK(ctx, dc::vec_dots3(ctx->gw, Ap, Ap, N, pp, s), "warm start");
    DC_CK(ctx, dc::vec_dots3(ctx->gw, Ap, A1, N, p1, s), "warm start");
    DC_CK(ctx, dc::vec_dots3(ctx->gw, A1, A1, N, q1, s), "warm start");
    DC_CK(ctx, dc::vec_dots3(ctx->gw, Ap, b, N, pb, s), "warm start");
    DC_CK(ctx, dc::vec_dots3(ctx->gw, A1, b, N, qb, s), "warm start");
    DC_CK(ctx, dc::vec_dots3(ctx->gw, b, b, N, bb, s), "warm start");
    double al[3], be[3];
    int mask = 0;
    for (int c = 0; c < 3; ++c) {
        double a = 0.0, q = 0.0;
        const double det = pp[c] * q1[c] - p1[c] * p1[c];
        if (det > 1e-12 * pp[c] * q1[c] && det > 0.0) {
            a = (pb[c] * q1[c] - qb[c] * p1[c]) / det;
            q = (pp[c] * qb[c] - p1[c] * pb[c]) / det;
        } else if (q1[c] > 0.0) {
            q = qb[c] / q1[c];          // the prediction adds nothing independent
        }
        if (!std::isfinite(a) || !std::isfinite(q)) a = q = 0.0;
        al[c] = a;
        be[c] = q;
        if (a != 0.0) mask |= 1 << c;
        const double r2 = std::max(0.0, bb[c] - a * pb[c] - q * qb[c]);
        if (stats) stats->warm_resid[c] = bb[c] > 0.0 ? std::sqrt(r2 / bb[c]) : 0.0;
    }
    DC_CK(ctx, dc::vec_combine3(ctx->sigma.ptr, nullptr, ctx->sigma.ptr, N, al, be, s), "warm start");
    // G_H x0 = alpha G_H sigma_p + beta G_H 1, for the first residual
    DC_CK(ctx, dc::vec_combine3(ctx->warm_ax.ptr, ctx->warm_a1.ptr, ctx->warm_ax.ptr, N, al, be, s), "warm start");
    if (stats) stats->used_warm = mask;
    return DC_OK;
}

dc_status dc_solve_density(dc_ctx *ctx, const double *x0, dc_solve_stats *stats) {
    if (!ctx) return DC_ERR_ARG;
    ctx->err.clear();
    if (ctx->state < 1) return fail(ctx, DC_ERR_STATE, "solve_density: call build_tree first");
    if (ctx->render_only) return fail(ctx, DC_ERR_STATE, "solve_density: a view context renders only");
    ctx->view_valid = false;
    if (ctx->opt.x0_mode == DC_X0_USER && !x0)
        return fail(ctx, DC_ERR_ARG, "solve_density: x0_mode is DC_X0_USER but x0 is NULL");
    if (ctx->opt.x0_mode == DC_X0_LEARNED && ctx->warm_hidden <= 0)
        return fail(ctx, DC_ERR_STATE, "solve_density: DC_X0_LEARNED needs a warm-start model");
    const int N = ctx->dg.N;
    cudaStream_t s = ctx->stream;
    if (stats) std::memset(stats, 0, sizeof(*stats));
    cudaEvent_t e0, e1;
    DC_CK(ctx, cudaEventCreate(&e0), "event");
    DC_CK(ctx, cudaEventCreate(&e1), "event");
    struct EvGuard {
        cudaEvent_t a, b;
        ~EvGuard() {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } guard{e0, e1};
    DC_CK(ctx, cudaEventRecord(e0, s), "event");
    if (ctx->mu_custom) {   // dc_solve_mixed set mu; the two-sided problem takes it from the colours
        DC_CK(ctx, dc::launch_mu(ctx->dg, ctx->mu.ptr, s), "mu");
        ctx->mu_custom = false;
    }
    // b = (u+ + u-)/2 - F_H mu  (Alg. 3)
    if (ctx->opt.form == DC_FORM_DENSE64) {
        DC_CK(ctx, dc::launch_dense_gemv(ctx->AF.ptr, N, ctx->mu.ptr, ctx->fmu.ptr, s), "rhs");
    } else {
        DC_CK(ctx, ctx->fmm->apply_double_layer(ctx->mu.ptr, ctx->fmu.ptr, s), "rhs");
    }
    DC_CK(ctx, dc::launch_rhs(ctx->dg, ctx->fmu.ptr, ctx->b.ptr, s), "rhs");
    DC_CK(ctx, cudaEventRecord(e1, s), "event");
    auto t0 = std::chrono::steady_clock::now();   // x0 (warm start included) and GMRES
    size_t n3b = size_t(3) * N * sizeof(double);
    if (ctx->opt.x0_mode == DC_X0_USER) {
        for (size_t i = 0; i < size_t(3) * N; ++i)
            if (!std::isfinite(x0[i])) return fail(ctx, DC_ERR_ARG, "solve_density: non-finite x0");
        DC_CK(ctx, cudaMemcpyAsync(ctx->sigma.ptr, x0, n3b, cudaMemcpyHostToDevice, s), "x0");
    } else if (ctx->opt.x0_mode == DC_X0_ZEROS) {
        DC_CK(ctx, cudaMemsetAsync(ctx->sigma.ptr, 0, n3b, s), "x0");
    } else if (ctx->opt.x0_mode == DC_X0_LEARNED) {
        auto w0 = std::chrono::steady_clock::now();
        dc_status ws = warm_start(ctx, stats);
        if (ws != DC_OK) return ws;
        if (stats)
            stats->ms_warm =
                std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - w0).count();
    } else {   // the paper's x0 = 1
        const double zero[3] = {0, 0, 0}, one[3] = {1, 1, 1};
        DC_CK(ctx, dc::vec_combine3(ctx->sigma.ptr, nullptr, ctx->sigma.ptr, N, zero, one, s), "x0");
    }
    // G_H x0 where it is known without an operator application
    const double *Ax0 = nullptr;
    if (ctx->opt.x0_mode == DC_X0_ONES && ctx->warm_a1_valid) Ax0 = ctx->warm_a1.ptr;
    if (ctx->opt.x0_mode == DC_X0_LEARNED) Ax0 = ctx->warm_ax.ptr;
    ctx->seg_density_valid = false;
    dc::GmresResult gr;
    std::string msg;
    cudaError_t ce;
    int n_refine = 0;
    if (ctx->opt.form == DC_FORM_DENSE64) {
        DenseOp op;
        op.A = ctx->AG.ptr;
        op.N = N;
        ce = dc::gmres_solve(ctx->gw, op, N, ctx->b.ptr, ctx->sigma.ptr, false, false, ctx->opt.gmres_tol,
                             ctx->opt.gmres_restart, ctx->opt.gmres_max_iter, s, gr, msg);
    } else {
        ce = ctx->fmm->solve(ctx->gw, ctx->b.ptr, ctx->sigma.ptr, ctx->opt, s, gr, msg, &n_refine, Ax0);
    }
    if (ce != cudaSuccess) return cuda_fail(ctx, ce, msg.empty() ? "gmres" : msg.c_str());
    DC_CK(ctx, cudaStreamSynchronize(s), "gmres");
    auto t1 = std::chrono::steady_clock::now();
    if (stats) {
        for (int c = 0; c < 3; ++c) {
            stats->iters[c] = gr.iters[c];
            stats->rel_resid[c] = gr.rel_resid[c];
            stats->true_rel_resid[c] = gr.true_rel_resid[c];
        }
        stats->converged = gr.converged;
        stats->n_matvec = gr.n_matvec + 1;
        stats->n_refine = n_refine;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        stats->ms_rhs = ms;
        stats->ms_solve = std::chrono::duration<double, std::milli>(t1 - t0).count();
        if (ctx->fmm) {
            stats->p2p_pairs = ctx->fmm->p2p_pairs_nodes();
            stats->m2l_pairs = ctx->fmm->m2l_pairs();
        }
    }
    ctx->state = 2;
    if (!gr.converged)
        return fail(ctx, DC_ERR_NOCONV, "solve_density: gmres_max_iter reached before gmres_tol");
    return DC_OK;
}

dc_status dc_set_density(dc_ctx *ctx, const double *sigma_in) {
    if (!ctx) return DC_ERR_ARG;
    ctx->err.clear();
    if (ctx->state < 1) return fail(ctx, DC_ERR_STATE, "set_density: call build_tree first");
    if (!sigma_in) return fail(ctx, DC_ERR_ARG, "set_density: NULL input");
    ctx->view_valid = false;
    size_t n3 = size_t(3) * ctx->dg.N;
    for (size_t i = 0; i < n3; ++i)
        if (!std::isfinite(sigma_in[i]))
            return fail(ctx, DC_ERR_ARG, "set_density: non-finite value");
    DC_CK(ctx,
          cudaMemcpyAsync(ctx->sigma.ptr, sigma_in, n3 * sizeof(double), cudaMemcpyHostToDevice,
                          ctx->stream),
          "set_density");
    DC_CK(ctx, cudaStreamSynchronize(ctx->stream), "set_density");
    ctx->seg_density_valid = false;
    ctx->state = 2;
    return DC_OK;
}

dc_status dc_eval_points_noalloc(dc_ctx *ctx, int n, const double *xy_dev, double *out_dev) {
    if (!ctx) return DC_ERR_ARG;
    ctx->err.clear();
    if (ctx->state < 2) return fail(ctx, DC_ERR_STATE, "eval_points_noalloc: no density yet");
    if (n < 0 || (n > 0 && (!xy_dev || !out_dev)))
        return fail(ctx, DC_ERR_ARG, "eval_points_noalloc: bad arguments");
    if (n == 0) return DC_OK;
    int cur = -1;
    DC_CK(ctx, cudaGetDevice(&cur), "eval_points_noalloc");
    if (cur != ctx->device)
        return fail(ctx, DC_ERR_STATE, "eval_points_noalloc: the current CUDA device is not the context's device");
    std::string msg;
    cudaError_t e = dc::eval_points_noalloc(ctx->dg, ctx->sigma.ptr, ctx->mu.ptr, xy_dev, n, out_dev,
                                            ctx->stream, msg);
    if (e == cudaErrorInvalidValue && !msg.empty()) return fail(ctx, DC_ERR_ARG, msg);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "eval_points_noalloc");
    return DC_OK;
}

dc_status dc_get_density(dc_ctx *ctx, double *sigma_out) {
    if (!ctx) return DC_ERR_ARG;
    ctx->err.clear();
    if (ctx->state < 2) return fail(ctx, DC_ERR_STATE, "get_density: no density yet");
    if (!sigma_out) return fail(ctx, DC_ERR_ARG, "get_density: NULL output");
    size_t n3 = size_t(3) * ctx->dg.N;
    DC_CK(ctx,
          cudaMemcpyAsync(sigma_out, ctx->sigma.ptr, n3 * sizeof(double), cudaMemcpyDeviceToHost,
                          ctx->stream),
          "get_density");
    DC_CK(ctx, cudaStreamSynchronize(ctx->stream), "get_density");
    return DC_OK;
}

dc_status dc_get_nodes(dc_ctx *ctx, double *xy, double *t, double *u_plus, double *u_minus) {
    if (!ctx) return DC_ERR_ARG;
    ctx->err.clear();
    if (ctx->state < 1) return fail(ctx, DC_ERR_STATE, "get_nodes: call build_tree first");
    const dc::Geometry &G = ctx->geo;
    if (xy) std::memcpy(xy, G.node_xy.data(), G.node_xy.size() * sizeof(double));
    if (t) std::memcpy(t, G.node_t.data(), G.node_t.size() * sizeof(double));
    if (u_plus) std::memcpy(u_plus, G.u_plus.data(), G.u_plus.size() * sizeof(double));
    if (u_minus) std::memcpy(u_minus, G.u_minus.data(), G.u_minus.size() * sizeof(double));
    return DC_OK;
}

dc_status dc_get_sizes(dc_ctx *ctx, dc_sizes *out) {
    if (!ctx || !out) return DC_ERR_ARG;
    std::memset(out, 0, sizeof(*out));
    if (ctx->state < 1) return fail(ctx, DC_ERR_STATE, "get_sizes: call build_tree first");
    out->n_curves = ctx->geo.n_curves;
    out->n_panels = ctx->geo.n_panels;
    out->n_nodes = ctx->geo.n_nodes();
    out->n_segments = ctx->geo.n_segments();
    if (ctx->fmm) ctx->fmm->fill_sizes(out);
    else out->n_pieces = out->n_segments;
    return DC_OK;
}

dc_status dc_render_viewport(dc_ctx *ctx, int n_vp, const dc_viewport *vps, void *rgb,
                             int rgb_dtype, unsigned char *rgb8, int out_where,
                             dc_render_stats *stats) {
    if (!ctx) return DC_ERR_ARG;
    ctx->err.clear();
    if (ctx->state < 2) return fail(ctx, DC_ERR_STATE, "render_viewport: no density yet");
    if (n_vp < 0 || (n_vp > 0 && !vps)) return fail(ctx, DC_ERR_ARG, "render_viewport: bad viewports");
    if (rgb && rgb_dtype != DC_F32 && rgb_dtype != DC_F64)
        return fail(ctx, DC_ERR_ARG, "render_viewport: rgb_dtype must be DC_F32 or DC_F64");
    if (out_where != DC_MEM_DEVICE && out_where != DC_MEM_HOST)
        return fail(ctx, DC_ERR_ARG, "render_viewport: out_where must be DC_MEM_DEVICE or DC_MEM_HOST");
    long long total = 0;
    for (int v = 0; v < n_vp; ++v) {
        const dc_viewport &vp = vps[v];
        if (vp.width < 0 || vp.height < 0 || vp.width > 65536 || vp.height > 65536)
            return fail(ctx, DC_ERR_ARG, "render_viewport: width/height must be in [0, 65536]");
        if (!std::isfinite(vp.x0) || !std::isfinite(vp.x1) || !std::isfinite(vp.y0) ||
            !std::isfinite(vp.y1))
            return fail(ctx, DC_ERR_ARG, "render_viewport: non-finite viewport");
        total += (long long)vp.width * vp.height;
    }
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (total == 0) return DC_OK;
    if (ctx->view && ctx->view_valid) {   // the viewport's evaluation polyline (Sec. 6.2)
        dc_status vs = dc_render_viewport(ctx->view, n_vp, vps, rgb, rgb_dtype, rgb8, out_where, stats);
        if (vs != DC_OK) return fail(ctx, vs, ctx->view->err);
        return DC_OK;
    }
    cudaStream_t s = ctx->stream;
    dc_status st = ensure_segment_density(ctx);
    if (st != DC_OK) return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (stats) {
        DC_CK(ctx, cudaEventCreate(&e0), "event");
        DC_CK(ctx, cudaEventCreate(&e1), "event");
        DC_CK(ctx, cudaEventRecord(e0, s), "event");
    }
    // destination buffers (device staging when the caller gave host memory)
    size_t esz = (rgb_dtype == DC_F64) ? sizeof(double) : sizeof(float);
    void *drgb = rgb;
    unsigned char *drgb8 = rgb8;
    if (out_where == DC_MEM_HOST) {
        if (rgb) {
            DC_CK(ctx, ctx->stage64.ensure((size_t(3) * total * esz + 7) / 8), "alloc staging");
            drgb = ctx->stage64.ptr;
        }
        if (rgb8) {
            DC_CK(ctx, ctx->stage8.ensure(size_t(3) * total), "alloc staging");
            drgb8 = ctx->stage8.ptr;
        }
    }
    if (ctx->fmm) {
        ctx->fmm->set_eval_timing(stats != nullptr);
        DC_CK(ctx, ctx->fmm->prepare_eval(ctx->sbar.ptr, ctx->mbar.ptr, s), "fmm passes");
    }
    double dense_eval_ms = 0.0;
    std::vector<dc::VpDev> vl;
    long long off = 0;
    for (int v = 0; v < n_vp; ++v) {
        const dc_viewport &vp = vps[v];
        long long np = (long long)vp.width * vp.height;
        dc::VpDev d;
        d.x0 = vp.x0;
        d.y0 = vp.y0;
        d.dx = vp.width > 0 ? (vp.x1 - vp.x0) / vp.width : 0.0;
        d.dy = vp.height > 0 ? (vp.y1 - vp.y0) / vp.height : 0.0;
        d.width = vp.width;
        d.height = vp.height;
        d.offset = off;
        vl.push_back(d);
        off += np;
    }
    if (ctx->opt.form == DC_FORM_DENSE64) {
        for (int v = 0; v < n_vp; ++v) {
            const dc::VpDev &d = vl[v];
            long long np = (long long)d.width * d.height;
            if (np == 0) continue;
            void *orgb = drgb ? static_cast<char *>(drgb) + size_t(3) * d.offset * esz : nullptr;
            unsigned char *orgb8 = drgb8 ? drgb8 + size_t(3) * d.offset : nullptr;
            DC_CK(ctx, ctx->u64.ensure(size_t(3) * np), "alloc");
            if (stats) DC_CK(ctx, cudaEventRecord(e1, s), "event");
            DC_CK(ctx,
                  dc::launch_dense_eval_grid(ctx->dg, ctx->sbar.ptr, ctx->mbar.ptr, d,
                                             ctx->u64.ptr, s),
                  "dense render");
            if (stats) {
                cudaEvent_t e2;
                DC_CK(ctx, cudaEventCreate(&e2), "event");
                DC_CK(ctx, cudaEventRecord(e2, s), "event");
                DC_CK(ctx, cudaEventSynchronize(e2), "event");
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e1, e2);
                cudaEventDestroy(e2);
                dense_eval_ms += ms;
            }
            DC_CK(ctx, dc::launch_write_outputs(ctx->u64.ptr, np, orgb, rgb_dtype, orgb8, s),
                  "outputs");
        }
    } else {
        std::string msg;
        dc_status fs = ctx->fmm->render_viewports(vl.data(), n_vp, ctx->sbar.ptr, ctx->mbar.ptr, drgb,
                                                  rgb_dtype, drgb8, s, msg);
        if (fs != DC_OK) return fail(ctx, fs, msg);
    }
    // quadtree anti-aliasing (Sec. 7): refined pixels overwrite their centre samples
    double aa_ms = 0.0;
    if (ctx->opt.aa_levels > 0 && (drgb || drgb8)) {
        if (n_vp > 65535) return fail(ctx, DC_ERR_ARG, "render_viewport: anti-aliasing takes at most 65535 viewports");
        cudaEvent_t a0 = nullptr, a1 = nullptr;
        if (stats) {
            DC_CK(ctx, cudaEventCreate(&a0), "event");
            DC_CK(ctx, cudaEventCreate(&a1), "event");
            DC_CK(ctx, cudaEventRecord(a0, s), "event");
        }
        std::string msg;
        cudaError_t ce = ctx->aa.prepare(ctx->dg, vl.data(), n_vp, total, ctx->opt.aa_levels, s, msg);
        if (ce != cudaSuccess) {
            if (!msg.empty()) return fail(ctx, DC_ERR_ARG, msg);
            return cuda_fail(ctx, ce, "anti-aliasing");
        }
        if (ctx->aa.n_samples > 0) {
            if (ctx->opt.form == DC_FORM_DENSE64) {
                DC_CK(ctx,
                      dc::launch_dense_eval_points(ctx->dg, ctx->sbar.ptr, ctx->mbar.ptr, ctx->aa.sxy.ptr,
                                                   ctx->aa.n_samples, ctx->aa.u.ptr, s),
                      "anti-aliasing samples");
            } else {
                dc_status fs = ctx->fmm->eval_points_dev(ctx->aa.sxy.ptr, ctx->aa.n_samples, ctx->sbar.ptr,
                                                         ctx->mbar.ptr, ctx->aa.u.ptr, s, msg);
                if (fs != DC_OK) return fail(ctx, fs, msg);
            }
            DC_CK(ctx, ctx->aa.finish(drgb, rgb_dtype, drgb8, s), "anti-aliasing");
        }
        if (stats) {
            DC_CK(ctx, cudaEventRecord(a1, s), "event");
            DC_CK(ctx, cudaEventSynchronize(a1), "event");
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a0, a1);
            aa_ms = ms;
            cudaEventDestroy(a0);
            cudaEventDestroy(a1);
        }
    }
    if (out_where == DC_MEM_HOST) {
        if (rgb)
            DC_CK(ctx,
                  cudaMemcpyAsync(rgb, drgb, size_t(3) * total * esz, cudaMemcpyDeviceToHost, s),
                  "copy out");
        if (rgb8)
            DC_CK(ctx, cudaMemcpyAsync(rgb8, drgb8, size_t(3) * total, cudaMemcpyDeviceToHost, s),
                  "copy out");
        DC_CK(ctx, cudaStreamSynchronize(s), "render");
    }
    if (stats) {
        DC_CK(ctx, cudaEventRecord(e1, s), "event");
        DC_CK(ctx, cudaEventSynchronize(e1), "event");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        stats->ms = ms;
        stats->pixels = total;
        if (ctx->opt.aa_levels > 0) {
            stats->aa_pixels = ctx->aa.n_edge;
            stats->aa_samples = ctx->aa.n_samples;
            stats->ms_aa = aa_ms;
        }
        if (ctx->fmm) {
            stats->p2p_pairs = ctx->fmm->last_render_p2p_pairs();
            stats->m2p_pairs = ctx->fmm->last_render_m2p_pairs();
            stats->m2l_pairs = ctx->fmm->m2l_pairs();
            stats->eval_flops = ctx->fmm->last_render_eval_flops();
            stats->ms_eval = ctx->fmm->last_render_eval_ms();
            ctx->fmm->set_eval_timing(false);
        } else {
            stats->p2p_pairs = total * (long long)ctx->dg.S;
            stats->eval_flops = 45.0 * double(stats->p2p_pairs);
            stats->ms_eval = dense_eval_ms;
        }
    }
    DC_CK(ctx, cudaGetLastError(), "render");
    return DC_OK;
}

dc_status dc_eval_points(dc_ctx *ctx, int n, const void *xy, int xy_where, void *out,
                         int out_dtype, int out_where) {
    if (!ctx) return DC_ERR_ARG;
    ctx->err.clear();
    if (ctx->state < 2) return fail(ctx, DC_ERR_STATE, "eval_points: no density yet");
    if (n < 0 || (n > 0 && (!xy || !out)))
        return fail(ctx, DC_ERR_ARG, "eval_points: bad arguments");
    if (out_dtype != DC_F32 && out_dtype != DC_F64)
        return fail(ctx, DC_ERR_ARG, "eval_points: out_dtype must be DC_F32 or DC_F64");
    if ((xy_where != DC_MEM_DEVICE && xy_where != DC_MEM_HOST) ||
        (out_where != DC_MEM_DEVICE && out_where != DC_MEM_HOST))
        return fail(ctx, DC_ERR_ARG, "eval_points: bad memory kind");
    if (n == 0) return DC_OK;
    cudaStream_t s = ctx->stream;
    dc_status st = ensure_segment_density(ctx);
    if (st != DC_OK) return st;
    const double *dxy = static_cast<const double *>(xy);
    if (xy_where == DC_MEM_HOST) {
        const double *h = static_cast<const double *>(xy);
        for (int i = 0; i < 2 * n; ++i)
            if (!std::isfinite(h[i])) return fail(ctx, DC_ERR_ARG, "eval_points: non-finite point");
        DC_CK(ctx, ctx->xy.ensure(size_t(2) * n), "alloc");
        DC_CK(ctx, cudaMemcpyAsync(ctx->xy.ptr, h, size_t(2) * n * sizeof(double),
                                   cudaMemcpyHostToDevice, s),
              "copy points");
        dxy = ctx->xy.ptr;
    }
    size_t esz = (out_dtype == DC_F64) ? sizeof(double) : sizeof(float);
    void *dout = out;
    if (out_where == DC_MEM_HOST) {
        DC_CK(ctx, ctx->stage64.ensure((size_t(3) * n * esz + 7) / 8), "alloc staging");
        dout = ctx->stage64.ptr;
    }
    if (ctx->opt.form == DC_FORM_DENSE64) {
        DC_CK(ctx, ctx->u64.ensure(size_t(3) * n), "alloc");
        DC_CK(ctx,
              dc::launch_dense_eval_points(ctx->dg, ctx->sbar.ptr, ctx->mbar.ptr, dxy, n,
                                           ctx->u64.ptr, s),
              "dense eval");
        DC_CK(ctx, dc::launch_write_outputs(ctx->u64.ptr, n, dout, out_dtype, nullptr, s),
              "outputs");
    } else {
        std::string msg;
        DC_CK(ctx, ctx->fmm->prepare_eval(ctx->sbar.ptr, ctx->mbar.ptr, s), "fmm passes");
        dc_status fs =
            ctx->fmm->eval_points(dxy, n, ctx->sbar.ptr, ctx->mbar.ptr, dout, out_dtype, s, msg);
        if (fs != DC_OK) return fail(ctx, fs, msg);
    }
    if (out_where == DC_MEM_HOST) {
        DC_CK(ctx, cudaMemcpyAsync(out, dout, size_t(3) * n * esz, cudaMemcpyDeviceToHost, s),
              "copy out");
        DC_CK(ctx, cudaStreamSynchronize(s), "eval_points");
    }
    DC_CK(ctx, cudaGetLastError(), "eval_points");
    return DC_OK;
}

dc_status dc_aux_feature_dims(dc_ctx *ctx, int *rows, int *n_features, int *n_out) {
    if (!ctx) return DC_ERR_ARG;
    ctx->err.clear();
    if (ctx->state < 1) return fail(ctx, DC_ERR_STATE, "feature_dims: call build_tree first");
    if (dc_status fs = ensure_features(ctx); fs != DC_OK) return fs;
    if (rows) *rows = ctx->pfeat.rows();
    if (n_features) *n_features = dc::PanelFeatures::n_features(ctx->dg.g);
    if (n_out) *n_out = ctx->dg.g;
    return DC_OK;
}

dc_status dc_aux_panel_features(dc_ctx *ctx, float *feat_dev, float *target_dev) {
    if (!ctx) return DC_ERR_ARG;
    ctx->err.clear();
    if (ctx->state < 1) return fail(ctx, DC_ERR_STATE, "panel_features: call build_tree first");
    if (dc_status fs = ensure_features(ctx); fs != DC_OK) return fs;
    if (target_dev && ctx->state < 2)
        return fail(ctx, DC_ERR_STATE, "panel_features: targets need a density");
    if (!feat_dev) return fail(ctx, DC_ERR_ARG, "panel_features: NULL feature buffer");
    DC_CK(ctx,
          ctx->pfeat.compute(ctx->dg, target_dev ? ctx->sigma.ptr : nullptr, feat_dev, target_dev,
                             ctx->stream),
          "panel_features");
    return DC_OK;
}

dc_status dc_aux_set_warm_start_model(dc_ctx *ctx, int hidden, const float *params, int where) {
    if (!ctx) return DC_ERR_ARG;
    ctx->err.clear();
    if (hidden == 0) {
        ctx->warm_hidden = 0;
        ctx->warm_params.release();
        return DC_OK;
    }
    if (hidden < 1 || hidden > 4096 || !params || (where != DC_MEM_HOST && where != DC_MEM_DEVICE))
        return fail(ctx, DC_ERR_ARG, "set_warm_start_model: bad arguments");
    const int g = ctx->opt.g;
    size_t n = dc_aux_mlp_param_count(dc::PanelFeatures::n_features(g), hidden, g);
    if (where == DC_MEM_HOST)
        for (size_t i = 0; i < n; ++i)
            if (!std::isfinite(params[i]))
                return fail(ctx, DC_ERR_ARG, "set_warm_start_model: non-finite parameter");
    DC_CK(ctx, ctx->warm_params.alloc(n), "alloc model");
    DC_CK(ctx,
          cudaMemcpyAsync(ctx->warm_params.ptr, params, n * sizeof(float),
                          where == DC_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                          ctx->stream),
          "copy model");
    DC_CK(ctx, cudaStreamSynchronize(ctx->stream), "copy model");
    ctx->warm_hidden = hidden;
    return DC_OK;
}

dc_status dc_aux_apply_operator(dc_ctx *ctx, int op, int inner, const double *x, double *y) {
    if (!ctx) return DC_ERR_ARG;
    ctx->err.clear();
    if (ctx->state < 1) return fail(ctx, DC_ERR_STATE, "apply_operator: call build_tree first");
    if ((op != 0 && op != 1) || !x || !y || x == y)
        return fail(ctx, DC_ERR_ARG, "apply_operator: need op 0 or 1 and distinct x, y");
    if (inner < 0 || inner > 3) return fail(ctx, DC_ERR_ARG, "apply_operator: inner must be 0..3");
    if (inner == 3 && (!ctx->fmm || op != 0))
        return fail(ctx, DC_ERR_UNSUPPORTED, "apply_operator: inner 3 needs an FMM form and op 0");
    if ((inner == 1 || inner == 2) && (ctx->opt.form != DC_FORM_FMM32 || op != 0))
        return fail(ctx, DC_ERR_UNSUPPORTED, "apply_operator: inner needs DC_FORM_FMM32 and op 0");
    cudaStream_t s = ctx->stream;
    const int N = ctx->dg.N;
    if (ctx->opt.form == DC_FORM_DENSE64) {
        DC_CK(ctx, dc::launch_dense_gemv(op == 0 ? ctx->AG.ptr : ctx->AF.ptr, N, x, y, s), "apply_operator");
    } else if (inner == 3) {
        DC_CK(ctx, ctx->fmm->apply_precond(x, y, s), "apply_operator");
    } else if (inner == 2) {
        DC_CK(ctx, ctx->fmm->apply_inner_raw(x, y, s), "apply_operator");
    } else if (inner) {
        DC_CK(ctx, ctx->fmm->apply_inner(x, y, s), "apply_operator");
    } else if (op == 0) {
        DC_CK(ctx, ctx->fmm->apply_single_layer(x, y, s), "apply_operator");
    } else {
        DC_CK(ctx, ctx->fmm->apply_double_layer(x, y, s), "apply_operator");
    }
    return DC_OK;
}

dc_status dc_aux_build_timings(dc_ctx *ctx, double *out) {
    if (!ctx) return DC_ERR_ARG;
    ctx->err.clear();
    if (!out) return fail(ctx, DC_ERR_ARG, "build_timings: NULL output");
    if (ctx->state < 1) return fail(ctx, DC_ERR_STATE, "build_timings: call build_tree first");
    for (int i = 0; i < 11; ++i) out[i] = ctx->build_ms[i];
    return DC_OK;
}

dc_status dc_aux_precond_info(dc_ctx *ctx, double *out) {
    if (!ctx) return DC_ERR_ARG;
    ctx->err.clear();
    if (!out) return fail(ctx, DC_ERR_ARG, "precond_info: NULL output");
    if (ctx->state < 1 || !ctx->fmm) return fail(ctx, DC_ERR_STATE, "precond_info: needs an FMM form after build_tree");
    ctx->fmm->precond_info(out);
    return DC_OK;
}

// ------------------------------------------------ adaptive subdivision --
dc_status dc_get_panels(dc_ctx *ctx, int *panel_ptr, double *panel_start) {
    if (!ctx) return DC_ERR_ARG;
    ctx->err.clear();
    if (ctx->state < 1) return fail(ctx, DC_ERR_STATE, "get_panels: call build_tree first");
    if (panel_ptr) std::memcpy(panel_ptr, ctx->in_ptr.data(), sizeof(int) * ctx->in_ptr.size());
    if (panel_start) std::memcpy(panel_start, ctx->in_start.data(), sizeof(double) * ctx->in_start.size());
    return DC_OK;
}

dc_status dc_aux_subdivision_info(dc_ctx *ctx, double *top_old, unsigned char *split_old,
                                  unsigned char *resolve_new) {
    if (!ctx) return DC_ERR_ARG;
    ctx->err.clear();
    if (ctx->last_top.empty()) return fail(ctx, DC_ERR_STATE, "subdivision_info: no dc_subdivide call yet");
    if (top_old) std::memcpy(top_old, ctx->last_top.data(), sizeof(double) * ctx->last_top.size());
    if (split_old) std::memcpy(split_old, ctx->last_split.data(), ctx->last_split.size());
    if (resolve_new) std::memcpy(resolve_new, ctx->last_resolve.data(), ctx->last_resolve.size());
    return DC_OK;
}

// dc_subdivide with an optional mask: only panels p with mask[p] != 0 may
// split (nullptr: all).
dc_status subdivide_impl(dc_ctx *ctx, const dc_subdivide_options *o, const unsigned char *mask,
                         dc_subdivide_stats *stats) {
    using clk = std::chrono::steady_clock;
    auto ms_since = [](clk::time_point a) { return std::chrono::duration<double, std::milli>(clk::now() - a).count(); };
    if (!ctx) return DC_ERR_ARG;
    ctx->err.clear();
    if (!o) return fail(ctx, DC_ERR_ARG, "subdivide: NULL options");
    if (ctx->state < 2) return fail(ctx, DC_ERR_STATE, "subdivide: needs a density (solve_density or set_density)");
    if (!std::isfinite(o->eps_coef) || o->eps_coef < 0.0 || !std::isfinite(o->eps_len) || o->eps_len < 0.0 ||
        o->resolve < DC_RESOLVE_LOCAL || o->resolve > DC_RESOLVE_NONE || !(o->label_ratio >= 0.0) ||
        !(o->label_ratio < 1.0))
        return fail(ctx, DC_ERR_ARG, "subdivide: need eps_coef, eps_len >= 0, a dc_resolve_mode and 0 <= label_ratio < 1");
    dc_subdivide_stats S;
    std::memset(&S, 0, sizeof(S));
    const double ratio = o->label_ratio > 0.0 ? o->label_ratio : 0.9;
    cudaStream_t s = ctx->stream;
    const int g = ctx->dg.g, P_old = ctx->dg.n_panels, N_old = ctx->dg.N, sp = ctx->dg.s;
    auto t0 = clk::now();
    // ---- Alg. 5: the highest Legendre coefficient of sigma per panel (device)
    std::vector<double> q(g);
    dc::legendre_top_row(g, q.data());
    DC_CK(ctx, ctx->ad_q.ensure(g), "subdivide: alloc");
    DC_CK(ctx, ctx->ad_top.ensure(P_old), "subdivide: alloc");
    DC_CK(ctx, cudaMemcpyAsync(ctx->ad_q.ptr, q.data(), sizeof(double) * g, cudaMemcpyHostToDevice, s), "subdivide");
    DC_CK(ctx, dc::launch_legendre_top(ctx->sigma.ptr, P_old, g, ctx->ad_q.ptr, ctx->ad_top.ptr, s), "subdivide: test");
    std::vector<double> top(P_old);
    DC_CK(ctx, cudaMemcpyAsync(top.data(), ctx->ad_top.ptr, sizeof(double) * P_old, cudaMemcpyDeviceToHost, s),
          "subdivide");
    DC_CK(ctx, cudaStreamSynchronize(s), "subdivide");
    // panel arc length: sum over its segments of chord x (arc / chord) weight
    std::vector<unsigned char> split(P_old, 0);
    int n_split = 0;
    for (int p = 0; p < P_old; ++p) {
        double len = 0.0;
        for (int k = 0; k < sp; ++k) {
            const double *e = &ctx->geo.seg_xy[4 * ((size_t)p * sp + k)];
            len += std::hypot(e[2] - e[0], e[3] - e[1]) * ctx->geo.seg_w[(size_t)p * sp + k];
        }
        if (top[p] > o->eps_coef && len >= o->eps_len && (!mask || mask[p])) {
            split[p] = 1;
            ++n_split;
        }
    }
    S.n_split = n_split;
    S.n_panels_before = S.n_panels_after = P_old;
    S.ms_test = ms_since(t0);
    ctx->last_top = top;
    ctx->last_split = split;
    if (n_split == 0) {
        ctx->last_resolve.assign(P_old, 0);
        S.converged = 1;
        if (stats) *stats = S;
        return DC_OK;
    }
    // ---- the refined panels: each split panel becomes its two halves in
    // arc-length fraction
    const int nc = ctx->in_ncurves;
    std::vector<int> new_ptr(nc + 1, 0);
    std::vector<double> new_start;
    std::vector<int2> pmap;
    for (int i = 0; i < nc; ++i) {
        for (int p = ctx->in_ptr[i]; p < ctx->in_ptr[i + 1]; ++p) {
            const double a = ctx->in_start[p], b = p + 1 < ctx->in_ptr[i + 1] ? ctx->in_start[p + 1] : 1.0;
            if (split[p]) {
                new_start.push_back(a);
                pmap.push_back(make_int2(p, 1));
                new_start.push_back(0.5 * (a + b));
                pmap.push_back(make_int2(p, 2));
            } else {
                new_start.push_back(a);
                pmap.push_back(make_int2(p, 0));
            }
        }
        new_ptr[i + 1] = int(new_start.size());
    }
    DC_CK(ctx, ctx->ad_sig_old.ensure(size_t(3) * N_old), "subdivide: alloc");
    DC_CK(ctx, cudaMemcpyAsync(ctx->ad_sig_old.ptr, ctx->sigma.ptr, sizeof(double) * 3 * N_old,
                               cudaMemcpyDeviceToDevice, s), "subdivide");
    // ---- update_quadtree / update_pre_FMM: the whole build on the refined
    // panels
    auto t1 = clk::now();
    {
        const std::vector<double> ctrl = ctx->in_ctrl, col = ctx->in_col;
        dc_status st = dc_build_tree(ctx, nc, ctrl.data(), new_ptr.data(), new_start.data(), col.data());
        if (st != DC_OK) return st;
    }
    S.ms_rebuild = ms_since(t1);
    const int P_new = ctx->dg.n_panels, N_new = ctx->dg.N;
    S.n_panels_after = P_new;
    // ---- warm start (Sec. 6.1): the old Legendre expansions at the new nodes
    std::vector<double> E((size_t)3 * g * g);
    dc::split_matrices(g, E.data());
    DC_CK(ctx, ctx->ad_E.ensure(E.size()), "subdivide: alloc");
    DC_CK(ctx, ctx->ad_pmap.ensure(pmap.size()), "subdivide: alloc");
    DC_CK(ctx, cudaMemcpyAsync(ctx->ad_E.ptr, E.data(), sizeof(double) * E.size(), cudaMemcpyHostToDevice, s),
          "subdivide");
    DC_CK(ctx, cudaMemcpyAsync(ctx->ad_pmap.ptr, pmap.data(), sizeof(int2) * pmap.size(), cudaMemcpyHostToDevice, s),
          "subdivide");
    DC_CK(ctx, dc::launch_split_interp(ctx->ad_sig_old.ptr, ctx->ad_pmap.ptr, ctx->ad_E.ptr, g, P_new,
                                       ctx->sigma.ptr, s), "subdivide: warm start");
    // ---- right-hand side of the refined system (Alg. 3), FP64
    auto apply_G = [&](const double *x, double *y) -> cudaError_t {
        if (ctx->opt.form == DC_FORM_DENSE64) return dc::launch_dense_gemv(ctx->AG.ptr, N_new, x, y, s);
        return ctx->fmm->apply_single_layer(x, y, s);
    };
    if (ctx->opt.form == DC_FORM_DENSE64)
        DC_CK(ctx, dc::launch_dense_gemv(ctx->AF.ptr, N_new, ctx->mu.ptr, ctx->fmu.ptr, s), "subdivide: rhs");
    else
        DC_CK(ctx, ctx->fmm->apply_double_layer(ctx->mu.ptr, ctx->fmu.ptr, s), "subdivide: rhs");
    DC_CK(ctx, dc::launch_rhs(ctx->dg, ctx->fmu.ptr, ctx->b.ptr, s), "subdivide: rhs");
    const size_t n3 = size_t(3) * N_new;
    DC_CK(ctx, ctx->ad_r0.ensure(n3), "subdivide: alloc");
    DC_CK(ctx, ctx->ad_tmp.ensure(n3), "subdivide: alloc");
    DC_CK(ctx, ctx->ad_tmp2.ensure(n3), "subdivide: alloc");
    DC_CK(ctx, ctx->ad_range.ensure(size_t(3) * P_new), "subdivide: alloc");
    // ---- label_curves (Eq. 40-41): unit density on each new half panel,
    // three per operator application (one per colour channel)
    auto t2 = clk::now();
    std::vector<unsigned char> res(P_new, 0);
    if (o->resolve == DC_RESOLVE_GLOBAL) {
        res.assign(P_new, 1);
    } else if (o->resolve == DC_RESOLVE_LOCAL) {
        std::vector<int> alpha;
        for (int p = 0; p < P_new; ++p)
            if (pmap[p].y != 0) {
                alpha.push_back(p);
                res[p] = 1;
            }
        std::vector<double> range((size_t)3 * P_new);
        for (size_t j = 0; j < alpha.size(); j += 3) {
            int three[3];
            for (int c = 0; c < 3; ++c) three[c] = j + c < alpha.size() ? alpha[j + c] : -1;
            DC_CK(ctx, dc::launch_unit_density(ctx->ad_tmp.ptr, N_new, g, three, s), "subdivide: labels");
            DC_CK(ctx, apply_G(ctx->ad_tmp.ptr, ctx->ad_tmp2.ptr), "subdivide: labels");
            DC_CK(ctx, dc::launch_panel_range(ctx->ad_tmp2.ptr, P_new, g, ctx->ad_range.ptr, s), "subdivide: labels");
            DC_CK(ctx, cudaMemcpyAsync(range.data(), ctx->ad_range.ptr, sizeof(double) * range.size(),
                                       cudaMemcpyDeviceToHost, s), "subdivide: labels");
            DC_CK(ctx, cudaStreamSynchronize(s), "subdivide: labels");
            S.n_label_matvec++;
            for (int c = 0; c < 3; ++c) {
                if (three[c] < 0) continue;
                const double da = range[3 * (size_t)three[c] + c];
                for (int b = 0; b < P_new; ++b)
                    if (range[3 * (size_t)b + c] > ratio * da) res[b] = 1;
            }
        }
    }
    S.ms_label = ms_since(t2);
    for (int p = 0; p < P_new; ++p) S.n_resolve_panels += res[p];
    ctx->last_resolve = res;
    // ---- the local system (Sec. 6.3): (G_H)_rr sigma_r = b_r - (G_H)_rc sigma_c,
    // solved for the correction delta_r of the warm start sigma0:
    //   (G_H)_rr delta_r = [b - G_H sigma0]_r
    auto t3 = clk::now();
    if (o->resolve != DC_RESOLVE_NONE) {
        DC_CK(ctx, ctx->ad_mask.ensure(P_new), "subdivide: alloc");
        DC_CK(ctx, cudaMemcpyAsync(ctx->ad_mask.ptr, res.data(), P_new, cudaMemcpyHostToDevice, s), "subdivide");
        DC_CK(ctx, apply_G(ctx->sigma.ptr, ctx->ad_tmp.ptr), "subdivide: residual");
        DC_CK(ctx, dc::vec_residual(ctx->b.ptr, ctx->ad_tmp.ptr, ctx->ad_r0.ptr, int(n3), s), "subdivide: residual");
        DC_CK(ctx, dc::launch_node_mask(ctx->ad_r0.ptr, ctx->ad_mask.ptr, N_new, g, s), "subdivide: residual");
        DC_CK(ctx, cudaMemcpyAsync(ctx->ad_tmp2.ptr, ctx->b.ptr, sizeof(double) * n3, cudaMemcpyDeviceToDevice, s),
              "subdivide");
        DC_CK(ctx, dc::launch_node_mask(ctx->ad_tmp2.ptr, ctx->ad_mask.ptr, N_new, g, s), "subdivide");
        double nb[3], nr[3];
        DC_CK(ctx, dc::vec_norms3(ctx->gw, ctx->ad_tmp2.ptr, N_new, nb, s), "subdivide");
        DC_CK(ctx, dc::vec_norms3(ctx->gw, ctx->ad_r0.ptr, N_new, nr, s), "subdivide");
        double rel = 1.0;
        bool need = false;
        for (int c = 0; c < 3; ++c)
            if (nr[c] > ctx->opt.gmres_tol * nb[c]) {
                need = true;
                rel = std::min(rel, ctx->opt.gmres_tol * nb[c] / nr[c]);
            }
        if (need) {
            MaskedOp op;
            op.ctx = ctx;
            op.pmask = ctx->ad_mask.ptr;
            DevBuf<double> z, t1b, t2b;
            DC_CK(ctx, z.alloc(n3), "subdivide: alloc");
            DC_CK(ctx, t1b.alloc(n3), "subdivide: alloc");
            DC_CK(ctx, t2b.alloc(n3), "subdivide: alloc");
            op.t1 = t1b.ptr;
            op.t2 = t2b.ptr;
            DC_CK(ctx, cudaMemsetAsync(z.ptr, 0, sizeof(double) * n3, s), "subdivide");
            dc::GmresResult gr;
            std::string msg;
            cudaError_t ce = dc::gmres_solve(ctx->gw, op, N_new, ctx->ad_r0.ptr, z.ptr, true, false,
                                             std::max(rel, 1e-15), ctx->opt.gmres_restart,
                                             ctx->opt.gmres_max_iter, s, gr, msg);
            if (ce != cudaSuccess) return cuda_fail(ctx, ce, msg.empty() ? "subdivide: gmres" : msg.c_str());
            for (int c = 0; c < 3; ++c) S.iters[c] = gr.iters[c];
            // delta = B z on r (the right preconditioner), sigma = sigma0 + delta
            if (ctx->opt.form == DC_FORM_DENSE64) {
                DC_CK(ctx, cudaMemcpyAsync(ctx->ad_tmp.ptr, z.ptr, sizeof(double) * n3, cudaMemcpyDeviceToDevice, s),
                      "subdivide");
            } else {
                DC_CK(ctx, dc::launch_node_mask(z.ptr, ctx->ad_mask.ptr, N_new, g, s), "subdivide");
                DC_CK(ctx, ctx->fmm->apply_block_jacobi(z.ptr, ctx->ad_tmp.ptr, s), "subdivide");
            }
            DC_CK(ctx, dc::launch_node_mask(ctx->ad_tmp.ptr, ctx->ad_mask.ptr, N_new, g, s), "subdivide");
            DC_CK(ctx, dc::vec_axpy(ctx->sigma.ptr, ctx->ad_tmp.ptr, int(n3), s), "subdivide");
        }
        // the local system's residual after the re-solve
        DC_CK(ctx, apply_G(ctx->sigma.ptr, ctx->ad_tmp.ptr), "subdivide: residual");
        DC_CK(ctx, dc::vec_residual(ctx->b.ptr, ctx->ad_tmp.ptr, ctx->ad_r0.ptr, int(n3), s), "subdivide: residual");
        DC_CK(ctx, dc::launch_node_mask(ctx->ad_r0.ptr, ctx->ad_mask.ptr, N_new, g, s), "subdivide: residual");
        DC_CK(ctx, dc::vec_norms3(ctx->gw, ctx->ad_r0.ptr, N_new, nr, s), "subdivide");
        S.converged = 1;
        for (int c = 0; c < 3; ++c) {
            S.rel_resid[c] = nb[c] > 0.0 ? nr[c] / nb[c] : 0.0;
            if (S.rel_resid[c] > 10.0 * ctx->opt.gmres_tol) S.converged = 0;
        }
    }
    S.ms_solve = ms_since(t3);
    ctx->state = 2;
    ctx->seg_density_valid = false;
    if (stats) *stats = S;
    return DC_OK;
}

dc_status dc_subdivide(dc_ctx *ctx, const dc_subdivide_options *o, dc_subdivide_stats *stats) {
    if (ctx && ctx->render_only) return fail(ctx, DC_ERR_STATE, "subdivide: a view context renders only");
    return subdivide_impl(ctx, o, nullptr, stats);
}

// ------------------------------------------------ viewport update (6.4) --
dc_status dc_view_update(dc_ctx *ctx, const dc_viewport *vp, const dc_view_options *o, dc_view_stats *stats) {
    using clk = std::chrono::steady_clock;
    auto ms_since = [](clk::time_point a) { return std::chrono::duration<double, std::milli>(clk::now() - a).count(); };
    if (!ctx) return DC_ERR_ARG;
    ctx->err.clear();
    if (!vp || !o) return fail(ctx, DC_ERR_ARG, "view_update: NULL viewport or options");
    if (ctx->render_only) return fail(ctx, DC_ERR_STATE, "view_update: a view context renders only");
    if (ctx->state < 2) return fail(ctx, DC_ERR_STATE, "view_update: needs a density (solve_density or set_density)");
    if (!(vp->width > 0 && vp->height > 0) || !std::isfinite(vp->x0) || !std::isfinite(vp->x1) ||
        !std::isfinite(vp->y0) || !std::isfinite(vp->y1) || !(vp->x1 > vp->x0) || !(vp->y1 > vp->y0))
        return fail(ctx, DC_ERR_ARG, "view_update: need a viewport with x1 > x0, y1 > y0 and pixels");
    if (!(o->eps_coef >= 0.0) || !std::isfinite(o->eps_coef) || !(o->eps_len_px >= 0.0) ||
        !std::isfinite(o->eps_len_px) || !(o->len_unit >= 0.0) || !std::isfinite(o->len_unit) || o->max_rounds < 0 ||
        o->max_rounds > 64 || o->resolve < DC_RESOLVE_LOCAL || o->resolve > DC_RESOLVE_NONE ||
        !(o->label_ratio >= 0.0) || !(o->label_ratio < 1.0))
        return fail(ctx, DC_ERR_ARG, "view_update: need eps_coef, eps_len_px, len_unit >= 0, max_rounds in [0, 64], "
                                     "a dc_resolve_mode and 0 <= label_ratio < 1");
    const double unit = o->len_unit > 0.0 ? o->len_unit : 1.0 / 512.0;
    const int max_rounds = o->max_rounds > 0 ? o->max_rounds : 4;
    const double px = std::max((vp->x1 - vp->x0) / vp->width, (vp->y1 - vp->y0) / vp->height);
    dc_view_stats S;
    std::memset(&S, 0, sizeof(S));
    S.converged = 1;
    const auto t0 = clk::now();
    ctx->view_valid = false;
    // panels whose solve polyline's box meets the viewport's closed rectangle
    auto meets = [&](std::vector<unsigned char> &m) {
        const int P = ctx->dg.n_panels, sp = ctx->dg.s;
        m.assign(P, 0);
        for (int p = 0; p < P; ++p) {
            double lo[2] = {1e300, 1e300}, hi[2] = {-1e300, -1e300};
            for (int k = 0; k < sp; ++k) {
                const double *e = &ctx->geo.seg_xy[4 * ((size_t)p * sp + k)];
                for (int q = 0; q < 2; ++q) {
                    lo[0] = std::min(lo[0], e[2 * q]);
                    hi[0] = std::max(hi[0], e[2 * q]);
                    lo[1] = std::min(lo[1], e[2 * q + 1]);
                    hi[1] = std::max(hi[1], e[2 * q + 1]);
                }
            }
            m[p] = hi[0] >= vp->x0 && lo[0] <= vp->x1 && hi[1] >= vp->y0 && lo[1] <= vp->y1;
        }
    };
    // Alg. 9: subdivide (Alg. 5, epsilon_1 in pixels, panels in the viewport
    // only) and re-solve while panels split
    std::vector<unsigned char> m, res_last;
    if (o->eps_coef > 0.0) {
        for (int r = 0; r < max_rounds; ++r) {
            meets(m);
            dc_subdivide_options so;
            std::memset(&so, 0, sizeof(so));
            so.eps_coef = o->eps_coef;
            so.eps_len = o->eps_len_px * px;
            so.resolve = o->resolve;
            so.label_ratio = o->label_ratio;
            dc_subdivide_stats ss;
            dc_status st = subdivide_impl(ctx, &so, m.data(), &ss);
            if (st != DC_OK) return st;
            if (ss.n_split == 0) break;
            ++S.rounds;
            S.n_split += ss.n_split;
            S.n_resolve_panels = ss.n_resolve_panels;
            if (!ss.converged) S.converged = 0;
            res_last = ctx->last_resolve;
        }
    }
    S.ms_subdivide = ms_since(t0);
    // labels of Sec. 6.4 and the e rule of Sec. 6.2 on the final panels
    meets(m);
    const int P = ctx->dg.n_panels, sp = ctx->dg.s;
    long long e = sp;
    for (int p = 0; p < P; ++p) {
        const bool re = (int)res_last.size() == P && res_last[p];
        if (re) ++S.n_resolving;
        else if (m[p]) ++S.n_interpolating;
        else ++S.n_fixed;
        if (!m[p]) continue;
        double len = 0.0;
        for (int k = 0; k < sp; ++k) {
            const double *q = &ctx->geo.seg_xy[4 * ((size_t)p * sp + k)];
            len += std::hypot(q[2] - q[0], q[3] - q[1]) * ctx->geo.seg_w[(size_t)p * sp + k];
        }
        const double add = std::ceil(len / (10.0 * unit));
        if (add > 4096.0) return fail(ctx, DC_ERR_ARG, "view_update: the e rule asks for more than 4096 segments per panel");
        e = std::max(e, (long long)add + sp);
    }
    if (e > 4096) return fail(ctx, DC_ERR_ARG, "view_update: the e rule asks for more than 4096 segments per panel");
    S.e = int(e);
    S.n_eval_segments = (long long)P * e;
    // the evaluation discretisation: a render-only context on the same
    // panels with e segments each, the same nodes and densities
    const auto t1 = clk::now();
    if (ctx->view && ctx->view->opt.s_per_panel != int(e)) {
        cudaStreamSynchronize(ctx->view->stream);
        delete ctx->view;
        ctx->view = nullptr;
    }
    if (!ctx->view) {
        dc_options vo = ctx->opt;
        vo.s_per_panel = int(e);
        vo.stream = ctx->stream;
        dc_ctx *v = nullptr;
        dc_status st = dc_create(&v, &vo);
        if (st != DC_OK) return fail(ctx, st, std::string("view_update: ") + dc_last_error(nullptr));
        v->render_only = true;
        ctx->view = v;
    }
    dc_ctx *v = ctx->view;
    {
        dc_status st = dc_build_tree(v, ctx->in_ncurves, ctx->in_ctrl.data(), ctx->in_ptr.data(),
                                     ctx->in_start.data(), ctx->in_col.data());
        if (st != DC_OK) return fail(ctx, st, std::string("view_update: ") + v->err);
    }
    const size_t n3 = size_t(3) * ctx->dg.N;
    if (v->dg.N != ctx->dg.N) return fail(ctx, DC_ERR_STATE, "view_update: node counts differ");
    DC_CK(ctx, cudaMemcpyAsync(v->sigma.ptr, ctx->sigma.ptr, n3 * sizeof(double), cudaMemcpyDeviceToDevice,
                               ctx->stream), "view_update");
    DC_CK(ctx, cudaMemcpyAsync(v->mu.ptr, ctx->mu.ptr, n3 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream),
          "view_update");
    DC_CK(ctx, cudaStreamSynchronize(ctx->stream), "view_update");
    v->seg_density_valid = false;
    v->state = 2;
    ctx->view_valid = true;
    S.ms_build = ms_since(t1);
    S.ms_total = ms_since(t0);
    if (stats) *stats = S;
    return DC_OK;
}

dc_status dc_aux_tree_compare(dc_ctx *ctx, double *out) {
    if (!ctx || !out) return DC_ERR_ARG;
    ctx->err.clear();
    if (ctx->state < 1 || !ctx->fmm) return fail(ctx, DC_ERR_STATE, "tree_compare: needs an FMM form after build_tree");
    ctx->fmm->compare_host_tree(ctx->geo, out);
    return DC_OK;
}

dc_status dc_view_reset(dc_ctx *ctx) {
    if (!ctx) return DC_ERR_ARG;
    ctx->err.clear();
    ctx->view_valid = false;
    return DC_OK;
}

dc_status dc_aux_adaptive_panels(int n_curves, const double *ctrl, double ratio, int max_level, int min_panels,
                                 double max_len, int capacity, int *panel_ptr, double *panel_start, int *n_panels) {
    if (n_curves < 1 || !ctrl || !panel_ptr || !n_panels || capacity < 0 || (capacity > 0 && !panel_start) ||
        !(ratio > 0.0) || max_level < 0 || max_level > 30 || min_panels < 1 || !(max_len > 0.0))
        return DC_ERR_ARG;
    for (int i = 0; i < 8 * n_curves; ++i)
        if (!std::isfinite(ctrl[i])) return DC_ERR_ARG;
    std::vector<int> ptr;
    std::vector<double> start;
    std::string msg;
    dc_status st = dc::adaptive_panels(n_curves, ctrl, ratio, max_level, min_panels, max_len, ptr, start, msg);
    if (st != DC_OK) return st;
    *n_panels = int(start.size());
    std::memcpy(panel_ptr, ptr.data(), sizeof(int) * ptr.size());
    if ((int)start.size() > capacity) return DC_ERR_ARG;
    std::memcpy(panel_start, start.data(), sizeof(double) * start.size());
    return DC_OK;
}

dc_status dc_aux_discretise(int n_curves, const double *ctrl, const int *panel_ptr, const double *panel_start,
                            const double *colours, int g, int s, double *node_xy, double *node_t, double *seg_xy,
                            double *seg_w, double *u_plus, double *u_minus) {
    dc::Geometry G;
    std::string msg;
    dc_status st = dc::discretise(n_curves, ctrl, panel_ptr, panel_start, colours, g, s, G, msg);
    if (st != DC_OK) return st;
    auto put = [](double *dst, const std::vector<double> &v) {
        if (dst && !v.empty()) std::memcpy(dst, v.data(), sizeof(double) * v.size());
    };
    put(node_xy, G.node_xy);
    put(node_t, G.node_t);
    put(seg_xy, G.seg_xy);
    put(seg_w, G.seg_w);
    put(u_plus, G.u_plus);
    put(u_minus, G.u_minus);
    return DC_OK;
}

// ------------------------------------------------------------- autotune --
dc_status dc_autotune(dc_ctx *ctx, int n_vp, const dc_viewport *vps, int n_leaf, const int *leaf_sizes,
                      int n_pinner, const int *p_inners, int n_tile, const int *eval_tiles, double tol,
                      int repeats, dc_autotune_row *rows, int *best) {
    if (!ctx) return DC_ERR_ARG;
    ctx->err.clear();
    if (ctx->state < 1) return fail(ctx, DC_ERR_STATE, "autotune: call build_tree first");
    if (ctx->opt.form != DC_FORM_FMM32) return fail(ctx, DC_ERR_UNSUPPORTED, "autotune: needs DC_FORM_FMM32");
    if (n_vp < 1 || !vps || n_leaf < 0 || n_pinner < 0 || n_tile < 0 || (n_leaf > 0 && !leaf_sizes) ||
        (n_pinner > 0 && !p_inners) || (n_tile > 0 && !eval_tiles) || !(tol > 0.0) || repeats < 1 || !rows || !best)
        return fail(ctx, DC_ERR_ARG, "autotune: bad arguments");
    long long npx = 0;
    for (int v = 0; v < n_vp; ++v) npx += (long long)vps[v].width * vps[v].height;
    if (npx <= 0) return fail(ctx, DC_ERR_ARG, "autotune: no pixels");
    const dc_options orig = ctx->opt;
    const int nc = ctx->in_ncurves;
    const std::vector<double> ctrl = ctx->in_ctrl, start = ctx->in_start, col = ctx->in_col;
    const std::vector<int> pptr = ctx->in_ptr;
    auto rebuild = [&](const dc_options &o) -> dc_status {
        ctx->opt = o;
        return dc_build_tree(ctx, nc, ctrl.data(), pptr.data(), start.data(), col.data());
    };
    cudaStream_t s = ctx->stream;
    // reference pixels: the plain FP64 FMM form of the same drawing and order
    DevBuf<double> ref;
    DevBuf<float> out;
    DevBuf<unsigned> dmax;
    DC_CK(ctx, ref.alloc(3 * (size_t)npx), "autotune: alloc");
    DC_CK(ctx, out.alloc(3 * (size_t)npx), "autotune: alloc");
    DC_CK(ctx, dmax.alloc(1), "autotune: alloc");
    {
        dc_options ro = orig;
        ro.form = DC_FORM_FMM64;
        if (ro.x0_mode == DC_X0_USER || ro.x0_mode == DC_X0_LEARNED) ro.x0_mode = DC_X0_ONES;
        dc_ctx *rc = nullptr;
        dc_status st = dc_create(&rc, &ro);
        if (st != DC_OK) return fail(ctx, st, std::string("autotune: reference context: ") + dc_last_error(nullptr));
        st = dc_build_tree(rc, nc, ctrl.data(), pptr.data(), start.data(), col.data());
        if (st == DC_OK) st = dc_solve_density(rc, nullptr, nullptr);
        if (st == DC_OK) st = dc_render_viewport(rc, n_vp, vps, ref.ptr, DC_F64, nullptr, DC_MEM_DEVICE, nullptr);
        if (st == DC_OK && cudaStreamSynchronize(rc->stream) != cudaSuccess) st = DC_ERR_CUDA;
        const std::string msg = st == DC_OK ? "" : rc->err;
        dc_destroy(rc);
        if (st != DC_OK) return fail(ctx, st, "autotune: reference: " + msg);
    }
    const int nl = std::max(n_leaf, 1), np = std::max(n_pinner, 1), nt = std::max(n_tile, 1);
    cudaEvent_t e0, e1;
    DC_CK(ctx, cudaEventCreate(&e0), "event");
    DC_CK(ctx, cudaEventCreate(&e1), "event");
    struct EvGuard {
        cudaEvent_t a, b;
        ~EvGuard() {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } guard{e0, e1};
    int k = 0, chosen = -1;
    for (int il = 0; il < nl; ++il)
        for (int ip = 0; ip < np; ++ip) {
            dc_options o = orig;
            if (o.x0_mode == DC_X0_USER) o.x0_mode = DC_X0_ONES;
            if (n_leaf > 0) o.leaf_size = leaf_sizes[il];
            if (n_pinner > 0) o.p_inner = std::min(p_inners[ip], o.p);
            std::string why;
            dc_status bst = check_options(o, why);
            if (bst == DC_OK) bst = rebuild(o);
            for (int it = 0; it < nt; ++it, ++k) {
                dc_autotune_row &r = rows[k];
                r.leaf_size = o.leaf_size;
                r.p_inner = o.p_inner;
                r.eval_tile = n_tile > 0 ? eval_tiles[it] : o.eval_tile;
                r.ms = -1.0;
                r.max_err = INFINITY;
                r.converged = 0;
                if (bst != DC_OK || r.eval_tile < 0 || r.eval_tile > 3) continue;
                ctx->opt.eval_tile = r.eval_tile;
                ctx->fmm->set_eval_tile(r.eval_tile);
                dc_solve_stats ss;
                dc_status st = dc_solve_density(ctx, nullptr, &ss);   // warm-up: graphs, buffers, tile plan
                if (st == DC_OK)
                    st = dc_render_viewport(ctx, n_vp, vps, out.ptr, DC_F32, nullptr, DC_MEM_DEVICE, nullptr);
                if (st != DC_OK) continue;
                float bestms = INFINITY;
                for (int rep = 0; rep < repeats && st == DC_OK; ++rep) {
                    DC_CK(ctx, cudaEventRecord(e0, s), "event");
                    st = dc_solve_density(ctx, nullptr, &ss);
                    if (st == DC_OK)
                        st = dc_render_viewport(ctx, n_vp, vps, out.ptr, DC_F32, nullptr, DC_MEM_DEVICE, nullptr);
                    DC_CK(ctx, cudaEventRecord(e1, s), "event");
                    DC_CK(ctx, cudaEventSynchronize(e1), "event");
                    float ms = 0.f;
                    DC_CK(ctx, cudaEventElapsedTime(&ms, e0, e1), "event");
                    bestms = std::min(bestms, ms);
                }
                if (st != DC_OK) continue;
                DC_CK(ctx, dc::launch_max_diff(out.ptr, ref.ptr, 3 * npx, dmax.ptr, s), "autotune: compare");
                unsigned bits = 0;
                DC_CK(ctx, cudaMemcpyAsync(&bits, dmax.ptr, sizeof(bits), cudaMemcpyDeviceToHost, s), "autotune");
                DC_CK(ctx, cudaStreamSynchronize(s), "autotune");
                float err;
                std::memcpy(&err, &bits, sizeof(err));
                r.ms = bestms;
                r.max_err = err;
                r.converged = ss.converged;
                if (r.converged && err <= tol && (chosen < 0 || r.ms < rows[chosen].ms)) chosen = k;
            }
        }
    *best = chosen;
    dc_options fin = orig;
    if (chosen >= 0) {
        fin.leaf_size = rows[chosen].leaf_size;
        fin.p_inner = rows[chosen].p_inner;
        fin.eval_tile = rows[chosen].eval_tile;
    }
    dc_status st = rebuild(fin);
    if (st != DC_OK) return st;
    return DC_OK;
}

// ------------------------------------------------ mixed conditions (4.3) --
dc_status dc_solve_mixed(dc_ctx *ctx, const unsigned char *neumann, const double *psi_star,
                         const double *u_star, dc_solve_stats *stats) {
    if (!ctx) return DC_ERR_ARG;
    ctx->err.clear();
    if (ctx->state < 1) return fail(ctx, DC_ERR_STATE, "solve_mixed: call build_tree first");
    if (ctx->render_only) return fail(ctx, DC_ERR_STATE, "solve_mixed: a view context renders only");
    ctx->view_valid = false;
    if (!neumann || !psi_star) return fail(ctx, DC_ERR_ARG, "solve_mixed: need the Neumann panels and psi");
    const int N = ctx->dg.N, g = ctx->dg.g, P = ctx->dg.n_panels;
    const size_t n3 = size_t(3) * N;
    for (size_t i = 0; i < n3; ++i)
        if (!std::isfinite(psi_star[i]) || (u_star && !std::isfinite(u_star[i])))
            return fail(ctx, DC_ERR_ARG, "solve_mixed: non-finite boundary data");
    // the region must lie on the left of the curves: positive total signed
    // area of the solve polyline (a necessary condition; loops are not traced)
    double area = 0.0;
    for (size_t k = 0; k < ctx->geo.seg_xy.size() / 4; ++k) {
        const double *e = &ctx->geo.seg_xy[4 * k];
        area += 0.5 * (e[0] * e[3] - e[2] * e[1]);
    }
    if (!(area > 0.0))
        return fail(ctx, DC_ERR_GEOMETRY, "solve_mixed: the curves must bound the region counter-clockwise");
    std::vector<unsigned char> nm(P), dm(P);
    int n_neu = 0;
    for (int p = 0; p < P; ++p) {
        nm[p] = neumann[p] ? 1 : 0;
        dm[p] = 1 - nm[p];
        n_neu += nm[p];
    }
    if (n_neu == P) return fail(ctx, DC_ERR_ARG, "solve_mixed: at least one panel needs a Dirichlet value");
    cudaStream_t s = ctx->stream;
    if (stats) std::memset(stats, 0, sizeof(*stats));
    auto t0 = std::chrono::steady_clock::now();
    DevBuf<unsigned char> dn, dd;
    DevBuf<double> ud, psin, b, z, x, t1, t2, t3;
    DC_CK(ctx, dn.alloc(P), "solve_mixed: alloc");
    DC_CK(ctx, dd.alloc(P), "solve_mixed: alloc");
    for (auto *bp : {&ud, &psin, &b, &z, &x, &t1, &t2, &t3}) DC_CK(ctx, bp->alloc(n3), "solve_mixed: alloc");
    DC_CK(ctx, cudaMemcpyAsync(dn.ptr, nm.data(), P, cudaMemcpyHostToDevice, s), "solve_mixed");
    DC_CK(ctx, cudaMemcpyAsync(dd.ptr, dm.data(), P, cudaMemcpyHostToDevice, s), "solve_mixed");
    DC_CK(ctx, cudaMemcpyAsync(psin.ptr, psi_star, n3 * sizeof(double), cudaMemcpyHostToDevice, s), "solve_mixed");
    if (u_star)
        DC_CK(ctx, cudaMemcpyAsync(ud.ptr, u_star, n3 * sizeof(double), cudaMemcpyHostToDevice, s), "solve_mixed");
    else
        DC_CK(ctx, cudaMemcpyAsync(ud.ptr, ctx->dg.u_minus.ptr, n3 * sizeof(double), cudaMemcpyDeviceToDevice, s),
              "solve_mixed");
    DC_CK(ctx, dc::launch_node_mask(ud.ptr, dd.ptr, N, g, s), "solve_mixed");
    DC_CK(ctx, dc::launch_node_mask(psin.ptr, dn.ptr, N, g, s), "solve_mixed");
    MixedOp op;
    op.ctx = ctx;
    op.nmask = dn.ptr;
    op.dmask = dd.ptr;
    op.t1 = t1.ptr;
    op.t2 = t2.ptr;
    op.t3 = t3.ptr;
    // b = u_d / 2 + F_H u_d - G_H psi_n
    const bool dense = ctx->opt.form == DC_FORM_DENSE64;
    DC_CK(ctx, dense ? dc::launch_dense_gemv(ctx->AF.ptr, N, ud.ptr, b.ptr, s)
                     : ctx->fmm->apply_double_layer(ud.ptr, b.ptr, s), "solve_mixed: rhs");
    DC_CK(ctx, dense ? dc::launch_dense_gemv(ctx->AG.ptr, N, psin.ptr, t1.ptr, s)
                     : ctx->fmm->apply_single_layer(psin.ptr, t1.ptr, s), "solve_mixed: rhs");
    {
        const double one[3] = {1, 1, 1}, half[3] = {0.5, 0.5, 0.5}, m1[3] = {-1, -1, -1};
        DC_CK(ctx, dc::vec_combine3(b.ptr, ud.ptr, b.ptr, N, one, half, s), "solve_mixed: rhs");
        DC_CK(ctx, dc::vec_combine3(b.ptr, t1.ptr, b.ptr, N, one, m1, s), "solve_mixed: rhs");
    }
    DC_CK(ctx, cudaMemsetAsync(z.ptr, 0, n3 * sizeof(double), s), "solve_mixed");
    dc::GmresResult gr;
    std::string msg;
    cudaError_t ce = dc::gmres_solve(ctx->gw, op, N, b.ptr, z.ptr, true, false, ctx->opt.gmres_tol,
                                     ctx->opt.gmres_restart, ctx->opt.gmres_max_iter, s, gr, msg);
    if (ce != cudaSuccess) return cuda_fail(ctx, ce, msg.empty() ? "solve_mixed: gmres" : msg.c_str());
    DC_CK(ctx, op.precond(z.ptr, x.ptr, s), "solve_mixed");
    // sigma = psi (psi_d from x, psi* given), mu = -u (u_n from x, u* given)
    DC_CK(ctx, dc::launch_blend(ctx->sigma.ptr, x.ptr, 1.0, psin.ptr, 1.0, dn.ptr, N, g, s), "solve_mixed");
    DC_CK(ctx, dc::launch_blend(ctx->mu.ptr, ud.ptr, -1.0, x.ptr, -1.0, dn.ptr, N, g, s), "solve_mixed");
    DC_CK(ctx, cudaStreamSynchronize(s), "solve_mixed");
    ctx->mu_custom = true;
    ctx->seg_density_valid = false;
    ctx->state = 2;
    if (stats) {
        for (int c = 0; c < 3; ++c) {
            stats->iters[c] = gr.iters[c];
            stats->rel_resid[c] = gr.rel_resid[c];
            stats->true_rel_resid[c] = gr.true_rel_resid[c];
        }
        stats->converged = gr.converged;
        stats->n_matvec = 2 * gr.n_matvec + 2;
        stats->ms_solve = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    return gr.converged ? DC_OK : fail(ctx, DC_ERR_NOCONV, "solve_mixed: GMRES did not reach gmres_tol");
}

dc_status dc_aux_fp32_peak(void *stream, double *out) {
    if (!out) return DC_ERR_ARG;
    double tf = 0.0, ms = 0.0;
    if (dc::measure_fp32_peak(static_cast<cudaStream_t>(stream), &tf, &ms) != cudaSuccess) return DC_ERR_CUDA;
    out[0] = tf;
    out[1] = ms;
    return DC_OK;
}

dc_status dc_aux_time_inner_m2l(dc_ctx *ctx, int reps, double *out) {
    if (!ctx) return DC_ERR_ARG;
    ctx->err.clear();
    if (!out || reps < 1) return fail(ctx, DC_ERR_ARG, "time_inner_m2l: need out and reps >= 1");
    if (ctx->state < 1 || !ctx->fmm) return fail(ctx, DC_ERR_STATE, "time_inner_m2l: needs an FMM form after build_tree");
    cudaError_t e = ctx->fmm->time_inner_m2l(reps, ctx->stream, out);
    if (e == cudaErrorNotSupported)
        return fail(ctx, DC_ERR_UNSUPPORTED, "time_inner_m2l: the context has no FP32 inner operator with list-2 pairs");
    DC_CK(ctx, e, "time_inner_m2l");
    return DC_OK;
}

dc_status dc_aux_test_skip_mma_tile(dc_ctx *ctx, int tile) {
    if (!ctx) return DC_ERR_ARG;
    ctx->err.clear();
    if (tile < -1) return fail(ctx, DC_ERR_ARG, "test_skip_mma_tile: tile must be >= -1");
    if (ctx->state < 1 || !ctx->fmm) return fail(ctx, DC_ERR_STATE, "test_skip_mma_tile: needs an FMM form after build_tree");
    cudaError_t e = ctx->fmm->set_mma_skip_tile(tile, ctx->stream);
    if (e == cudaErrorNotSupported)
        return fail(ctx, DC_ERR_UNSUPPORTED, "test_skip_mma_tile: the inner operator does not run its M2L on the tensor cores");
    DC_CK(ctx, e, "test_skip_mma_tile");
    DC_CK(ctx, cudaStreamSynchronize(ctx->stream), "test_skip_mma_tile");
    return DC_OK;
}

}  // extern "C"
