"""Python binding of libdc_fmm (argument marshalling only).

Every computation runs in the native library's CUDA kernels; this module
only converts arrays to pointers.  It raises ImportError when the native
library has not been built (``paper_2311_14312_gb300.build.build()``): there
is no fallback path.

The names mirror the C ABI in ``include/dc_fmm.h`` (``dc_create``,
``dc_build_tree``, ``dc_solve_density``, ``dc_render_viewport``, ...);
:class:`Context` wraps them for convenience.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

try:      # torch owns the CUDA runtime in this process; load it first
    import torch  # noqa: F401
except Exception:  # pragma: no cover - torch is a hard dependency of the tests
    torch = None

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libdc_fmm.so")

# enums (dc_fmm.h)
DC_OK, DC_ERR_ARG, DC_ERR_STATE, DC_ERR_CUDA, DC_ERR_OOM = 0, 1, 2, 3, 4
DC_ERR_NOCONV, DC_ERR_TIMEOUT, DC_ERR_GEOMETRY, DC_ERR_UNSUPPORTED = 5, 6, 7, 8
DC_FORM_DENSE64, DC_FORM_FMM64, DC_FORM_FMM32 = 0, 1, 2
DC_X0_ONES, DC_X0_ZEROS, DC_X0_USER, DC_X0_LEARNED = 0, 1, 2, 3
DC_MEM_DEVICE, DC_MEM_HOST = 0, 1
DC_F32, DC_F64 = 0, 1
DC_M2L_TENSOR, DC_M2L_CUDA_CORES = 0, 1
DC_RESOLVE_LOCAL, DC_RESOLVE_GLOBAL, DC_RESOLVE_NONE = 0, 1, 2
RESOLVE = {"local": DC_RESOLVE_LOCAL, "global": DC_RESOLVE_GLOBAL, "none": DC_RESOLVE_NONE}

FORMS = {"dense64": DC_FORM_DENSE64, "fmm64": DC_FORM_FMM64, "fmm32": DC_FORM_FMM32}


class dc_options(ctypes.Structure):
    _fields_ = [("form", ctypes.c_int), ("g", ctypes.c_int), ("s_per_panel", ctypes.c_int),
                ("p", ctypes.c_int), ("leaf_size", ctypes.c_int), ("max_depth", ctypes.c_int),
                ("gmres_tol", ctypes.c_double), ("gmres_restart", ctypes.c_int),
                ("gmres_max_iter", ctypes.c_int), ("x0_mode", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("domain", ctypes.c_double * 4),
                ("p_inner", ctypes.c_int), ("inner_tol", ctypes.c_double), ("m2l_engine", ctypes.c_int),
                ("coarse_max", ctypes.c_int), ("adapt_ratio", ctypes.c_double),
                ("adapt_max_level", ctypes.c_int), ("adapt_min_panels", ctypes.c_int),
                ("adapt_max_len", ctypes.c_double), ("eval_tile", ctypes.c_int),
                ("aa_levels", ctypes.c_int)]


class dc_sizes(ctypes.Structure):
    _fields_ = [("n_curves", ctypes.c_int), ("n_panels", ctypes.c_int), ("n_nodes", ctypes.c_int),
                ("n_segments", ctypes.c_int), ("n_pieces", ctypes.c_int),
                ("n_cells", ctypes.c_int), ("n_leaves", ctypes.c_int), ("depth", ctypes.c_int),
                ("root", ctypes.c_double * 3)]


class dc_solve_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int * 3), ("rel_resid", ctypes.c_double * 3),
                ("converged", ctypes.c_int), ("n_matvec", ctypes.c_int),
                ("ms_rhs", ctypes.c_double), ("ms_solve", ctypes.c_double),
                ("p2p_pairs", ctypes.c_longlong), ("m2l_pairs", ctypes.c_longlong),
                ("used_warm", ctypes.c_int), ("warm_resid", ctypes.c_double * 3),
                ("ms_warm", ctypes.c_double), ("n_refine", ctypes.c_int),
                ("true_rel_resid", ctypes.c_double * 3)]


class dc_subdivide_options(ctypes.Structure):
    _fields_ = [("eps_coef", ctypes.c_double), ("eps_len", ctypes.c_double), ("resolve", ctypes.c_int),
                ("label_ratio", ctypes.c_double)]


class dc_subdivide_stats(ctypes.Structure):
    _fields_ = [("n_split", ctypes.c_int), ("n_panels_before", ctypes.c_int),
                ("n_panels_after", ctypes.c_int), ("n_resolve_panels", ctypes.c_int),
                ("n_label_matvec", ctypes.c_int), ("iters", ctypes.c_int * 3),
                ("rel_resid", ctypes.c_double * 3), ("converged", ctypes.c_int),
                ("ms_test", ctypes.c_double), ("ms_rebuild", ctypes.c_double),
                ("ms_label", ctypes.c_double), ("ms_solve", ctypes.c_double)]


class dc_view_options(ctypes.Structure):
    _fields_ = [("eps_coef", ctypes.c_double), ("eps_len_px", ctypes.c_double), ("len_unit", ctypes.c_double),
                ("resolve", ctypes.c_int), ("max_rounds", ctypes.c_int), ("label_ratio", ctypes.c_double)]


class dc_view_stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int), ("n_split", ctypes.c_int), ("n_resolve_panels", ctypes.c_int),
                ("n_fixed", ctypes.c_int), ("n_interpolating", ctypes.c_int), ("n_resolving", ctypes.c_int),
                ("e", ctypes.c_int), ("n_eval_segments", ctypes.c_longlong), ("converged", ctypes.c_int),
                ("ms_subdivide", ctypes.c_double), ("ms_build", ctypes.c_double), ("ms_total", ctypes.c_double)]


class dc_autotune_row(ctypes.Structure):
    _fields_ = [("leaf_size", ctypes.c_int), ("p_inner", ctypes.c_int), ("eval_tile", ctypes.c_int),
                ("ms", ctypes.c_double), ("max_err", ctypes.c_double), ("converged", ctypes.c_int)]


class dc_viewport(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_double), ("y0", ctypes.c_double), ("x1", ctypes.c_double),
                ("y1", ctypes.c_double), ("width", ctypes.c_int), ("height", ctypes.c_int)]


class dc_render_stats(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double), ("ms_eval", ctypes.c_double),
                ("pixels", ctypes.c_longlong), ("p2p_pairs", ctypes.c_longlong),
                ("m2p_pairs", ctypes.c_longlong), ("m2l_pairs", ctypes.c_longlong),
                ("eval_flops", ctypes.c_double), ("aa_pixels", ctypes.c_longlong),
                ("aa_samples", ctypes.c_longlong), ("ms_aa", ctypes.c_double)]


EXPORTS = ["dc_default_options", "dc_create", "dc_destroy", "dc_build_tree", "dc_solve_density",
           "dc_render_viewport", "dc_eval_points", "dc_get_density", "dc_set_density",
           "dc_get_nodes", "dc_get_sizes", "dc_last_error", "dc_status_string",
           "dc_abi_version", "dc_aux_tree_check", "dc_aux_kernel_launches",
           "dc_eval_points_noalloc", "dc_aux_mlp_param_count", "dc_aux_mlp_workspace_floats",
           "dc_aux_mlp_forward", "dc_aux_mlp_loss_grad", "dc_aux_mlp_adam", "dc_aux_feature_dims",
           "dc_aux_panel_features", "dc_aux_set_warm_start_model", "dc_aux_apply_operator", "dc_aux_precond_info",
           "dc_aux_build_timings", "dc_aux_test_skip_mma_tile", "dc_aux_fp32_peak",
           "dc_aux_time_inner_m2l", "dc_subdivide", "dc_get_panels", "dc_aux_subdivision_info",
           "dc_aux_adaptive_panels", "dc_autotune", "dc_solve_mixed", "dc_view_update", "dc_view_reset",
           "dc_aux_tree_compare", "dc_aux_discretise"]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -m paper_2311_14312_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.dc_default_options.argtypes = [ctypes.POINTER(dc_options)]
    lib.dc_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(dc_options)]
    lib.dc_destroy.argtypes = [P]
    lib.dc_destroy.restype = None
    lib.dc_build_tree.argtypes = [P, I, P, P, P, P]
    lib.dc_solve_density.argtypes = [P, P, ctypes.POINTER(dc_solve_stats)]
    lib.dc_solve_mixed.argtypes = [P, P, P, P, ctypes.POINTER(dc_solve_stats)]
    lib.dc_render_viewport.argtypes = [P, I, ctypes.POINTER(dc_viewport), P, I, P, I,
                                       ctypes.POINTER(dc_render_stats)]
    lib.dc_eval_points.argtypes = [P, I, P, I, P, I, I]
    lib.dc_eval_points_noalloc.argtypes = [P, I, P, P]
    lib.dc_get_density.argtypes = [P, P]
    lib.dc_set_density.argtypes = [P, P]
    lib.dc_get_nodes.argtypes = [P, P, P, P, P]
    lib.dc_get_sizes.argtypes = [P, ctypes.POINTER(dc_sizes)]
    lib.dc_last_error.argtypes = [P]
    lib.dc_last_error.restype = ctypes.c_char_p
    lib.dc_status_string.argtypes = [I]
    lib.dc_status_string.restype = ctypes.c_char_p
    lib.dc_abi_version.restype = I
    lib.dc_aux_tree_check.argtypes = [I, P, P, I, I, P]
    lib.dc_aux_kernel_launches.argtypes = []
    lib.dc_aux_kernel_launches.restype = ctypes.c_longlong
    Z, F = ctypes.c_size_t, ctypes.c_float
    lib.dc_aux_mlp_param_count.argtypes = [I, I, I]
    lib.dc_aux_mlp_param_count.restype = Z
    lib.dc_aux_mlp_workspace_floats.argtypes = [I, I, I, I]
    lib.dc_aux_mlp_workspace_floats.restype = Z
    lib.dc_aux_mlp_forward.argtypes = [I, I, I, P, I, P, P, P, P]
    lib.dc_aux_mlp_loss_grad.argtypes = [I, I, I, P, I, P, P, P, P, P, P]
    lib.dc_aux_mlp_adam.argtypes = [Z, P, P, P, P, F, F, F, F, I, P]
    lib.dc_aux_feature_dims.argtypes = [P, P, P, P]
    lib.dc_aux_panel_features.argtypes = [P, P, P]
    lib.dc_aux_set_warm_start_model.argtypes = [P, I, P, I]
    lib.dc_aux_apply_operator.argtypes = [P, I, I, P, P]
    lib.dc_aux_precond_info.argtypes = [P, P]
    lib.dc_aux_build_timings.argtypes = [P, P]
    lib.dc_aux_test_skip_mma_tile.argtypes = [P, I]
    lib.dc_aux_fp32_peak.argtypes = [P, P]
    lib.dc_aux_time_inner_m2l.argtypes = [P, I, P]
    lib.dc_subdivide.argtypes = [P, ctypes.POINTER(dc_subdivide_options), ctypes.POINTER(dc_subdivide_stats)]
    lib.dc_get_panels.argtypes = [P, P, P]
    lib.dc_view_update.argtypes = [P, ctypes.POINTER(dc_viewport), ctypes.POINTER(dc_view_options),
                                   ctypes.POINTER(dc_view_stats)]
    lib.dc_view_reset.argtypes = [P]
    lib.dc_aux_tree_compare.argtypes = [P, P]
    lib.dc_aux_subdivision_info.argtypes = [P, P, P, P]
    lib.dc_aux_adaptive_panels.argtypes = [I, P, D, I, I, D, I, P, P, P]
    lib.dc_aux_discretise.argtypes = [I, P, P, P, P, I, I, P, P, P, P, P, P]
    lib.dc_autotune.argtypes = [P, I, ctypes.POINTER(dc_viewport), I, P, I, P, I, P, D, I,
                                ctypes.POINTER(dc_autotune_row), P]
    for name in EXPORTS:
        if name not in ("dc_destroy", "dc_last_error", "dc_status_string", "dc_abi_version",
                        "dc_aux_kernel_launches", "dc_aux_mlp_param_count",
                        "dc_aux_mlp_workspace_floats"):
            getattr(lib, name).restype = I
    _ = D
    return lib


_lib = None


def _get_lib():
    """The native library (loaded on first use; ImportError if not built)."""
    global _lib
    if _lib is None:
        _lib = _load()
    return _lib


def __getattr__(name):
    if name == "lib":
        return _get_lib()
    raise AttributeError(name)


class DcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"[{status}] {msg}")
        self.status = status


def _ptr(a) -> ctypes.c_void_p:
    if a is None:
        return ctypes.c_void_p(0)
    if isinstance(a, np.ndarray):
        return ctypes.c_void_p(a.ctypes.data)
    return ctypes.c_void_p(a.data_ptr())       # torch tensor


def _is_device(a) -> bool:
    return a is not None and not isinstance(a, np.ndarray) and a.is_cuda


def default_options(**overrides) -> dc_options:
    o = dc_options()
    _get_lib().dc_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        if k == "form" and isinstance(v, str):
            v = FORMS[v]
        if k == "domain":
            for i in range(4):
                o.domain[i] = float(v[i])
            continue
        setattr(o, k, v)
    return o


class Context:
    """One drawing on the current CUDA device (wraps a dc_ctx)."""

    def __init__(self, stream=None, **opts):
        if stream is None and torch is not None and torch.cuda.is_available():
            stream = torch.cuda.current_stream().cuda_stream
        self.options = default_options(stream=stream, **opts)
        h = ctypes.c_void_p()
        st = _get_lib().dc_create(ctypes.byref(h), ctypes.byref(self.options))
        if st != DC_OK:
            raise DcError(st, _get_lib().dc_last_error(None).decode())
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _get_lib().dc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int, allow=()):
        if st != DC_OK and st not in allow:
            raise DcError(st, _get_lib().dc_last_error(self._h).decode())
        return st

    # ------------------------------------------------------------ build --
    def build_tree(self, ctrl, panel_ptr, panel_start, colours):
        ctrl = np.ascontiguousarray(ctrl, dtype=np.float64)
        ptr = np.ascontiguousarray(panel_ptr, dtype=np.int32)
        start = np.ascontiguousarray(panel_start, dtype=np.float64)
        col = np.ascontiguousarray(colours, dtype=np.float64)
        self._check(_get_lib().dc_build_tree(self._h, int(ctrl.shape[0]), _ptr(ctrl), _ptr(ptr),
                                      _ptr(start), _ptr(col)))
        return self

    def build_curves(self, ctrl, colours):
        """dc_build_tree with the library's adaptive panel rule (panel_ptr
        and panel_start NULL)."""
        ctrl = np.ascontiguousarray(ctrl, dtype=np.float64)
        col = np.ascontiguousarray(colours, dtype=np.float64)
        self._check(_get_lib().dc_build_tree(self._h, int(ctrl.shape[0]), _ptr(ctrl), None, None, _ptr(col)))
        return self

    def build_drawing(self, drawing):
        return self.build_tree(drawing.ctrl, drawing.panel_ptr, drawing.panel_start,
                               drawing.colours)

    def sizes(self) -> dc_sizes:
        s = dc_sizes()
        self._check(_get_lib().dc_get_sizes(self._h, ctypes.byref(s)))
        return s

    def nodes(self):
        n = self.sizes().n_nodes
        xy, t = np.zeros((n, 2)), np.zeros(n)
        up, um = np.zeros((n, 3)), np.zeros((n, 3))
        self._check(_get_lib().dc_get_nodes(self._h, _ptr(xy), _ptr(t), _ptr(up), _ptr(um)))
        return xy, t, up, um

    # ------------------------------------------------------------ solve --
    def solve_density(self, x0=None, allow_noconv=False) -> dc_solve_stats:
        stats = dc_solve_stats()
        x = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
        allow = (DC_ERR_NOCONV,) if allow_noconv else ()
        self._check(_get_lib().dc_solve_density(self._h, _ptr(x), ctypes.byref(stats)), allow)
        return stats

    def solve_mixed(self, neumann, psi, u=None, allow_noconv=False) -> dc_solve_stats:
        """Mixed Dirichlet / Neumann solve (Sec. 4.3) on closed curves:
        neumann [n_panels] bool, psi [n_nodes, 3] = du/dn on the Neumann
        panels, u [n_nodes, 3] on the Dirichlet panels (None: the colours on
        the left of the curves)."""
        stats = dc_solve_stats()
        nm = np.ascontiguousarray(np.asarray(neumann, dtype=bool).astype(np.uint8))
        ps = np.ascontiguousarray(psi, dtype=np.float64)
        uu = None if u is None else np.ascontiguousarray(u, dtype=np.float64)
        n = self.sizes()
        if nm.shape != (n.n_panels,) or ps.shape != (n.n_nodes, 3) or (uu is not None and uu.shape != ps.shape):
            raise ValueError("solve_mixed: neumann must be [n_panels], psi and u [n_nodes, 3]")
        allow = (DC_ERR_NOCONV,) if allow_noconv else ()
        self._check(_get_lib().dc_solve_mixed(self._h, _ptr(nm), _ptr(ps), _ptr(uu), ctypes.byref(stats)), allow)
        return stats

    def get_density(self) -> np.ndarray:
        out = np.zeros((self.sizes().n_nodes, 3))
        self._check(_get_lib().dc_get_density(self._h, _ptr(out)))
        return out

    def set_density(self, sigma):
        s = np.ascontiguousarray(sigma, dtype=np.float64)
        self._check(_get_lib().dc_set_density(self._h, _ptr(s)))

    # ----------------------------------------------------------- render --
    def render_viewport(self, viewports, rgb=None, rgb8=None, stats=False):
        """viewports: list of (x0, y0, x1, y1, width, height).  rgb / rgb8:
        preallocated [sum h w, 3] arrays (torch CUDA tensors for device
        output, numpy arrays for host output); rgb float32 or float64."""
        n = len(viewports)
        arr = (dc_viewport * max(n, 1))()
        for i, v in enumerate(viewports):
            arr[i] = dc_viewport(float(v[0]), float(v[1]), float(v[2]), float(v[3]),
                                 int(v[4]), int(v[5]))
        where = DC_MEM_DEVICE if (_is_device(rgb) or _is_device(rgb8)) else DC_MEM_HOST
        dt = DC_F64
        if rgb is not None:
            dt = DC_F64 if str(rgb.dtype) in ("float64", "torch.float64") else DC_F32
        st = dc_render_stats()
        self._check(_get_lib().dc_render_viewport(self._h, n, arr, _ptr(rgb), dt, _ptr(rgb8), where,
                                           ctypes.byref(st) if stats else None))
        return st if stats else None

    def apply_operator(self, x, y, op=0, inner=False):
        """dc_aux_apply_operator: y = G_H x (op 0) or F_H x (op 1) at the
        nodes; x, y [n_nodes, 3] float64 torch CUDA tensors; inner 1 / 2:
        the FP32 inner operator with / without the preconditioner; inner 3:
        the preconditioner alone."""
        self._check(_get_lib().dc_aux_apply_operator(self._h, int(op), int(inner), _ptr(x),
                                                     _ptr(y)))
        return y

    def precond_info(self) -> dict:
        """dc_aux_precond_info as a dict."""
        out = np.zeros(5)
        self._check(_get_lib().dc_aux_precond_info(self._h, _ptr(out)))
        return dict(zip(["two_level", "panels", "near_pairs", "inverse_check", "aggregate"], out.tolist()))

    def test_skip_mma_tile(self, tile: int):
        """dc_aux_test_skip_mma_tile: hold back the MMAs of one tensor-core
        M2L tile (its bounded wait then runs out); -1 switches it off."""
        self._check(_get_lib().dc_aux_test_skip_mma_tile(self._h, int(tile)))

    # ---------------------------------------------------- subdivision --
    def subdivide(self, eps_coef, eps_len=0.0, resolve="local", label_ratio=0.0) -> dc_subdivide_stats:
        """dc_subdivide: one round of Alg. 5 and the re-solve of Alg. 7."""
        o = dc_subdivide_options(float(eps_coef), float(eps_len), RESOLVE.get(resolve, resolve),
                                 float(label_ratio))
        st = dc_subdivide_stats()
        self._check(_get_lib().dc_subdivide(self._h, ctypes.byref(o), ctypes.byref(st)))
        return st

    def view_update(self, viewport, eps_coef=0.0, eps_len_px=0.0, len_unit=0.0, resolve="local", max_rounds=0,
                    label_ratio=0.0) -> dc_view_stats:
        """dc_view_update: Alg. 9 for the viewport (x0, y0, x1, y1, width,
        height): viewport-masked subdivision and re-solve, then the
        evaluation polyline of e = length / 10 + s segments per panel that
        the next renders use."""
        v = dc_viewport(*[float(x) for x in viewport[:4]], int(viewport[4]), int(viewport[5]))
        o = dc_view_options(float(eps_coef), float(eps_len_px), float(len_unit), RESOLVE.get(resolve, resolve),
                            int(max_rounds), float(label_ratio))
        st = dc_view_stats()
        self._check(_get_lib().dc_view_update(self._h, ctypes.byref(v), ctypes.byref(o), ctypes.byref(st)))
        return st

    def tree_compare(self) -> dict:
        """dc_aux_tree_compare: the device-built quadtree against the host build."""
        out = np.zeros(6)
        self._check(_get_lib().dc_aux_tree_compare(self._h, _ptr(out)))
        return dict(identical=bool(out[0]), max_xy_diff=float(out[1]), cells=int(out[2]), pieces=int(out[3]),
                    ms_cut=float(out[4]), ms_lists=float(out[5]))

    def view_reset(self):
        self._check(_get_lib().dc_view_reset(self._h))

    def panels(self):
        """dc_get_panels: (panel_ptr, panel_start) of the current panels."""
        sz = self.sizes()
        ptr = np.zeros(sz.n_curves + 1, np.int32)
        start = np.zeros(sz.n_panels)
        self._check(_get_lib().dc_get_panels(self._h, _ptr(ptr), _ptr(start)))
        return ptr, start

    def subdivision_info(self, n_before: int):
        """dc_aux_subdivision_info: (top_old, split_old, resolve_new)."""
        top = np.zeros(n_before)
        split = np.zeros(n_before, np.uint8)
        res = np.zeros(self.sizes().n_panels, np.uint8)
        self._check(_get_lib().dc_aux_subdivision_info(self._h, _ptr(top), _ptr(split), _ptr(res)))
        return top, split.astype(bool), res.astype(bool)

    def autotune(self, viewports, leaf_sizes=(), p_inners=(), eval_tiles=(), tol=1e-5, repeats=2):
        """dc_autotune: (best row index or -1, list of row dicts).  The
        context is left built with the chosen options and no density."""
        n = len(viewports)
        arr = (dc_viewport * n)()
        for i, v in enumerate(viewports):
            arr[i] = dc_viewport(float(v[0]), float(v[1]), float(v[2]), float(v[3]), int(v[4]), int(v[5]))
        L = np.ascontiguousarray(leaf_sizes, dtype=np.int32)
        Pi = np.ascontiguousarray(p_inners, dtype=np.int32)
        T = np.ascontiguousarray(eval_tiles, dtype=np.int32)
        nrows = max(len(L), 1) * max(len(Pi), 1) * max(len(T), 1)
        rows = (dc_autotune_row * nrows)()
        best = ctypes.c_int(-1)
        self._check(_get_lib().dc_autotune(self._h, n, arr, len(L), _ptr(L) if len(L) else None, len(Pi),
                                           _ptr(Pi) if len(Pi) else None, len(T), _ptr(T) if len(T) else None,
                                           float(tol), int(repeats), rows, ctypes.byref(best)))
        keys = ["leaf_size", "p_inner", "eval_tile", "ms", "max_err", "converged"]
        return best.value, [{k: getattr(r, k) for k in keys} for r in rows]

    def time_inner_m2l(self, reps: int = 20) -> dict:
        """dc_aux_time_inner_m2l as a dict."""
        out = np.zeros(6)
        self._check(_get_lib().dc_aux_time_inner_m2l(self._h, int(reps), _ptr(out)))
        return dict(zip(["ms_main", "ms_reduce", "flops", "tensor_flops", "engine", "pairs"], out.tolist()))

    def build_timings(self) -> dict:
        """dc_aux_build_timings as a dict of wall ms per build phase."""
        out = np.zeros(11)
        self._check(_get_lib().dc_aux_build_timings(self._h, _ptr(out)))
        return dict(zip(["discretise", "upload", "tree_lists", "schedules", "preconditioner", "rows",
                         "near_far", "fp32", "features", "gh1", "total"], out.tolist()))

    # ---------------------------------------------------- warm start --
    def feature_dims(self):
        """(rows, n_features, n_out) of dc_aux_panel_features."""
        r, f, o = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(_get_lib().dc_aux_feature_dims(self._h, ctypes.byref(r), ctypes.byref(f),
                                                   ctypes.byref(o)))
        return r.value, f.value, o.value

    def panel_features(self, feat, target=None):
        """feat [rows, n_features] and target [rows, n_out] float32 torch
        CUDA tensors (target optional; needs a density)."""
        self._check(_get_lib().dc_aux_panel_features(self._h, _ptr(feat), _ptr(target)))
        return feat, target

    def set_warm_start_model(self, hidden, params):
        """params: float32 numpy array (host) or torch CUDA tensor; hidden 0
        removes the model."""
        if hidden == 0:
            self._check(_get_lib().dc_aux_set_warm_start_model(self._h, 0, None, DC_MEM_HOST))
            return
        where = DC_MEM_DEVICE if _is_device(params) else DC_MEM_HOST
        if where == DC_MEM_HOST:
            params = np.ascontiguousarray(params, dtype=np.float32)
        self._check(_get_lib().dc_aux_set_warm_start_model(self._h, int(hidden), _ptr(params), where))

    def eval_points_noalloc(self, xy, out):
        """dc_eval_points_noalloc: xy [n, 2] and out [n, 3] float64 torch
        CUDA tensors; nothing is allocated by the call."""
        self._check(_get_lib().dc_eval_points_noalloc(self._h, int(xy.shape[0]), _ptr(xy), _ptr(out)))
        return out

    def eval_points(self, xy, out):
        """xy [n, 2] float64 and out [n, 3] (float32/float64), both numpy
        (host) or both torch CUDA tensors (device)."""
        n = int(xy.shape[0])
        xw = DC_MEM_DEVICE if _is_device(xy) else DC_MEM_HOST
        ow = DC_MEM_DEVICE if _is_device(out) else DC_MEM_HOST
        dt = DC_F64 if str(out.dtype) in ("float64", "torch.float64") else DC_F32
        if isinstance(xy, np.ndarray):
            xy = np.ascontiguousarray(xy, dtype=np.float64)
        self._check(_get_lib().dc_eval_points(self._h, n, _ptr(xy), xw, _ptr(out), dt, ow))
        return out


def aux_tree_check(seg_xy, domain=(0.0, 0.0, 1.0, 1.0), leaf_size=64, max_depth=30):
    """Host-only quadtree check (dc_aux_tree_check): returns a dict."""
    seg = np.ascontiguousarray(seg_xy, dtype=np.float64).reshape(-1, 4)
    dom = np.ascontiguousarray(domain, dtype=np.float64)
    out = np.zeros(6)
    st = _get_lib().dc_aux_tree_check(int(seg.shape[0]), _ptr(seg), _ptr(dom), int(leaf_size),
                                      int(max_depth), _ptr(out))
    if st != DC_OK:
        raise DcError(st, "dc_aux_tree_check failed")
    keys = ["cells", "leaves", "depth", "pieces", "bad_pairs", "clip_rel_err"]
    return dict(zip(keys, out.tolist()))


def fp32_peak(stream=None) -> dict:
    """dc_aux_fp32_peak: measured FP32 FMA peak of the current device."""
    out = np.zeros(2)
    st = _get_lib().dc_aux_fp32_peak(_stream(stream), _ptr(out))
    if st != DC_OK:
        raise DcError(st, "dc_aux_fp32_peak failed")
    return {"tflops": float(out[0]), "ms": float(out[1])}


def aux_adaptive_panels(ctrl, ratio=0.2, max_level=8, min_panels=2, max_len=0.5):
    """Host-only adaptive panel rule (dc_aux_adaptive_panels):
    (panel_ptr, panel_start)."""
    ctrl = np.ascontiguousarray(ctrl, dtype=np.float64)
    n = int(ctrl.shape[0])
    ptr = np.zeros(n + 1, np.int32)
    cnt = ctypes.c_int()
    lib = _get_lib()
    lib.dc_aux_adaptive_panels(n, _ptr(ctrl), float(ratio), int(max_level), int(min_panels), float(max_len), 0,
                               _ptr(ptr), None, ctypes.byref(cnt))
    start = np.zeros(max(cnt.value, 1))
    st = lib.dc_aux_adaptive_panels(n, _ptr(ctrl), float(ratio), int(max_level), int(min_panels), float(max_len),
                                    cnt.value, _ptr(ptr), _ptr(start), ctypes.byref(cnt))
    if st != DC_OK:
        raise DcError(st, "dc_aux_adaptive_panels failed")
    return ptr, start[:cnt.value]


def aux_discretise(ctrl, panel_ptr, panel_start, colours, g=16, s_per_panel=80):
    """Host-only discretisation (dc_aux_discretise): dict of node_xy [N, 2],
    node_t [N], seg_xy [S, 4], seg_w [S], u_plus / u_minus [N, 3]."""
    ctrl = np.ascontiguousarray(ctrl, dtype=np.float64)
    ptr = np.ascontiguousarray(panel_ptr, dtype=np.int32)
    start = np.ascontiguousarray(panel_start, dtype=np.float64)
    col = np.ascontiguousarray(colours, dtype=np.float64)
    n = int(ctrl.shape[0])
    P = int(ptr[n])
    N, S = P * int(g), P * int(s_per_panel)
    out = dict(node_xy=np.zeros((N, 2)), node_t=np.zeros(N), seg_xy=np.zeros((S, 4)), seg_w=np.zeros(S),
               u_plus=np.zeros((N, 3)), u_minus=np.zeros((N, 3)))
    st = _get_lib().dc_aux_discretise(n, _ptr(ctrl), _ptr(ptr), _ptr(start), _ptr(col), int(g), int(s_per_panel),
                                      _ptr(out["node_xy"]), _ptr(out["node_t"]), _ptr(out["seg_xy"]),
                                      _ptr(out["seg_w"]), _ptr(out["u_plus"]), _ptr(out["u_minus"]))
    if st != DC_OK:
        raise DcError(st, "dc_aux_discretise failed")
    return out


def kernel_launches() -> int:
    """Kernels launched by libdc_fmm in this process so far."""
    return int(_get_lib().dc_aux_kernel_launches())


# ------------------------------------------------------------- network --
def _stream(stream):
    if stream is None and torch is not None and torch.cuda.is_available():
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(stream or 0)


def mlp_param_count(n_in: int, hidden: int, n_out: int) -> int:
    return int(_get_lib().dc_aux_mlp_param_count(n_in, hidden, n_out))


def mlp_workspace_floats(n_in: int, hidden: int, n_out: int, batch: int) -> int:
    return int(_get_lib().dc_aux_mlp_workspace_floats(n_in, hidden, n_out, batch))


def mlp_forward(n_in, hidden, n_out, params, x, y, work, stream=None):
    """dc_aux_mlp_forward on float32 torch CUDA tensors."""
    st = _get_lib().dc_aux_mlp_forward(n_in, hidden, n_out, _ptr(params), int(x.shape[0]), _ptr(x),
                                       _ptr(y), _ptr(work), _stream(stream))
    if st != DC_OK:
        raise DcError(st, "dc_aux_mlp_forward failed")
    return y


def mlp_loss_grad(n_in, hidden, n_out, params, x, target, grad, loss, work, stream=None):
    """dc_aux_mlp_loss_grad on float32 torch CUDA tensors (loss: 1 element)."""
    st = _get_lib().dc_aux_mlp_loss_grad(n_in, hidden, n_out, _ptr(params), int(x.shape[0]),
                                         _ptr(x), _ptr(target), _ptr(grad), _ptr(loss), _ptr(work),
                                         _stream(stream))
    if st != DC_OK:
        raise DcError(st, "dc_aux_mlp_loss_grad failed")


def mlp_adam(params, grad, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    """dc_aux_mlp_adam on float32 torch CUDA tensors."""
    st = _get_lib().dc_aux_mlp_adam(int(params.numel()), _ptr(params), _ptr(grad), _ptr(m), _ptr(v),
                                    float(lr), float(beta1), float(beta2), float(eps), int(step),
                                    _stream(stream))
    if st != DC_OK:
        raise DcError(st, "dc_aux_mlp_adam failed")
