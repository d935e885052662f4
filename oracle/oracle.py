"""FP64 CPU oracle of the hybrid BIE diffusion-curve method.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the package's smoke
check and by the benchmark's CPU-baseline leg, never by the product path.
It shares no code with the CUDA library.  The C part (``dc_oracle.c``) holds
the per-pair loops; this file orchestrates them with numpy, whose library
routines (``solve`` = LAPACK LU, ``@``) serve as single steps.

Paper: Bang, Serkh, Stein, Jacobson, "An Adaptive Fast-Multipole-Accelerated
Hybrid Boundary Integral Equation Method for Accurate Diffusion Curves",
TOG 42(6) 215, 2023.  Cited by section / equation / algorithm.

Readings of the paper taken here (the paper is silent or garbled):
  * nodes and segment vertices are placed in arc length (Sec. 4.2, App. B);
  * a node's collocation point is the point of the solve polyline at the
    node's arc length; its own segment is integrated with Eq. 52 / Eq. 53
    (App. C.1), both neighbours when it sits on a vertex;
  * "arc length integration" (App. A) scales each segment integral by
    (arc length of the segment) / (chord length);
  * the normal is the right-hand normal of the direction of travel; the "+"
    side is the side it points to (Eq. 21);
  * boundary colours are linear in the Bezier parameter t;
  * Eq. 50/51 (garbled) are replaced by antiderivatives written out from
    the integrands.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "dc_oracle.c")

_lib_handle = None


def build(force: bool = False) -> str:
    """Compile the C oracle (plain gcc, IEEE double, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _lib_handle
    if _lib_handle is None:
        lib = ctypes.CDLL(build())
        D, I = ctypes.c_double, ctypes.c_int
        P = ctypes.c_void_p
        lib.orc_num_threads.restype = I
        lib.orc_gauss_legendre.argtypes = [I, P, P]
        lib.orc_legendre_values.argtypes = [I, D, P]
        lib.orc_arclen.argtypes = [P, D]
        lib.orc_arclen.restype = D
        lib.orc_t_of_s.argtypes = [P, D, D]
        lib.orc_t_of_s.restype = D
        lib.orc_discretise.argtypes = [I, P, P, P, I, I, P, P, P, P, P, P, P, P]
        lib.orc_discretise.restype = I
        lib.orc_segment_GF.argtypes = [D, D, D, D, D, D, I, P, P]
        lib.orc_hybrid_rows.argtypes = [I, P, P, P, I, I, I, P, P, P, P, P]
        lib.orc_layer_potential.argtypes = [I, P, P, P, I, P, P, P, P, P]
        _lib_handle = lib
    return _lib_handle


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(_lib().orc_num_threads())


# ------------------------------------------------ Legendre (Eq. 10-11) --
def gauss_legendre(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    _lib().orc_gauss_legendre(n, _p(x), _p(w))
    return x, w


def legendre_values(n: int, x: float) -> np.ndarray:
    P = np.zeros(n)
    _lib().orc_legendre_values(n, float(x), _p(P))
    return P


def interpolation_matrix(g: int, nseg: int) -> np.ndarray:
    """Lambda = Pbar Pring^-1 (Sec. 4.2): maps the g node values of a panel
    to its nseg segment-midpoint values.  Pring[m, k] = P_k(x_m) at the
    Gauss-Legendre nodes, Pbar[j, k] = P_k(xbar_j) at the arc-length
    midpoints xbar_j = -1 + (2 j + 1) / nseg."""
    x, _ = gauss_legendre(g)
    Pring = np.array([legendre_values(g, xm) for xm in x])
    xbar = -1.0 + (2.0 * np.arange(nseg) + 1.0) / nseg
    Pbar = np.array([legendre_values(g, xb) for xb in xbar])
    return np.linalg.solve(Pring.T, Pbar.T).T


# ------------------------------------------------------- Bezier (App. B) --
def arclen(ctrl4x2: np.ndarray, t: float) -> float:
    c = np.ascontiguousarray(ctrl4x2, dtype=np.float64).reshape(8)
    return float(_lib().orc_arclen(_p(c), float(t)))


def t_of_s(ctrl4x2: np.ndarray, T: float, Ltot: float) -> float:
    c = np.ascontiguousarray(ctrl4x2, dtype=np.float64).reshape(8)
    return float(_lib().orc_t_of_s(_p(c), float(T), float(Ltot)))


# -------------------------------------------------------- discretisation --
@dataclass
class Discretisation:
    g: int
    nseg: int
    n_panels: int
    node_xy: np.ndarray
    node_t: np.ndarray
    node_seg: np.ndarray
    node_seg2: np.ndarray
    node_curve: np.ndarray
    seg_xy: np.ndarray
    seg_w: np.ndarray
    curve_len: np.ndarray
    Lambda: np.ndarray

    @property
    def n_nodes(self) -> int:
        return self.n_panels * self.g

    @property
    def n_segments(self) -> int:
        return self.n_panels * self.nseg


def discretise(drawing) -> Discretisation:
    g, nseg = int(drawing.g), int(drawing.s_per_panel)
    n = drawing.n_curves
    P = drawing.n_panels
    N, S = P * g, P * nseg
    ctrl = np.ascontiguousarray(drawing.ctrl, dtype=np.float64).reshape(n, 8)
    ptr = np.ascontiguousarray(drawing.panel_ptr, dtype=np.int32)
    start = np.ascontiguousarray(drawing.panel_start, dtype=np.float64)
    node_xy = np.zeros((N, 2))
    node_t = np.zeros(N)
    node_seg = np.zeros(N, np.int32)
    node_seg2 = np.zeros(N, np.int32)
    node_curve = np.zeros(N, np.int32)
    seg_xy = np.zeros((S, 4))
    seg_w = np.zeros(S)
    curve_len = np.zeros(n)
    rc = _lib().orc_discretise(n, _p(ctrl), _p(ptr), _p(start), g, nseg,
                               _p(node_xy), _p(node_t), _p(node_seg),
                               _p(node_seg2), _p(node_curve), _p(seg_xy),
                               _p(seg_w), _p(curve_len))
    if rc != 0:
        raise RuntimeError("oracle discretisation failed")
    return Discretisation(g, nseg, P, node_xy, node_t, node_seg, node_seg2,
                          node_curve, seg_xy, seg_w, curve_len,
                          interpolation_matrix(g, nseg))


def boundary_values(drawing, disc: Discretisation):
    """u+ and u- at the nodes: colours linear in the Bezier parameter t."""
    t = disc.node_t[:, None]
    col = drawing.colours[disc.node_curve]          # [N, side, end, 3]
    u_plus = (1.0 - t) * col[:, 0, 0, :] + t * col[:, 0, 1, :]
    u_minus = (1.0 - t) * col[:, 1, 0, :] + t * col[:, 1, 1, :]
    return u_plus, u_minus


def to_segments(disc: Discretisation, node_vals: np.ndarray) -> np.ndarray:
    """sigma_bar = Pbar Pring^-1 sigma_ring, panel by panel (Sec. 4.2)."""
    v = node_vals.reshape(disc.n_panels, disc.g, -1)
    out = np.einsum("kg,pgc->pkc", disc.Lambda, v)
    return out.reshape(disc.n_panels * disc.nseg, -1)


# ------------------------------------------------- closed forms (App. D) --
def segment_GF(p1, p2, q, singular: bool = False):
    G = ctypes.c_double()
    F = ctypes.c_double()
    _lib().orc_segment_GF(float(p1[0]), float(p1[1]), float(p2[0]), float(p2[1]),
                          float(q[0]), float(q[1]), int(bool(singular)),
                          ctypes.byref(G), ctypes.byref(F))
    return G.value, F.value


def hybrid_rows(disc: Discretisation, rows=None):
    """Rows of G_H and F_H (Eq. 19, Eq. 27) at the collocation nodes."""
    idx = np.arange(disc.n_nodes) if rows is None else np.asarray(rows)
    txy = np.ascontiguousarray(disc.node_xy[idx])
    ts = np.ascontiguousarray(disc.node_seg[idx])
    ts2 = np.ascontiguousarray(disc.node_seg2[idx])
    ncol = disc.n_nodes
    AG = np.zeros((len(idx), ncol))
    AF = np.zeros((len(idx), ncol))
    lam = np.ascontiguousarray(disc.Lambda)
    _lib().orc_hybrid_rows(len(idx), _p(txy), _p(ts), _p(ts2), disc.n_panels,
                           disc.nseg, disc.g, _p(disc.seg_xy), _p(disc.seg_w),
                           _p(lam), _p(AG), _p(AF))
    return AG, AF


def layer_potential(disc: Discretisation, points: np.ndarray, sigma_nodes,
                    mu_nodes, tgt_seg=None, tgt_seg2=None) -> np.ndarray:
    """u(x) = sum over segments of sigma_bar int G + mu_bar int F (Eq. 23)."""
    pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 2)
    sb = np.ascontiguousarray(to_segments(disc, np.asarray(sigma_nodes, np.float64)))
    mb = np.ascontiguousarray(to_segments(disc, np.asarray(mu_nodes, np.float64)))
    u = np.zeros((pts.shape[0], 3))
    s1 = None if tgt_seg is None else np.ascontiguousarray(tgt_seg, dtype=np.int32)
    s2 = None if tgt_seg2 is None else np.ascontiguousarray(tgt_seg2, dtype=np.int32)
    _lib().orc_layer_potential(pts.shape[0], _p(pts),
                               None if s1 is None else _p(s1),
                               None if s2 is None else _p(s2),
                               disc.n_segments, _p(disc.seg_xy), _p(disc.seg_w),
                               _p(sb), _p(mb), _p(u))
    return u


# ------------------------------------------------- solve (Alg. 3, Eq. 27) --
@dataclass
class Solution:
    sigma: np.ndarray      # [N, 3] density at the nodes
    mu: np.ndarray         # [N, 3] jump u+ - u- at the nodes
    b: np.ndarray          # [N, 3] right-hand side
    AG: np.ndarray | None = None


def solve_values(disc: Discretisation, u_plus: np.ndarray, u_minus: np.ndarray,
                 keep_matrix=False) -> Solution:
    """Solve Eq. 27 for sigma given u+ and u- at the nodes: mu = u+ - u-,
    b = (u+ + u-)/2 - F_H mu, sigma = G_H^-1 b by dense LU."""
    AG, AF = hybrid_rows(disc)
    mu = u_plus - u_minus
    b = 0.5 * (u_plus + u_minus) - AF @ mu
    sigma = np.linalg.solve(AG, b)
    return Solution(sigma, mu, b, AG if keep_matrix else None)


def solve(drawing, disc: Discretisation | None = None, keep_matrix=False) -> Solution:
    """Alg. 3 with a direct solve: colours of the drawing as u+ / u-."""
    disc = disc or discretise(drawing)
    up, um = boundary_values(drawing, disc)
    return solve_values(disc, up, um, keep_matrix)


def gmres(matvec, b: np.ndarray, x0: np.ndarray, tol: float, restart: int = 200,
          maxiter: int = 2000):
    """Plain GMRES(restart) with modified Gram-Schmidt and Givens rotations,
    stopping at ||b - A x|| <= tol ||b|| (Sec. 5.5, GMRES(f, x0, y, eps))."""
    x = x0.astype(np.float64).copy()
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return np.zeros_like(b), 0, 0.0
    it = 0
    while True:
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        if beta <= tol * nb or it >= maxiter:
            return x, it, beta / nb
        m = restart
        V = np.zeros((m + 1, b.size))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        e = np.zeros(m + 1)
        e[0] = beta
        V[0] = r / beta
        k_done = 0
        for k in range(m):
            w = matvec(V[k])
            for j in range(k + 1):
                H[j, k] = np.dot(V[j], w)
                w = w - H[j, k] * V[j]
            H[k + 1, k] = np.linalg.norm(w)
            if H[k + 1, k] != 0.0:
                V[k + 1] = w / H[k + 1, k]
            for j in range(k):
                a, bb = H[j, k], H[j + 1, k]
                H[j, k] = cs[j] * a + sn[j] * bb
                H[j + 1, k] = -sn[j] * a + cs[j] * bb
            den = np.hypot(H[k, k], H[k + 1, k])
            cs[k], sn[k] = H[k, k] / den, H[k + 1, k] / den
            H[k, k] = den
            H[k + 1, k] = 0.0
            e[k + 1] = -sn[k] * e[k]
            e[k] = cs[k] * e[k]
            it += 1
            k_done = k + 1
            if abs(e[k + 1]) <= tol * nb or it >= maxiter:
                break
        y = np.linalg.solve(np.triu(H[:k_done, :k_done]), e[:k_done])
        x = x + V[:k_done].T @ y


# ------------------------------------------------------ render (Alg. 4) --
def pixel_centres(viewport, width: int, height: int, idx=None) -> np.ndarray:
    """Pixel (r, c) -> (x0 + (c + 1/2) dx, y0 + (r + 1/2) dy); row 0 at y0."""
    x0, y0, x1, y1 = viewport
    if idx is None:
        idx = np.arange(width * height)
    idx = np.asarray(idx, dtype=np.int64)
    r, c = idx // width, idx % width
    return np.stack([x0 + (c + 0.5) * (x1 - x0) / width,
                     y0 + (r + 0.5) * (y1 - y0) / height], axis=1)


def render(disc: Discretisation, sol: Solution, viewport, width: int, height: int,
           idx=None) -> np.ndarray:
    """u at pixel centres = single layer of sigma + double layer of mu."""
    pts = pixel_centres(viewport, width, height, idx)
    return layer_potential(disc, pts, sol.sigma, sol.mu)


def quantise(u: np.ndarray) -> np.ndarray:
    """8-bit colour: floor(255 clamp(u, 0, 1) + 1/2)."""
    return np.floor(255.0 * np.clip(u, 0.0, 1.0) + 0.5).astype(np.uint8)
