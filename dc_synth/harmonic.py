"""Closed-form harmonic functions for regions bounded by curves: boundary
data (values and normal derivatives) of mixed Dirichlet / Neumann problems,
and the exact solution inside to compare with.  Input generation only; none
of the boundary-integral method's arithmetic."""
from __future__ import annotations

import numpy as np

from .drawings import Drawing, curve_tangent


def fields(P: np.ndarray, hole=(0.45, 0.52)):
    """Three harmonic channels at points P [n, 2] and their gradients:
    exp(2x) cos(2y); x^2 - y^2 + xy + log|P - hole|; the constant 0.7.
    Returns u [n, 3] and grad [n, 2, 3]."""
    P = np.asarray(P, float)
    x, y = P[:, 0], P[:, 1]
    e = np.exp(2.0 * x)
    d = P - np.asarray(hole, float)
    r2 = (d ** 2).sum(1)
    u = np.stack([e * np.cos(2 * y), x * x - y * y + x * y + 0.5 * np.log(r2), np.full(len(x), 0.7)], 1)
    gx = np.stack([2 * e * np.cos(2 * y), 2 * x + y + d[:, 0] / r2, np.zeros(len(x))], 1)
    gy = np.stack([-2 * e * np.sin(2 * y), -2 * y + x + d[:, 1] / r2, np.zeros(len(x))], 1)
    return u, np.stack([gx, gy], 1)


def right_normals(drawing: Drawing, node_curve, node_t) -> np.ndarray:
    """Unit right-hand normals (T_y, -T_x) / |T| of the curves at the nodes;
    for a counter-clockwise outer loop and clockwise holes they point out of
    the region."""
    T = curve_tangent(drawing, node_curve, node_t)
    return np.stack([T[:, 1], -T[:, 0]], 1) / np.linalg.norm(T, axis=1)[:, None]


def boundary_data(drawing: Drawing, node_xy, node_curve, node_t, hole=(0.45, 0.52)):
    """u and du/dn (outward) of ``fields`` at the nodes: ([N, 3], [N, 3])."""
    u, grad = fields(node_xy, hole)
    n = right_normals(drawing, node_curve, node_t)
    return u, np.einsum("nk,nkc->nc", n, grad)
