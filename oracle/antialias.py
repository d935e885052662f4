"""FP64 CPU oracle of the quadtree anti-aliasing of Sec. 7.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` alone, never by the product
path; it shares no code with the CUDA library.  Plain numpy and Python loops
on top of the oracle's discretisation and direct sum (``oracle.py``).

Sec. 7 replaces the centre sample of a pixel by an area-weighted mean: a
cell's value is the area-weighted sum of its children's values, cells that
hold a boundary curve are subdivided below the pixel size, and the other
cells keep one sample.  Readings taken here:
  * a cell "holds a curve" when its closed rectangle meets a closed segment
    of the solve polyline (the segments the colours are integrated over);
  * the hierarchy is per pixel: the pixel is level 0, a cell of level k < m
    that meets a segment splits into its four quarters (children ordered
    lower-left, lower-right, upper-left, upper-right), every cell that does
    not split takes u at its centre, weighted by its area (4^-k of the
    pixel); m = ``levels`` >= 1;
  * a pixel that meets no segment keeps its centre sample;
  * corners and centres of a cell of level k in pixel (c, r) of a viewport
    with lower-left corner (x0, y0) and pixel size (dx, dy) are
    x0 + (c + f) dx, y0 + (r + f') dy with dyadic fractions f, f' (the
    product and the sum each rounded once), so the decisions are the same
    IEEE operations wherever they are made.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O

TIE = 1e-11     # world units: decisions this close to flipping are reported


def meets(seg: np.ndarray, x0: float, y0: float, x1: float, y1: float):
    """Closed segments seg [n, 4] (px, py, qx, qy) against the closed
    rectangle [x0, x1] x [y0, y1] by separating axes: the boxes overlap and
    the rectangle's corners are not all strictly on one side of the
    segment's line.  Returns (meets [n] bool, tie [n] bool)."""
    px, py, qx, qy = seg[:, 0], seg[:, 1], seg[:, 2], seg[:, 3]
    lo_x, hi_x = np.minimum(px, qx), np.maximum(px, qx)
    lo_y, hi_y = np.minimum(py, qy), np.maximum(py, qy)
    box = (hi_x >= x0) & (lo_x <= x1) & (hi_y >= y0) & (lo_y <= y1)
    ex, ey = qx - px, qy - py
    s = np.stack([ex * (cy - py) - ey * (cx - px)
                  for cx, cy in ((x0, y0), (x1, y0), (x0, y1), (x1, y1))])
    one_side = np.all(s > 0, axis=0) | np.all(s < 0, axis=0)
    box_margin = np.min(np.abs(np.stack([hi_x - x0, x1 - lo_x, hi_y - y0, y1 - lo_y])), axis=0)
    line_dist = np.min(np.abs(s), axis=0) / np.maximum(np.hypot(ex, ey), 1e-300)
    tie = (box_margin < TIE) | (box & (line_dist < TIE))
    return box & ~one_side, tie


def pixel_samples(seg: np.ndarray, viewport, width: int, height: int, pixel: int, levels: int):
    """Sample points and area weights of one pixel (row-major index, row 0
    at the viewport's bottom edge): ([k, 2], [k], edge, tie)."""
    vx0, vy0, vx1, vy1 = viewport
    dx, dy = (vx1 - vx0) / width, (vy1 - vy0) / height
    r, c = divmod(int(pixel), int(width))
    pts, wts = [], []
    tie_any = False

    def visit(k, i, j, cand):
        nonlocal tie_any
        h = 2.0 ** -k
        fx0, fx1 = c + i * h, c + (i + 1) * h
        fy0, fy1 = r + j * h, r + (j + 1) * h
        m, t = meets(cand, vx0 + fx0 * dx, vy0 + fy0 * dy, vx0 + fx1 * dx, vy0 + fy1 * dy)
        tie_any = tie_any or bool(t.any())
        if k == levels or not m.any():
            pts.append((vx0 + (c + (i + 0.5) * h) * dx, vy0 + (r + (j + 0.5) * h) * dy))
            wts.append(h * h)
            return k > 0
        sub = cand[m]
        for a, b in ((0, 0), (1, 0), (0, 1), (1, 1)):
            visit(k + 1, 2 * i + a, 2 * j + b, sub)
        return True

    edge = visit(0, 0, 0, seg)
    return np.asarray(pts), np.asarray(wts), edge, tie_any


def render_aa(disc: O.Discretisation, sigma, mu, viewport, width: int, height: int,
              pixels, levels: int):
    """Anti-aliased colours at the given pixels: Sum_j w_j u(x_j) over each
    pixel's samples, u by the direct sum of Eq. 23.  Returns (u [n, 3],
    edge [n] bool, tie [n] bool, samples [n] int)."""
    seg = np.ascontiguousarray(disc.seg_xy, np.float64)
    vx0, vy0, vx1, vy1 = viewport
    dx, dy = (vx1 - vx0) / width, (vy1 - vy0) / height
    allp, allw, owner = [], [], []
    edge = np.zeros(len(pixels), bool)
    tie = np.zeros(len(pixels), bool)
    nsamp = np.zeros(len(pixels), int)
    pad = 2 * TIE
    for n, p in enumerate(pixels):
        r, c = divmod(int(p), int(width))
        # segments whose box can touch the pixel (a superset; meets decides)
        near = seg[(np.maximum(seg[:, 0], seg[:, 2]) >= vx0 + c * dx - pad)
                   & (np.minimum(seg[:, 0], seg[:, 2]) <= vx0 + (c + 1) * dx + pad)
                   & (np.maximum(seg[:, 1], seg[:, 3]) >= vy0 + r * dy - pad)
                   & (np.minimum(seg[:, 1], seg[:, 3]) <= vy0 + (r + 1) * dy + pad)]
        P, W, e, t = pixel_samples(near, viewport, width, height, p, levels)
        edge[n], tie[n], nsamp[n] = e, t, len(W)
        allp.append(P)
        allw.append(W)
        owner.append(np.full(len(W), n))
    P = np.concatenate(allp)
    W = np.concatenate(allw)
    own = np.concatenate(owner)
    u = O.layer_potential(disc, P, sigma, mu)
    out = np.zeros((len(pixels), 3))
    np.add.at(out, own, W[:, None] * u)
    return out, edge, tie, nsamp


def edge_pixels(disc: O.Discretisation, viewport, width: int, height: int):
    """Row-major indices of the pixels whose closed square meets a segment
    (the pixels Sec. 7 refines), and of those whose decision is a tie.
    Every (segment, pixel) pair within one pixel of the segment's box is
    tested with ``meets``."""
    seg = np.ascontiguousarray(disc.seg_xy, np.float64)
    vx0, vy0, vx1, vy1 = viewport
    dx, dy = (vx1 - vx0) / width, (vy1 - vy0) / height
    lox, hix = np.minimum(seg[:, 0], seg[:, 2]), np.maximum(seg[:, 0], seg[:, 2])
    loy, hiy = np.minimum(seg[:, 1], seg[:, 3]), np.maximum(seg[:, 1], seg[:, 3])
    c0 = np.clip(np.floor((lox - vx0) / dx) - 1, 0, width - 1).astype(np.int64)
    c1 = np.clip(np.floor((hix - vx0) / dx) + 1, 0, width - 1).astype(np.int64)
    r0 = np.clip(np.floor((loy - vy0) / dy) - 1, 0, height - 1).astype(np.int64)
    r1 = np.clip(np.floor((hiy - vy0) / dy) + 1, 0, height - 1).astype(np.int64)
    inside = (np.floor((hix - vx0) / dx) + 1 >= 0) & (np.floor((lox - vx0) / dx) - 1 <= width - 1) \
        & (np.floor((hiy - vy0) / dy) + 1 >= 0) & (np.floor((loy - vy0) / dy) - 1 <= height - 1)
    nc, nr = c1 - c0 + 1, r1 - r0 + 1
    k = np.where(inside, nc * nr, 0)
    sid = np.repeat(np.arange(len(seg)), k)
    j = np.arange(k.sum()) - np.repeat(np.cumsum(k) - k, k)
    c = c0[sid] + j % nc[sid]
    r = r0[sid] + j // nc[sid]
    m, t = meets(seg[sid], vx0 + c * dx, vy0 + r * dy, vx0 + (c + 1) * dx, vy0 + (r + 1) * dy)
    pix = r * width + c
    return np.unique(pix[m]), np.unique(pix[t])
