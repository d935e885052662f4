"""FP64 CPU oracle of the viewport update (Sec. 6.2, 6.4; Alg. 9).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` alone, never by the product
path; it shares no code with the CUDA library.  Plain numpy on top of the
oracle's discretisation, dense rows and adaptive subdivision (``oracle.py``,
``adaptive.py``).

Sec. 6.2 renders with e line segments per curve, e = (length of curve) / 10
+ s, and Sec. 6.4 labels the curves for a viewport: fixed (outside it),
re-solving (subdivided, and their neighbours by Eq. 40-41), interpolating
(the rest of those that meet it; their density is carried to the finer
segments by Legendre interpolation).  Alg. 9 solves, then subdivides (Alg. 5,
epsilon_1 tied to the pixel size) and re-solves locally while panels split,
then renders.  Readings taken here:
  * the paper's "curves" in Sec. 6 are panels (as in ``adaptive.py``);
  * a panel meets the viewport when the bounding box of its solve polyline
    meets the viewport's closed rectangle;
  * only panels that meet the viewport may split; epsilon_1 = eps_len_px
    times the pixel size, the larger side of a pixel; eps_coef = 0 turns the
    subdivision off;
  * the length in the e rule is the panel's arc length in units of
    ``unit`` (default 1/512 of the unit canvas, the paper's 512-pixel
    images), rounded up: e_p = ceil(L_p / (10 unit)) + s;
  * one e for the whole drawing: the largest e_p over the panels that meet
    the viewport (s when none does); the render evaluates the layer
    potentials on the polyline of e equal arc-length segments per panel with
    sigma_bar = Lambda_e sigma at the same nodes (Eq. 23 with Lambda_e).
"""
from __future__ import annotations

import copy

import numpy as np

from . import adaptive as A
from . import oracle as O


def panel_boxes(disc: O.Discretisation) -> np.ndarray:
    """[P, 4] (x0, y0, x1, y1) of each panel's solve polyline."""
    seg = disc.seg_xy.reshape(disc.n_panels, disc.nseg, 4)
    xs = np.concatenate([seg[:, :, 0], seg[:, :, 2]], axis=1)
    ys = np.concatenate([seg[:, :, 1], seg[:, :, 3]], axis=1)
    return np.stack([xs.min(1), ys.min(1), xs.max(1), ys.max(1)], 1)


def meets_viewport(disc: O.Discretisation, viewport) -> np.ndarray:
    x0, y0, x1, y1 = viewport
    b = panel_boxes(disc)
    return (b[:, 2] >= x0) & (b[:, 0] <= x1) & (b[:, 3] >= y0) & (b[:, 1] <= y1)


def pixel_size(viewport, width: int, height: int) -> float:
    x0, y0, x1, y1 = viewport
    return max((x1 - x0) / width, (y1 - y0) / height)


def eval_segments(disc: O.Discretisation, meets: np.ndarray, unit: float = 1.0 / 512) -> int:
    """The e rule of Sec. 6.2 over the panels that meet the viewport."""
    if not np.any(meets):
        return disc.nseg
    L = A.panel_lengths(disc)[np.asarray(meets, bool)]
    return int(np.max(np.ceil(L / (10.0 * unit)))) + disc.nseg


def view_update(drawing, sigma, viewport, width: int, height: int, eps_coef: float, eps_len_px: float,
                unit: float = 1.0 / 512, max_rounds: int = 4, ratio: float = 0.9):
    """Alg. 9 from a solved density: rounds of viewport-masked subdivision
    and local re-solve, then the evaluation discretisation.  Returns a dict
    with the refined drawing, its discretisation, sigma, the evaluation
    discretisation (e segments per panel), e, the labels (0 fixed,
    1 interpolating, 2 re-solving in the last round), rounds and splits."""
    d = drawing
    disc = O.discretise(d)
    sig = np.asarray(sigma, np.float64).copy()
    h = pixel_size(viewport, width, height)
    resolve = np.zeros(disc.n_panels, bool)
    rounds = n_split = 0
    for _ in range(max_rounds if eps_coef > 0 else 0):   # eps_coef = 0: no subdivision
        m = meets_viewport(disc, viewport)
        d2, split, pmap = A.subdivide(d, disc, sig, eps_coef, eps_len_px * h, mask=m)
        if not split.any():
            break
        rounds += 1
        n_split += int(split.sum())
        disc2 = O.discretise(d2)
        AG, AF = O.hybrid_rows(disc2)
        s0 = A.warm_start(disc, sig, pmap)
        resolve = A.label_panels(disc2, AG, pmap, ratio)
        sig = A.local_resolve(d2, disc2, s0, resolve, AG, AF)
        d, disc = d2, disc2
    m = meets_viewport(disc, viewport)
    e = eval_segments(disc, m, unit)
    de = copy.copy(d)
    de.s_per_panel = e
    disc_e = O.discretise(de)
    labels = np.where(resolve, 2, np.where(m, 1, 0))
    return dict(drawing=d, disc=disc, sigma=sig, disc_e=disc_e, e=e, labels=labels, rounds=rounds,
                n_split=n_split)


def render(disc_e: O.Discretisation, sigma, mu, viewport, width: int, height: int, pixels) -> np.ndarray:
    """Colours at pixel centres on the evaluation polyline (Eq. 23 with the
    densities interpolated by Lambda_e from the same nodes)."""
    pts = O.pixel_centres(viewport, width, height, pixels)
    return O.layer_potential(disc_e, pts, sigma, mu)
