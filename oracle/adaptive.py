"""FP64 CPU oracle of adaptive subdivision and the local re-solve.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` alone, never by the product
path; it shares no code with the CUDA library.  Plain numpy on top of the
oracle's discretisation and dense rows (``oracle.py``).

Paper: Bang, Serkh, Stein, Jacobson, TOG 42(6) 215, 2023.
  * Sec. 6.1, Alg. 5: a panel is subdivided when the highest-order
    coefficient of the Legendre expansion of its density exceeds a global
    threshold epsilon_2, unless its length is below epsilon_1.  Reading taken
    here: the density's g node values on a panel are expanded as
    sum_k c_k P_k(x) on the panel's arc-length coordinate x in [-1, 1]
    (P_k(1) = 1); the test value is max over the colour channels of
    |c_{g-1}|; a panel splits into its two halves in arc-length fraction.
  * Sec. 6.1, warm start: the old density is interpolated to the new nodes,
    i.e. the old panel's Legendre expansion is evaluated there.
  * Sec. 6.3, Eq. 40-41 (label_curves): for each new panel alpha, v = G_H
    applied to the unit density on alpha; a panel beta needs re-solving when
    max v - min v over beta's nodes exceeds 0.9 times that over alpha.
    Reading: the paper's "curves" (its units of subdivision) are panels here,
    and each half of a split panel is one of the new curves S_alpha.
  * Sec. 6.3, local system: (G_H)_rr sigma_r = b_r - (G_H)_rc sigma_c with
    sigma_c the constrained panels' densities kept from the warm start.
    Reading: b = (u+ + u-)/2 - F_H mu of the refined discretisation, computed
    exactly (the paper re-interpolates b; Alg. 7 step 5).
"""
from __future__ import annotations

import numpy as np

from . import oracle as O


def _vandermonde(g: int) -> np.ndarray:
    """V[m, k] = P_k(x_m) at the g Gauss-Legendre nodes (Eq. 10-11)."""
    x, _ = O.gauss_legendre(g)
    return np.array([O.legendre_values(g, xm) for xm in x])


def legendre_coefficients(disc: O.Discretisation, sigma: np.ndarray) -> np.ndarray:
    """c[p, k, ch]: the Legendre coefficients of each panel's density, from
    V c = sigma (a plain linear solve per panel)."""
    g = disc.g
    S = np.asarray(sigma, np.float64).reshape(disc.n_panels, g, 3)
    V = _vandermonde(g)
    return np.stack([np.linalg.solve(V, S[p]) for p in range(disc.n_panels)])


def top_coefficient(disc: O.Discretisation, sigma: np.ndarray) -> np.ndarray:
    """Alg. 5's test value per panel: max over channels of |c_{g-1}|."""
    return np.abs(legendre_coefficients(disc, sigma)[:, disc.g - 1, :]).max(axis=1)


def panel_lengths(disc: O.Discretisation) -> np.ndarray:
    """Arc length of each panel: its segments' chords times their arc/chord
    weights (App. A)."""
    chord = np.hypot(disc.seg_xy[:, 2] - disc.seg_xy[:, 0], disc.seg_xy[:, 3] - disc.seg_xy[:, 1])
    return (chord * disc.seg_w).reshape(disc.n_panels, disc.nseg).sum(axis=1)


def subdivide(drawing, disc: O.Discretisation, sigma: np.ndarray, eps_coef: float, eps_len: float,
              mask=None):
    """Alg. 5: returns (refined drawing, split flags per old panel, pmap)
    with pmap[new panel] = (old panel, 0 kept / 1 left half / 2 right half).
    mask: panels that may split (Sec. 6.4: those within the viewport); all
    when None."""
    import copy
    top = top_coefficient(disc, sigma)
    length = panel_lengths(disc)
    split = (top > eps_coef) & (length >= eps_len)
    if mask is not None:
        split &= np.asarray(mask, bool)
    ptr, start = drawing.panel_ptr, drawing.panel_start
    new_ptr = [0]
    new_start, pmap = [], []
    for i in range(drawing.n_curves):
        for p in range(ptr[i], ptr[i + 1]):
            a = start[p]
            b = start[p + 1] if p + 1 < ptr[i + 1] else 1.0
            if split[p]:
                new_start += [a, 0.5 * (a + b)]
                pmap += [(p, 1), (p, 2)]
            else:
                new_start.append(a)
                pmap.append((p, 0))
        new_ptr.append(len(new_start))
    d2 = copy.copy(drawing)
    d2.panel_ptr = np.asarray(new_ptr, np.int32)
    d2.panel_start = np.asarray(new_start, np.float64)
    return d2, split, np.asarray(pmap, np.int64)


def warm_start(disc_old: O.Discretisation, sigma: np.ndarray, pmap: np.ndarray) -> np.ndarray:
    """Sec. 6.1: the old Legendre expansion of each panel at the nodes of the
    new panels (identity for kept panels)."""
    g = disc_old.g
    C = legendre_coefficients(disc_old, sigma)            # [P_old, g, 3]
    x, _ = O.gauss_legendre(g)
    S = np.asarray(sigma, np.float64).reshape(disc_old.n_panels, g, 3)
    out = np.zeros((len(pmap), g, 3))
    for q, (p, kind) in enumerate(pmap):
        if kind == 0:
            out[q] = S[p]
            continue
        xo = 0.5 * (x - 1.0) if kind == 1 else 0.5 * (x + 1.0)
        Pm = np.array([O.legendre_values(g, v) for v in xo])   # [n, k]
        out[q] = Pm @ C[p]
    return out.reshape(-1, 3)


def label_panels(disc_new: O.Discretisation, AG: np.ndarray, pmap: np.ndarray,
                 ratio: float = 0.9) -> np.ndarray:
    """Eq. 40-41: re-solving flags per new panel."""
    g, P = disc_new.g, disc_new.n_panels
    res = np.zeros(P, bool)
    alpha = [q for q in range(P) if pmap[q][1] != 0]
    for a in alpha:
        res[a] = True
        v = AG[:, a * g:(a + 1) * g].sum(axis=1)          # G_H applied to 1 on alpha
        V = v.reshape(P, g)
        rng = V.max(axis=1) - V.min(axis=1)
        res |= rng > ratio * rng[a]
    return res


def local_resolve(drawing_new, disc_new: O.Discretisation, sigma0: np.ndarray, res: np.ndarray,
                  AG: np.ndarray, AF: np.ndarray) -> np.ndarray:
    """Sec. 6.3: sigma_c = sigma0 on the constrained panels, sigma_r from
    (G_H)_rr sigma_r = b_r - (G_H)_rc sigma_c by LU."""
    up, um = O.boundary_values(drawing_new, disc_new)
    mu = up - um
    b = 0.5 * (up + um) - AF @ mu
    r = np.repeat(res, disc_new.g)
    c = ~r
    sigma = np.array(sigma0, np.float64, copy=True)
    rhs = b[r] - AG[np.ix_(r, c)] @ sigma[c]
    sigma[r] = np.linalg.solve(AG[np.ix_(r, r)], rhs)
    return sigma
