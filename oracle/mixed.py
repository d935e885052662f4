"""FP64 CPU oracle of mixed Dirichlet / Neumann conditions on closed curves.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` alone, never by the product
path; it shares no code with the CUDA library.  Plain numpy on top of the
oracle's discretisation and dense rows (``oracle.py``).

Paper: Bang, Serkh, Stein, Jacobson, TOG 42(6) 215, 2023, Sec. 4.3 (Neumann
boundary condition).  For a region V bounded by closed curves, Green's third
identity represents u inside by its boundary values and normal derivatives;
at the Gauss-Legendre nodes, with u* given on the Dirichlet panels and
psi* = du/dn on the Neumann panels, the unknowns are psi on the Dirichlet
panels and u on the Neumann panels (the block system of Sec. 4.3).

Readings taken here (the conventions of oracle.py):
  * curves are closed and counter-clockwise, so the right-hand normal n points
    out of V and the inside is the "-" side; psi = du/dn along that n;
  * the layer densities of the representation are sigma = psi and
    mu = u+ - u- = 0 - u = -u (u vanishes outside by Green's identity), and
    on the curve from inside u = G_H sigma + F_H mu - mu / 2 (jump of the
    double layer), i.e.  u / 2 = G_H psi - F_H u  at the nodes;
  * the Dirichlet data are the drawing's inside colours u- at the nodes.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O


def signed_areas(drawing, disc: O.Discretisation) -> np.ndarray:
    """Signed area of each curve's solve polyline (shoelace formula);
    positive for a counter-clockwise curve."""
    seg = disc.seg_xy.reshape(drawing.n_panels, disc.nseg, 4)
    areas = np.zeros(drawing.n_curves)
    for i in range(drawing.n_curves):
        s = seg[drawing.panel_ptr[i]:drawing.panel_ptr[i + 1]].reshape(-1, 4)
        areas[i] = 0.5 * np.sum(s[:, 0] * s[:, 3] - s[:, 2] * s[:, 1])
    return areas


def solve_mixed(drawing, disc: O.Discretisation, neumann_panels: np.ndarray, psi_star: np.ndarray,
                u_star: np.ndarray | None = None):
    """Sec. 4.3's block system by dense LU.  neumann_panels: [n_panels] bool;
    psi_star: [N, 3] du/dn on the Neumann nodes (other rows ignored);
    u_star: [N, 3] Dirichlet values (default: the drawing's inside colours).
    Returns (sigma, mu, psi_d_and_u_n) with sigma = psi, mu = -u at every node."""
    g = disc.g
    nmask = np.repeat(np.asarray(neumann_panels, bool), g)
    dmask = ~nmask
    AG, AF = O.hybrid_rows(disc)
    u_minus = O.boundary_values(drawing, disc)[1] if u_star is None else np.asarray(u_star, np.float64)
    N = disc.n_nodes
    half_plus_F = 0.5 * np.eye(N) + AF
    A = np.zeros((N, N))
    A[:, dmask] = AG[:, dmask]
    A[:, nmask] = -half_plus_F[:, nmask]
    u_d = np.where(dmask[:, None], u_minus, 0.0)
    psi_n = np.where(nmask[:, None], psi_star, 0.0)
    b = half_plus_F @ u_d - AG @ psi_n
    x = np.linalg.solve(A, b)
    psi = np.where(dmask[:, None], x, psi_n)
    u = np.where(nmask[:, None], x, u_d)
    return psi, -u, x
