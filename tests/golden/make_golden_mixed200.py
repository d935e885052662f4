"""Writes stored expected values for the bench drawing "mixed200" under
tests/golden/ from the oracle alone (no GPU, no library):

  * the drawing: 200 cubic Bezier curves (120 open, 80 closed, seed
    20231126), adaptive panels, g = 16, s = 80: 27,888 unknowns per channel,
    139,440 segments;
  * G_H and F_H assembled densely row block by row block (Eq. 19, Eq. 27),
    b = (u+ + u-)/2 - F_H mu with mu = u+ - u- (Alg. 3), sigma = G_H^-1 b by
    LAPACK LU (one library step), for all three colour channels;
  * sigma at 512 seeded nodes;
  * the colour u (Eq. 23, Alg. 4) at 4096 pixel centres of the 2048 x 2048
    render of [0,1]^2, stratified: 2048 drawn uniformly over the image and
    2048 drawn uniformly among pixels whose centre lies within 0.003 (about
    six pixel widths, a few quadtree leaves) of a segment vertex, where the
    near-field closed forms decide the value.

Run from the repository root (about 3 minutes and 13 GB of host memory on an
8-core host):

    python tests/golden/make_golden_mixed200.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from dc_synth import drawing_by_name, pixel_sample  # noqa: E402
from oracle import oracle  # noqa: E402

W = H = 2048
VIEWPORT = (0.0, 0.0, 1.0, 1.0)
NODE_SEED, PIX_SEED, NEAR_SEED = 51, 52, 53
N_NODES, N_UNIFORM, N_NEAR = 512, 2048, 2048
NEAR_DIST = 0.003
BLOCK = 1024


def near_pixels(disc, count, seed):
    """Pixel indices whose centre lies within NEAR_DIST of a segment vertex."""
    from scipy.spatial import cKDTree
    verts = np.concatenate([disc.seg_xy[:, :2], disc.seg_xy[:, 2:]])
    tree = cKDTree(verts)
    allpix = oracle.pixel_centres(VIEWPORT, W, H)
    d, _ = tree.query(allpix, distance_upper_bound=NEAR_DIST)
    cand = np.flatnonzero(np.isfinite(d))
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(cand, size=count, replace=False)).astype(np.int64)


def main():
    t0 = time.time()
    d = drawing_by_name("mixed200")
    disc = oracle.discretise(d)
    N = disc.n_nodes
    up, um = oracle.boundary_values(d, disc)
    mu = up - um
    b = 0.5 * (up + um)
    AG = np.empty((N, N))
    for r0 in range(0, N, BLOCK):
        rows = np.arange(r0, min(N, r0 + BLOCK))
        g_blk, f_blk = oracle.hybrid_rows(disc, rows)
        AG[rows] = g_blk
        b[rows] -= f_blk @ mu
    t_asm = time.time() - t0
    t1 = time.time()
    sigma = np.linalg.solve(AG, b)
    t_lu = time.time() - t1
    rel_res = np.linalg.norm(AG @ sigma - b, axis=0) / np.linalg.norm(b, axis=0)
    del AG
    nodes = np.sort(np.random.default_rng(NODE_SEED).choice(N, N_NODES, replace=False))
    pu = pixel_sample(W, H, N_UNIFORM, seed=PIX_SEED)
    pn = near_pixels(disc, N_NEAR, NEAR_SEED)
    pix = np.unique(np.concatenate([pu, pn]))
    u = oracle.render(disc, oracle.Solution(sigma, mu, b), VIEWPORT, W, H, pix)
    near = np.isin(pix, pn)
    head = (f"# mixed200 (seed 20231126; {N} nodes, {disc.n_segments} segments): written by\n"
            f"# tests/golden/make_golden_mixed200.py from the oracle (dense G_H, F_H of Eq. 19/27,\n"
            f"# LU, Alg. 3); relative residual of the LU solve per channel "
            f"{rel_res[0]:.1e} {rel_res[1]:.1e} {rel_res[2]:.1e};\n"
            f"# assembly {t_asm:.0f} s, LU {t_lu:.0f} s on {oracle.num_threads()} threads\n")
    with open(os.path.join(HERE, "mixed200_sigma.txt"), "w") as f:
        f.write(head)
        f.write("# density sigma at seeded nodes; columns: node r g b\n")
        for i in nodes:
            f.write(f"{i:d} {sigma[i, 0]:.17e} {sigma[i, 1]:.17e} {sigma[i, 2]:.17e}\n")
    with open(os.path.join(HERE, "mixed200_pixels.txt"), "w") as f:
        f.write(head)
        f.write("# colour u (Eq. 23, Alg. 4) at pixel centres of the 2048x2048 render of [0,1]^2;\n")
        f.write("# columns: pixel index (row-major, row 0 at y = 0), near (1 = within 0.003 of a\n")
        f.write("# segment vertex), r g b\n")
        for k, i in enumerate(pix):
            f.write(f"{i:d} {int(near[k]):d} {u[k, 0]:.17e} {u[k, 1]:.17e} {u[k, 2]:.17e}\n")
    print(f"assembly {t_asm:.1f} s, LU {t_lu:.1f} s, residual {rel_res}, total {time.time() - t0:.1f} s")


if __name__ == "__main__":
    main()
