"""Writes the stored expected values under tests/golden/ from the oracle
alone (no GPU, no library): the closed4 drawing (4 closed cubics, 16 panels
of 16 Gauss-Legendre nodes each, seed 20231125), its density from the dense
LU solve of the hybrid system (Eq. 27, Alg. 3) at 24 seeded nodes, and its
colour (Eq. 23, Alg. 4) at 32 seeded pixel centres of the 128 x 128 render of
[0,1]^2.  Run from the repository root:

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from dc_synth import drawing_by_name  # noqa: E402
from oracle import oracle  # noqa: E402

W = H = 128
NODE_SEED, PIX_SEED = 41, 42


def main():
    d = drawing_by_name("closed4")
    disc = oracle.discretise(d)
    sol = oracle.solve(d, disc)
    nodes = np.sort(np.random.default_rng(NODE_SEED).choice(disc.n_nodes, 24, replace=False))
    pix = np.sort(np.random.default_rng(PIX_SEED).choice(W * H, 32, replace=False))
    u = oracle.render(disc, sol, (0.0, 0.0, 1.0, 1.0), W, H, pix)
    with open(os.path.join(HERE, "closed4_sigma.txt"), "w") as f:
        f.write("# closed4 (seed 20231125): density sigma at nodes, dense LU solve of Eq. 27\n")
        f.write("# written by tests/golden/make_golden.py from the oracle; columns: node r g b\n")
        for i in nodes:
            f.write(f"{i:d} {sol.sigma[i, 0]:.17e} {sol.sigma[i, 1]:.17e} {sol.sigma[i, 2]:.17e}\n")
    with open(os.path.join(HERE, "closed4_pixels.txt"), "w") as f:
        f.write("# closed4 (seed 20231125): colour u at pixel centres of the 128x128 render of\n")
        f.write("# [0,1]^2 (Eq. 23, Alg. 4); written by tests/golden/make_golden.py from the\n")
        f.write("# oracle; columns: pixel index (row-major, row 0 at y = 0) r g b\n")
        for k, i in enumerate(pix):
            f.write(f"{i:d} {u[k, 0]:.17e} {u[k, 1]:.17e} {u[k, 2]:.17e}\n")


if __name__ == "__main__":
    main()
