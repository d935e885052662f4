"""Stored expected values (tests/golden/, written by make_golden.py from the
oracle alone): the oracle must keep reproducing them, and the library must
match them through the C ABI."""
import os

import numpy as np
import pytest

from dc_synth import drawing_by_name

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    a = np.loadtxt(os.path.join(HERE, name))
    return a[:, 0].astype(np.int64), a[:, 1:]


def test_oracle_reproduces_stored_values(oracle_mod):
    d = drawing_by_name("closed4")
    disc = oracle_mod.discretise(d)
    sol = oracle_mod.solve(d, disc)
    nodes, sig = load("closed4_sigma.txt")
    np.testing.assert_allclose(sol.sigma[nodes], sig, rtol=1e-12, atol=1e-12)
    pix, u = load("closed4_pixels.txt")
    got = oracle_mod.render(disc, sol, (0.0, 0.0, 1.0, 1.0), 128, 128, pix)
    np.testing.assert_allclose(got, u, rtol=1e-12, atol=1e-12)


@pytest.mark.gpu
# sigma bars (max error / max |sigma|) at the accuracy each form reaches on
# closed4: dense FP64 rows, FP64 FMM at p = 30 (App. E.1: the error decays
# geometrically in p), the chosen FP32 form after FP64 refinement
# (measured on GB300: 1.2e-11, 1.0e-10, 3.1e-10)
@pytest.mark.parametrize("form,tol,tol_sigma", [("dense64", 1e-10, 1e-9), ("fmm64", 1e-8, 1e-9),
                                                ("fmm32", 1e-5, 1e-8)])
def test_library_matches_stored_values(dcmod, cuda_ok, form, tol, tol_sigma):
    import torch
    d = drawing_by_name("closed4")
    extra = dict(p=30, leaf_size=32) if form == "fmm64" else {}
    ctx = dcmod.Context(form=form, g=d.g, s_per_panel=d.s_per_panel,
                        gmres_tol=1e-12 if form == "dense64" else 1e-10,
                        gmres_restart=400, gmres_max_iter=4000, **extra)
    ctx.build_drawing(d)
    ctx.solve_density()
    nodes, sig = load("closed4_sigma.txt")
    got = ctx.get_density()[nodes]
    scale = np.abs(sig).max()
    print(f"{form}: sigma max rel err {np.abs(got - sig).max() / scale:.2e}")
    assert np.abs(got - sig).max() <= tol_sigma * scale
    pix, u = load("closed4_pixels.txt")
    rgb = torch.empty((128 * 128, 3), dtype=torch.float64, device="cuda")
    ctx.render_viewport([(0.0, 0.0, 1.0, 1.0, 128, 128)], rgb)
    torch.cuda.synchronize()
    assert np.abs(rgb.cpu().numpy()[pix] - u).max() <= tol
