"""The bench workload at full size (200 curves, 27,888 nodes, 139,440
segments, 2048^2 pixels) in the launch configuration bench.py times.

The oracle cannot solve this size in bounded time, so:
  * the render is checked on sampled pixels against the oracle's direct sum
    with a seeded density set through the ABI (inputs from the generator);
  * the solve is checked through a property that holds at any size: its
    density, put into oracle rows of G_H and F_H (Eq. 27) at sampled nodes,
    leaves a residual far below the right-hand side.
"""
import numpy as np
import pytest

from dc_synth import drawing_by_name, pixel_sample, random_node_values

pytestmark = pytest.mark.gpu

W = H = 2048
OPTS = dict(p=24, leaf_size=64, gmres_tol=1e-10, gmres_restart=200, gmres_max_iter=3000)


@pytest.fixture(scope="module")
def big(oracle_mod):
    d = drawing_by_name("mixed200")
    disc = oracle_mod.discretise(d)
    return d, disc


def test_fullsize_render_sampled_pixels(dcmod, cuda_ok, big, oracle_mod):
    import torch
    d, disc = big
    up, um = oracle_mod.boundary_values(d, disc)
    sig = random_node_values(disc.n_nodes, seed=31, scale=5.0)
    ctx = dcmod.Context(form="fmm32", g=d.g, s_per_panel=d.s_per_panel, **OPTS)
    ctx.build_drawing(d)
    ctx.set_density(sig)
    rgb = torch.empty((W * H, 3), dtype=torch.float32, device="cuda")
    rgb8 = torch.empty((W * H, 3), dtype=torch.uint8, device="cuda")
    ctx.render_viewport([(0, 0, 1, 1, W, H)], rgb, rgb8)
    torch.cuda.synchronize()
    idx = pixel_sample(W, H, 2500, seed=32)
    ref = oracle_mod.layer_potential(disc, oracle_mod.pixel_centres((0, 0, 1, 1), W, H, idx),
                                     sig, up - um)
    got = rgb.cpu().numpy()[idx].astype(np.float64)
    err = np.abs(got - ref).max()
    print(f"full-size render, seeded density: max abs err {err:.2e} over {len(idx)} pixels "
          f"(|u| up to {np.abs(ref).max():.2f})")
    assert err <= 1e-5 * max(1.0, np.abs(ref).max())


def test_fullsize_solve_residual_property(dcmod, cuda_ok, big, oracle_mod):
    d, disc = big
    ctx = dcmod.Context(form="fmm32", g=d.g, s_per_panel=d.s_per_panel, **OPTS)
    ctx.build_drawing(d)
    st = ctx.solve_density()
    assert st.converged == 1 and max(st.rel_resid) <= 1e-10
    sig = ctx.get_density()
    rows = np.sort(np.random.default_rng(33).choice(disc.n_nodes, 256, replace=False))
    AG, AF = oracle_mod.hybrid_rows(disc, rows)
    up, um = oracle_mod.boundary_values(d, disc)
    b = 0.5 * (up[rows] + um[rows]) - AF @ (up - um)
    r = AG @ sig - b
    rel = np.abs(r).max() / np.abs(b).max()
    print(f"full-size solve: oracle-row residual {rel:.2e} (GMRES iters {list(st.iters)})")
    # the FMM (p = 24) approximates the exact rows to ~1e-8; a wrong solve
    # leaves O(1) residuals
    assert rel <= 1e-6
