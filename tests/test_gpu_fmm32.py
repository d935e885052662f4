"""Chosen form (FP32 FMM, FP64 GMRES with iterative refinement) on the GPU
against the FP64 oracle.  Bar: 1e-5 absolute colour error (colours in
[0, 1]) and identical 8-bit output for every pixel whose oracle colour is
farther than 1e-5 from a rounding boundary."""
import numpy as np
import pytest

from dc_synth import drawing_by_name, pixel_sample, random_node_values

pytestmark = pytest.mark.gpu

TOL_COLOUR = 1e-5


def band_mask(u_ref, tol):
    v = 255.0 * np.clip(u_ref, 0, 1)
    return np.abs(v - np.floor(v) - 0.5) <= 255.0 * tol + 1e-12


def quant(u):
    return np.floor(255 * np.clip(u, 0, 1) + 0.5).astype(np.uint8)


@pytest.fixture(scope="module")
def closed4(oracle_mod):
    d = drawing_by_name("closed4")
    disc = oracle_mod.discretise(d)
    sol = oracle_mod.solve(d, disc)
    u = oracle_mod.render(disc, sol, (0, 0, 1, 1), 128, 128)
    return d, disc, sol, u


@pytest.fixture(scope="module")
def mixed16(oracle_mod):
    d = drawing_by_name("mixed16")
    disc = oracle_mod.discretise(d)
    sol = oracle_mod.solve(d, disc)
    return d, disc, sol


def make_ctx(P, d, **kw):
    kw.setdefault("gmres_tol", 1e-10)
    ctx = P.Context(form="fmm32", g=d.g, s_per_panel=d.s_per_panel, **kw)
    ctx.build_drawing(d)
    return ctx


def test_fmm32_solve_closed4(dcmod, cuda_ok, closed4):
    import torch
    d, disc, sol, u_ref = closed4
    ctx = make_ctx(dcmod, d, p=24, leaf_size=32)
    st = ctx.solve_density()
    assert st.converged == 1 and max(st.rel_resid) <= 1e-10
    sig = ctx.get_density()
    es = np.abs(sig - sol.sigma).max() / np.abs(sol.sigma).max()
    rgb = torch.empty((128 * 128, 3), dtype=torch.float32, device="cuda")
    rgb8 = torch.empty((128 * 128, 3), dtype=torch.uint8, device="cuda")
    ctx.render_viewport([(0, 0, 1, 1, 128, 128)], rgb, rgb8)
    torch.cuda.synchronize()
    u = rgb.cpu().numpy().astype(np.float64)
    ep = np.abs(u - u_ref).max()
    ok = ~band_mask(u_ref, TOL_COLOUR)
    mism = int((rgb8.cpu().numpy()[ok] != quant(u_ref)[ok]).sum())
    print(f"fmm32 closed4: iters {list(st.iters)} matvecs {st.n_matvec} sigma rel {es:.2e} "
          f"pixel abs {ep:.2e} band {int((~ok).sum())} 8-bit mismatches {mism}")
    assert es <= 1e-6
    assert ep <= TOL_COLOUR
    assert mism == 0


def test_fmm32_solve_mixed16(dcmod, cuda_ok, mixed16, oracle_mod):
    d, disc, sol = mixed16
    ctx = make_ctx(dcmod, d, p=24, leaf_size=16)
    st = ctx.solve_density()
    assert st.converged == 1
    sig = ctx.get_density()
    es = np.abs(sig - sol.sigma).max() / np.abs(sol.sigma).max()
    W = H = 256
    idx = pixel_sample(W, H, 4000, seed=8)
    ref = oracle_mod.render(disc, sol, (0, 0, 1, 1), W, H, idx)
    out = np.zeros((W * H, 3), np.float32)
    ctx.render_viewport([(0, 0, 1, 1, W, H)], out)
    ep = np.abs(out[idx] - ref).max()
    print(f"fmm32 mixed16: iters {list(st.iters)} sigma rel {es:.2e} pixel abs {ep:.2e}")
    assert es <= 1e-6
    assert ep <= TOL_COLOUR


@pytest.mark.parametrize("leaf", [4, 16, 64])
def test_fmm32_render_deep_trees(dcmod, cuda_ok, mixed16, oracle_mod, leaf):
    d, disc, sol = mixed16
    ctx = make_ctx(dcmod, d, p=24, leaf_size=leaf)
    ctx.set_density(sol.sigma)
    W = H = 256
    idx = pixel_sample(W, H, 3000, seed=9)
    out = np.zeros((W * H, 3))
    ctx.render_viewport([(0, 0, 1, 1, W, H)], out)
    ref = oracle_mod.render(disc, sol, (0, 0, 1, 1), W, H, idx)
    err = np.abs(out[idx] - ref).max()
    print(f"fmm32 deep leaf={leaf}: depth {ctx.sizes().depth} err {err:.2e}")
    assert err <= TOL_COLOUR


def test_fmm32_points_near_curves(dcmod, cuda_ok, mixed16, oracle_mod):
    d, disc, sol = mixed16
    ctx = make_ctx(dcmod, d, p=24, leaf_size=16)
    ctx.set_density(sol.sigma)
    rng = np.random.default_rng(12)
    k = rng.integers(0, disc.n_segments, 400)
    seg = disc.seg_xy[k]
    t = rng.uniform(0.05, 0.95, 400)[:, None]
    base = seg[:, :2] + t * (seg[:, 2:] - seg[:, :2])
    tan = seg[:, 2:] - seg[:, :2]
    nrm = np.stack([tan[:, 1], -tan[:, 0]], 1) / np.linalg.norm(tan, axis=1)[:, None]
    dist = 10 ** rng.uniform(-9, -2, 400) * rng.choice([-1, 1], 400)
    pts = base + dist[:, None] * nrm
    ref = oracle_mod.layer_potential(disc, pts, sol.sigma, sol.mu)
    out = np.zeros((400, 3))
    ctx.eval_points(pts, out)
    err = np.abs(out - ref).max()
    print(f"fmm32 near-curve points: max err {err:.2e}")
    assert err <= TOL_COLOUR


def test_fmm32_random_density_full_canvas(dcmod, cuda_ok, closed4, oracle_mod):
    """Render path alone with a seeded density of unit scale."""
    d, disc, sol, _ = closed4
    sig = random_node_values(disc.n_nodes, seed=21, scale=0.2)
    ctx = make_ctx(dcmod, d, p=24, leaf_size=32)
    ctx.set_density(sig)
    W, H = 160, 96
    out = np.zeros((W * H, 3))
    ctx.render_viewport([(0, 0, 1, 1, W, H)], out)
    ref = oracle_mod.render(disc, type(sol)(sig, sol.mu, sol.b), (0, 0, 1, 1), W, H)
    err = np.abs(out - ref).max()
    print(f"fmm32 random density: err {err:.2e}")
    assert err <= TOL_COLOUR
