"""Plain dense FP64 form on the GPU against the FP64 oracle (the brute-force
hybrid method, Table 1): nodes, densities (Eq. 27), pixels (Alg. 4) and
8-bit output.  Bar: 1e-10 relative for densities, 1e-10 absolute for
colours in [0, 1]."""
import numpy as np
import pytest

from dc_synth import drawing_by_name, pixel_sample, random_node_values

pytestmark = pytest.mark.gpu

TOL_PLAIN = 1e-10


def band_mask(u_ref, tol):
    """Pixels whose reference colour lies within tol of an 8-bit rounding
    boundary, where two correct results may quantise differently."""
    v = 255.0 * np.clip(u_ref, 0, 1)
    frac = np.abs(v - np.floor(v) - 0.5)
    return frac <= 255.0 * tol + 1e-12


@pytest.fixture(scope="module")
def closed4(oracle_mod):
    d = drawing_by_name("closed4")
    disc = oracle_mod.discretise(d)
    sol = oracle_mod.solve(d, disc)
    u = oracle_mod.render(disc, sol, (0, 0, 1, 1), 128, 128)
    return d, disc, sol, u


def make_ctx(P, d, form="dense64", **kw):
    kw.setdefault("gmres_tol", 1e-12)
    kw.setdefault("gmres_restart", 400)
    ctx = P.Context(form=form, g=d.g, s_per_panel=d.s_per_panel, **kw)
    ctx.build_drawing(d)
    return ctx


def test_nodes_match_oracle(dcmod, cuda_ok, closed4):
    d, disc, _, _ = closed4
    ctx = make_ctx(dcmod, d)
    xy, t, up, um = ctx.nodes()
    np.testing.assert_allclose(xy, disc.node_xy, atol=1e-13)
    np.testing.assert_allclose(t, disc.node_t, atol=1e-13)
    ou, om = __import__("oracle.oracle", fromlist=["x"]).boundary_values(d, disc)
    np.testing.assert_allclose(up, ou, atol=1e-13)
    np.testing.assert_allclose(um, om, atol=1e-13)
    s = ctx.sizes()
    assert (s.n_nodes, s.n_segments, s.n_panels) == (1024, 5120, 64)


def test_dense_solve_matches_oracle(dcmod, cuda_ok, closed4):
    d, disc, sol, _ = closed4
    ctx = make_ctx(dcmod, d)
    st = ctx.solve_density()
    assert st.converged == 1
    assert max(st.rel_resid) <= 1e-12
    sig = ctx.get_density()
    err = np.abs(sig - sol.sigma).max() / np.abs(sol.sigma).max()
    assert err <= TOL_PLAIN, err


def test_dense_render_matches_oracle(dcmod, cuda_ok, closed4):
    import torch
    d, disc, sol, u_ref = closed4
    ctx = make_ctx(dcmod, d)
    ctx.solve_density()
    rgb = torch.empty((128 * 128, 3), dtype=torch.float64, device="cuda")
    rgb8 = torch.empty((128 * 128, 3), dtype=torch.uint8, device="cuda")
    ctx.render_viewport([(0, 0, 1, 1, 128, 128)], rgb, rgb8)
    torch.cuda.synchronize()
    u = rgb.cpu().numpy()
    assert np.abs(u - u_ref).max() <= TOL_PLAIN
    q_ref = np.floor(255 * np.clip(u_ref, 0, 1) + 0.5).astype(np.uint8)
    ok = ~band_mask(u_ref, TOL_PLAIN)
    np.testing.assert_array_equal(rgb8.cpu().numpy()[ok], q_ref[ok])
    # host outputs equal device outputs (same kernels, copied back)
    h = np.zeros((128 * 128, 3))
    h8 = np.zeros((128 * 128, 3), np.uint8)
    ctx.render_viewport([(0, 0, 1, 1, 128, 128)], h, h8)
    np.testing.assert_array_equal(h, u)
    np.testing.assert_array_equal(h8, rgb8.cpu().numpy())


def test_dense_eval_points_near_curves(dcmod, cuda_ok, closed4, oracle_mod):
    d, disc, sol, _ = closed4
    ctx = make_ctx(dcmod, d)
    ctx.solve_density()
    rng = np.random.default_rng(11)
    # points at distance 1e-3 .. 1e-7 from random segment midpoints, both sides
    k = rng.integers(0, disc.n_segments, 200)
    seg = disc.seg_xy[k]
    mid = 0.5 * (seg[:, :2] + seg[:, 2:])
    tan = seg[:, 2:] - seg[:, :2]
    nrm = np.stack([tan[:, 1], -tan[:, 0]], 1) / np.linalg.norm(tan, axis=1)[:, None]
    dist = 10 ** rng.uniform(-7, -3, 200) * rng.choice([-1, 1], 200)
    pts = np.concatenate([mid + dist[:, None] * nrm, rng.uniform(0, 1, (200, 2))])
    ref = oracle_mod.layer_potential(disc, pts, sol.sigma, sol.mu)
    out = np.zeros((pts.shape[0], 3))
    ctx.eval_points(pts, out)
    assert np.abs(out - ref).max() <= 1e-9


def test_dense_mixed_open_closed(dcmod, cuda_ok, oracle_mod):
    d = drawing_by_name("mixed16")
    disc = oracle_mod.discretise(d)
    sol = oracle_mod.solve(d, disc)
    ctx = make_ctx(dcmod, d)
    st = ctx.solve_density()
    assert st.converged == 1
    sig = ctx.get_density()
    assert np.abs(sig - sol.sigma).max() <= TOL_PLAIN * np.abs(sol.sigma).max()
    W = H = 256
    idx = pixel_sample(W, H, 4000, seed=5)
    ref = oracle_mod.render(disc, sol, (0, 0, 1, 1), W, H, idx)
    out = np.zeros((W * H, 3))
    ctx.render_viewport([(0, 0, 1, 1, W, H)], out)
    assert np.abs(out[idx] - ref).max() <= TOL_PLAIN


def test_set_density_then_render(dcmod, cuda_ok, closed4, oracle_mod):
    """Render path alone: a seeded density set through the ABI, two uneven
    viewports in one call (one zoomed onto a curve)."""
    d, disc, sol, _ = closed4
    ctx = make_ctx(dcmod, d)
    sig = random_node_values(disc.n_nodes, seed=3)
    ctx.set_density(sig)
    # zoom window near (not centred on) a polyline vertex: no pixel centre
    # falls on the curve, where the double layer jumps
    c = disc.seg_xy[100, :2] + np.array([1.17e-4, -0.73e-4])
    vps = [(0.0, 0.0, 1.0, 1.0, 40, 24), (c[0] - 1e-3, c[1] - 1e-3, c[0] + 1e-3, c[1] + 1e-3, 33, 17)]
    n = sum(v[4] * v[5] for v in vps)
    out = np.zeros((n, 3))
    ctx.render_viewport(vps, out)
    ref = np.concatenate([oracle_mod.render(disc, type(sol)(sig, sol.mu, sol.b), v[:4], v[4], v[5])
                          for v in vps])
    assert np.abs(out - ref).max() <= 1e-9 * max(1.0, np.abs(ref).max())


def test_solve_is_deterministic(dcmod, cuda_ok, closed4):
    d = closed4[0]
    a = make_ctx(dcmod, d)
    a.solve_density()
    b = make_ctx(dcmod, d)
    b.solve_density()
    np.testing.assert_array_equal(a.get_density(), b.get_density())


def test_errors_are_reported_not_raised_on_device(dcmod, cuda_ok, closed4):
    P = dcmod
    d = closed4[0]
    ctx = P.Context(form="dense64", g=d.g, s_per_panel=d.s_per_panel)
    with pytest.raises(P.DcError) as e:
        ctx.solve_density()
    assert e.value.status == P.DC_ERR_STATE
    with pytest.raises(P.DcError) as e:
        ctx.build_tree(d.ctrl, d.panel_ptr, d.panel_start[::-1], d.colours)
    assert e.value.status == P.DC_ERR_ARG
    bad = d.ctrl.copy()
    bad[0, 0, 0] = np.nan
    with pytest.raises(P.DcError) as e:
        ctx.build_tree(bad, d.panel_ptr, d.panel_start, d.colours)
    assert e.value.status == P.DC_ERR_ARG
    ctx.build_drawing(d)
    with pytest.raises(P.DcError) as e:
        ctx.render_viewport([(0, 0, 1, 1, 4, 4)], np.zeros((16, 3)))
    assert e.value.status == P.DC_ERR_STATE
    ctx2 = make_ctx(P, d, gmres_max_iter=2)
    with pytest.raises(P.DcError) as e:
        ctx2.solve_density()
    assert e.value.status == P.DC_ERR_NOCONV
    s = ctx2.solve_density(allow_noconv=True)
    assert s.converged == 0 and max(s.iters) == 2
    with pytest.raises(P.DcError) as e:
        ctx2.render_viewport([(0, 0, 1, 1, -3, 4)], np.zeros((16, 3)))
    assert e.value.status == P.DC_ERR_ARG
