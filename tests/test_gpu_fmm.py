"""FMM forms on the GPU (App. E, Alg. 8) against the FP64 oracle: densities,
pixels, points near curves, deep trees that exercise lists 3 and 4, and the
root-domain contract."""
import numpy as np
import pytest

from dc_synth import drawing_by_name, pixel_sample, random_node_values

pytestmark = pytest.mark.gpu


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
    return d, disc


def make_ctx(P, d, form, **kw):
    kw.setdefault("gmres_tol", 1e-12)
    kw.setdefault("gmres_restart", 400)
    ctx = P.Context(form=form, g=d.g, s_per_panel=d.s_per_panel, **kw)
    ctx.build_drawing(d)
    return ctx


# measured on GB300: p=12 1.5e-6 / 5.8e-7, p=20 1.2e-9 / 8.2e-10,
# p=30 2.9e-11 / 1.4e-12 (sigma relative / pixel absolute); the bars keep a
# margin of about 10x and follow the geometric decay of App. E.1
@pytest.mark.parametrize("p,leaf,tol_sigma,tol_px", [(12, 32, 2e-5, 6e-6), (20, 32, 2e-8, 1e-8),
                                                     (30, 16, 3e-10, 1e-10)])
def test_fmm64_solve_and_render(dcmod, cuda_ok, closed4, p, leaf, tol_sigma, tol_px):
    d, disc, sol, u_ref = closed4
    ctx = make_ctx(dcmod, d, "fmm64", p=p, leaf_size=leaf)
    st = ctx.solve_density()
    assert st.converged == 1
    sig = ctx.get_density()
    es = np.abs(sig - sol.sigma).max() / np.abs(sol.sigma).max()
    out = np.zeros((128 * 128, 3))
    ctx.render_viewport([(0, 0, 1, 1, 128, 128)], out)
    ep = np.abs(out - u_ref).max()
    sz = ctx.sizes()
    print(f"fmm64 p={p} leaf={leaf}: sigma rel {es:.2e}  pixel abs {ep:.2e}  iters {list(st.iters)} "
          f"cells {sz.n_cells} depth {sz.depth} pieces {sz.n_pieces}")
    assert es <= tol_sigma
    assert ep <= tol_px


@pytest.mark.parametrize("leaf", [4, 16, 64])
def test_fmm64_render_deep_trees(dcmod, cuda_ok, mixed16, oracle_mod, leaf):
    """A seeded density rendered through the FMM with small leaves (deep,
    strongly non-uniform trees: lists 3 and 4 are populated)."""
    d, disc = mixed16
    sig = random_node_values(disc.n_nodes, seed=7)
    up, um = oracle_mod.boundary_values(d, disc)
    ctx = make_ctx(dcmod, d, "fmm64", p=30, leaf_size=leaf)
    ctx.set_density(sig)
    W = H = 256
    idx = pixel_sample(W, H, 3000, seed=2)
    out = np.zeros((W * H, 3))
    ctx.render_viewport([(0, 0, 1, 1, W, H)], out)
    ref = oracle_mod.layer_potential(disc, oracle_mod.pixel_centres((0, 0, 1, 1), W, H, idx),
                                     sig, up - um)
    err = np.abs(out[idx] - ref).max()
    print(f"deep tree leaf={leaf}: depth {ctx.sizes().depth}, max abs err {err:.2e}")
    assert err <= 1e-11 * max(1.0, np.abs(ref).max())


def test_fmm64_points_near_curves(dcmod, cuda_ok, mixed16, oracle_mod):
    d, disc = mixed16
    sol = oracle_mod.solve(d, disc)
    ctx = make_ctx(dcmod, d, "fmm64", p=30, leaf_size=16)
    ctx.set_density(sol.sigma)
    rng = np.random.default_rng(4)
    k = rng.integers(0, disc.n_segments, 300)
    seg = disc.seg_xy[k]
    mid = 0.5 * (seg[:, :2] + seg[:, 2:])
    tan = seg[:, 2:] - seg[:, :2]
    nrm = np.stack([tan[:, 1], -tan[:, 0]], 1) / np.linalg.norm(tan, axis=1)[:, None]
    dist = 10 ** rng.uniform(-7, -2, 300) * rng.choice([-1, 1], 300)
    pts = mid + dist[:, None] * nrm
    ref = oracle_mod.layer_potential(disc, pts, sol.sigma, sol.mu)
    out = np.zeros((300, 3))
    ctx.eval_points(pts, out)
    assert np.abs(out - ref).max() <= 1e-8


def test_fmm64_solve_mixed(dcmod, cuda_ok, mixed16, oracle_mod):
    d, disc = mixed16
    sol = oracle_mod.solve(d, disc)
    ctx = make_ctx(dcmod, d, "fmm64", p=30, leaf_size=16)
    st = ctx.solve_density()
    assert st.converged == 1
    sig = ctx.get_density()
    assert np.abs(sig - sol.sigma).max() <= 1e-7 * np.abs(sol.sigma).max()


def test_fmm_domain_contract(dcmod, cuda_ok, closed4, oracle_mod):
    P = dcmod
    d, disc, sol, _ = closed4
    ctx = make_ctx(P, d, "fmm64", p=24)
    ctx.set_density(sol.sigma)
    with pytest.raises(P.DcError) as e:
        ctx.render_viewport([(-2.0, -2.0, 3.0, 3.0, 16, 16)], np.zeros((256, 3)))
    assert e.value.status == P.DC_ERR_ARG
    wide = make_ctx(P, d, "fmm64", p=30, domain=(-2.0, -2.0, 3.0, 3.0))
    wide.set_density(sol.sigma)
    out = np.zeros((32 * 32, 3))
    wide.render_viewport([(-2.0, -2.0, 3.0, 3.0, 32, 32)], out)
    ref = oracle_mod.render(disc, sol, (-2.0, -2.0, 3.0, 3.0), 32, 32)
    assert np.abs(out - ref).max() <= 1e-8
