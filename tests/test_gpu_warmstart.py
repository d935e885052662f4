"""Learned warm start through the C ABI: the panel features, the network's
forward pass, gradient and Adam step against the FP64 oracle (oracle/mlp.py),
and the DC_X0_LEARNED solve mode (per channel the start a x_pred + c 1 of
least residual, never worse than zeros or the paper's ones)."""
import numpy as np
import pytest

from dc_synth import drawing_by_name, random_node_values

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    from oracle import mlp
    return mlp


def dense_ctx(P, d, **kw):
    return P.Context(form="dense64", g=d.g, s_per_panel=d.s_per_panel, gmres_tol=1e-12,
                     gmres_restart=400, gmres_max_iter=4000, **kw)


def test_panel_features_match_oracle(dcmod, cuda_ok, M, oracle_mod):
    import torch
    d = drawing_by_name("mixed16")
    disc = oracle_mod.discretise(d)
    up, um = oracle_mod.boundary_values(d, disc)
    sig = random_node_values(disc.n_nodes, seed=21, scale=3.0)
    ctx = dense_ctx(dcmod, d)
    ctx.build_drawing(d)
    rows, nf, no = ctx.feature_dims()
    assert (rows, nf, no) == (3 * d.n_panels, M.n_features(d.g), d.g)
    feat = torch.full((rows, nf), float("nan"), dtype=torch.float32, device="cuda")
    with pytest.raises(dcmod.DcError):           # targets need a density
        ctx.panel_features(feat, torch.empty((rows, no), dtype=torch.float32, device="cuda"))
    ctx.set_density(sig)
    targ = torch.full((rows, no), float("nan"), dtype=torch.float32, device="cuda")
    ctx.panel_features(feat, targ)
    torch.cuda.synchronize()
    rf, rt = M.panel_features(disc, up, um, sig)
    gf, gt = feat.cpu().numpy().astype(np.float64), targ.cpu().numpy().astype(np.float64)
    assert np.abs(gf - rf).max() <= 1e-6 * max(1.0, np.abs(rf).max())
    assert np.abs(gt - rt).max() <= 1e-6 * max(1.0, np.abs(rt).max())


@pytest.mark.parametrize("batch", [1, 300])
def test_mlp_forward_and_gradient_match_oracle(dcmod, cuda_ok, M, batch):
    import torch
    n_in, H, n_out = M.n_features(8), 72, 8        # 72: one full 64-tile and a ragged one
    rng = np.random.default_rng(22 + batch)
    n = dcmod.mlp_param_count(n_in, H, n_out)
    assert n == M.param_count(n_in, H, n_out)
    p = (rng.standard_normal(n) * 0.1).astype(np.float32)
    x = rng.uniform(-1, 1, (batch, n_in)).astype(np.float32)
    t = rng.standard_normal((batch, n_out)).astype(np.float32)
    dev = lambda a: torch.from_numpy(a).cuda()
    work = torch.empty(dcmod.mlp_workspace_floats(n_in, H, n_out, batch), dtype=torch.float32,
                       device="cuda")
    y = torch.empty((batch, n_out), dtype=torch.float32, device="cuda")
    dcmod.mlp_forward(n_in, H, n_out, dev(p), dev(x), y, work)
    grad = torch.empty(n, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    dcmod.mlp_loss_grad(n_in, H, n_out, dev(p), dev(x), dev(t), grad, loss, work)
    torch.cuda.synchronize()
    ry, _ = M.forward(p.astype(np.float64), x, n_in, H, n_out)
    rl, rg = M.loss_grad(p.astype(np.float64), x, t, n_in, H, n_out)
    gy = y.cpu().numpy()
    assert np.abs(gy - ry).max() <= 1e-5 * max(1.0, np.abs(ry).max())
    assert abs(loss.item() - rl) <= 1e-5 * rl
    gg = grad.cpu().numpy()
    assert np.abs(gg - rg).max() <= 1e-4 * np.abs(rg).max()


def test_adam_matches_oracle(dcmod, cuda_ok, M):
    import torch
    rng = np.random.default_rng(23)
    n = 1000
    p = rng.standard_normal(n).astype(np.float32)
    dp = torch.from_numpy(p.copy()).cuda()
    m = torch.zeros(n, dtype=torch.float32, device="cuda")
    v = torch.zeros_like(m)
    rp, rm, rv = p.astype(np.float64), np.zeros(n), np.zeros(n)
    for step in range(1, 4):
        g = rng.standard_normal(n).astype(np.float32)
        dcmod.mlp_adam(dp, torch.from_numpy(g).cuda(), m, v, 1e-2, step)
        rp = M.adam_step(rp, g.astype(np.float64), rm, rv, 1e-2, 0.9, 0.999, 1e-8, step)
    torch.cuda.synchronize()
    assert np.abs(dp.cpu().numpy() - rp).max() <= 1e-6


def _initial_residuals(P, ctx, d):
    """||b - G_H x|| / ||b|| per channel for x = 0 and x = 1, through the ABI
    (b = (u+ + u-)/2 - F_H mu, Alg. 3)."""
    import torch
    _, _, up, um = ctx.nodes()
    mu = torch.from_numpy(up - um).cuda()
    fmu = torch.empty_like(mu)
    ctx.apply_operator(mu, fmu, op=1)
    b = torch.from_numpy(0.5 * (up + um)).cuda() - fmu
    g1 = torch.empty_like(b)
    ctx.apply_operator(torch.ones_like(b), g1, op=0)
    bn = torch.linalg.norm(b, dim=0)
    return (torch.linalg.norm(b - g1, dim=0) / bn).cpu().numpy()


def test_learned_mode_needs_a_model_and_falls_back(dcmod, cuda_ok, M):
    d = drawing_by_name("mixed16")
    n_in, H = M.n_features(d.g), 16
    n = dcmod.mlp_param_count(n_in, H, d.g)
    ref = dense_ctx(dcmod, d)
    ref.build_drawing(d)
    ref.solve_density()
    sig0 = ref.get_density()
    ctx = dense_ctx(dcmod, d, x0_mode=dcmod.DC_X0_LEARNED)
    ctx.build_drawing(d)
    with pytest.raises(dcmod.DcError) as e:
        ctx.solve_density()
    assert e.value.status == dcmod.DC_ERR_STATE
    with pytest.raises(dcmod.DcError):
        ctx.set_warm_start_model(H, np.full(n, np.nan, dtype=np.float32))
    # a network that predicts zero: nothing to use, the start is the best
    # multiple of the paper's x0 = 1
    ctx.set_warm_start_model(H, np.zeros(n, dtype=np.float32))
    st = ctx.solve_density()
    assert st.used_warm == 0 and st.converged == 1
    ones = _initial_residuals(dcmod, ctx, d)
    assert np.all(np.array(st.warm_resid) <= np.minimum(1.0, ones) * (1 + 1e-9))
    np.testing.assert_allclose(ctx.get_density(), sig0, rtol=0, atol=1e-8 * np.abs(sig0).max())
    # an untrained network (random weights): the start is never worse than
    # zeros or ones, and the solve reaches the same density
    rng = np.random.default_rng(24)
    ctx.set_warm_start_model(H, (rng.standard_normal(n) * 0.3).astype(np.float32))
    st = ctx.solve_density()
    assert st.converged == 1
    assert np.all(np.array(st.warm_resid) <= np.minimum(1.0, ones) * (1 + 1e-9))
    np.testing.assert_allclose(ctx.get_density(), sig0, rtol=0, atol=1e-8 * np.abs(sig0).max())


def test_trained_warm_start_cuts_the_initial_residual(dcmod, cuda_ok, M):
    import torch
    from paper_2311_14312_gb300 import warmstart
    feats, targs = [], []
    for i in range(12):               # training drawings: same recipe, other seeds
        d = drawing_by_name("mixed16", seed=100 + i)
        c = dense_ctx(dcmod, d)
        c.build_drawing(d)
        c.solve_density()
        f, t = warmstart.collect(c)
        feats.append(f)
        targs.append(t)
    feat, targ = torch.cat(feats), torch.cat(targs)
    params, hist = warmstart.train(feat, targ, hidden=64, steps=1500, batch=512, lr=2e-3,
                                   seed=5, log_every=500)
    assert hist[-1][1] < hist[0][1]
    d = drawing_by_name("mixed16")            # held out
    cold = dense_ctx(dcmod, d)                # x0 = ones, the paper's choice
    cold.build_drawing(d)
    sc = cold.solve_density()
    warm = dense_ctx(dcmod, d, x0_mode=dcmod.DC_X0_LEARNED)
    warm.build_drawing(d)
    warm.set_warm_start_model(64, params)
    sw = warm.solve_density()
    ones = _initial_residuals(dcmod, warm, d)
    print(f"train loss {hist[0][1]:.3e} -> {hist[-1][1]:.3e}; initial residual: x0 = 1 "
          f"{[round(float(r), 4) for r in ones]}, learned {[round(r, 4) for r in sw.warm_resid]}; "
          f"iterations cold {list(sc.iters)} warm {list(sw.iters)}; warm-start cost "
          f"{sw.ms_warm:.2f} ms")
    assert sw.converged == 1 and sc.converged == 1
    assert sw.used_warm == 7
    assert np.all(np.array(sw.warm_resid) < np.minimum(1.0, ones))
    ref = cold.get_density()
    np.testing.assert_allclose(warm.get_density(), ref, rtol=0, atol=1e-8 * np.abs(ref).max())


def test_learned_mode_in_the_chosen_form(dcmod, cuda_ok):
    """DC_X0_LEARNED in the FP32 form (refinement around the FP32 inner
    GMRES): a briefly trained network's start lowers the initial residual
    below the paper's x0 = 1, and the solve reaches the same density."""
    from paper_2311_14312_gb300 import warmstart
    import torch
    kw = dict(form="fmm32", p=24, leaf_size=32, gmres_tol=1e-10)
    feats, targs = [], []
    for i in range(8):
        d = drawing_by_name("mixed16", seed=200 + i)
        c = dcmod.Context(g=d.g, s_per_panel=d.s_per_panel, **kw)
        c.build_drawing(d)
        c.solve_density()
        f, t = warmstart.collect(c)
        feats.append(f)
        targs.append(t)
        c.close()
    params, hist = warmstart.train(torch.cat(feats), torch.cat(targs), hidden=64, steps=1000, batch=512,
                                   lr=2e-3, seed=6, log_every=500)
    d = drawing_by_name("mixed16")
    cold = dcmod.Context(g=d.g, s_per_panel=d.s_per_panel, **kw)
    cold.build_drawing(d)
    sc = cold.solve_density()
    warm = dcmod.Context(g=d.g, s_per_panel=d.s_per_panel, x0_mode=dcmod.DC_X0_LEARNED, **kw)
    warm.build_drawing(d)
    warm.set_warm_start_model(64, params)
    sw = warm.solve_density()
    ones = _initial_residuals(dcmod, warm, d)
    print(f"fmm32: initial residual x0 = 1 {[round(float(r), 4) for r in ones]}, learned "
          f"{[round(r, 4) for r in sw.warm_resid]}; iterations cold {list(sc.iters)} warm {list(sw.iters)}")
    assert sc.converged == 1 and sw.converged == 1
    assert np.all(np.array(sw.warm_resid) < np.minimum(1.0, ones))
    ref = cold.get_density()
    assert np.abs(warm.get_density() - ref).max() <= 1e-8 * np.abs(ref).max()
