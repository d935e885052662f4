"""Mixed Dirichlet / Neumann conditions (Sec. 4.3) through the C ABI
(dc_solve_mixed) against the oracle's dense LU of the same block system
(oracle/mixed.py), on a disc with a hole bounded by eight cubic quarter
arcs (128 panels, g = 16, s = 80: 2048 nodes, 10,240 segments), Dirichlet
data on half of the outer loop, Neumann data elsewhere:

  * psi on the Dirichlet panels (the library's sigma) within 1e-8 (dense
    form) or 2e-7 (FMM forms) of the oracle's, relative to max |psi|: the
    block matrix has condition number 1.5e4 (numpy's 2-norm estimate on the
    oracle's matrix), which amplifies the GMRES residual (1e-13) and the
    FMM's relative operator error at p = 24 (below 1e-11);
  * the colour at 2000 interior, exterior and near-boundary points by the
    FP64 direct sum (dc_eval_points_noalloc) within 1e-9 of the oracle's
    direct sum of its own (sigma, mu), which checks mu = -u on the Neumann
    panels too; the form's own dc_eval_points within 1e-10 (FP64 forms) or
    2e-6 (FP32 form) relative to max |u|;
  * the next dc_solve_density restores mu from the colours;
  * a clockwise outer loop is DC_ERR_GEOMETRY, all-Neumann DC_ERR_ARG.
"""
import numpy as np
import pytest
import torch

from dc_synth import circle_loops, harmonic

pytestmark = pytest.mark.gpu

HOLE = (0.45, 0.52)
LOOPS = [(0.5, 0.5, 0.35, True), (HOLE[0], HOLE[1], 0.12, False)]
PPA, G, S = 16, 16, 80
OPTS = dict(p=24, leaf_size=32, gmres_tol=1e-13, gmres_restart=400, gmres_max_iter=4000)


@pytest.fixture(scope="module")
def ref(oracle_mod):
    from oracle import mixed as M
    O = oracle_mod
    d = circle_loops(LOOPS, panels_per_arc=PPA, g=G, s_per_panel=S)
    disc = O.discretise(d)
    u, psi = harmonic.boundary_data(d, disc.node_xy, disc.node_curve, disc.node_t, HOLE)
    neu = np.repeat(np.arange(d.n_curves), PPA) >= 2
    sig, mu, _ = M.solve_mixed(d, disc, neu, psi, u)
    rng = np.random.default_rng(5)
    Q = rng.uniform(0.1, 0.9, (1600, 2))
    # 400 points within 1e-3 of the nodes, both sides
    k = rng.choice(disc.n_nodes, 400, replace=False)
    Q = np.vstack([Q, disc.node_xy[k] + rng.uniform(-1e-3, 1e-3, (400, 2))])
    uq = O.layer_potential(disc, Q, sig, mu)
    sol = O.solve(d, disc)
    return dict(d=d, disc=disc, u=u, psi=psi, neu=neu, sig=sig, mu=mu, Q=Q, uq=uq, sol=sol)


def _ctx(P, d, form):
    ctx = P.Context(form=form, g=d.g, s_per_panel=d.s_per_panel, **OPTS)
    ctx.build_drawing(d)
    return ctx


@pytest.mark.parametrize("form", ["dense64", "fmm64", "fmm32"])
def test_mixed_matches_oracle(dcmod, cuda_ok, ref, form):
    r = ref
    ctx = _ctx(dcmod, r["d"], form)
    st = ctx.solve_mixed(r["neu"], r["psi"], r["u"])
    assert st.converged == 1
    sig = ctx.get_density()
    e_sig = np.abs(sig - r["sig"]).max() / np.abs(r["sig"]).max()
    xy = torch.from_numpy(r["Q"]).cuda()
    out = torch.zeros((len(r["Q"]), 3), dtype=torch.float64, device="cuda")
    ctx.eval_points_noalloc(xy, out)
    e_u = np.abs(out.cpu().numpy() - r["uq"]).max()
    own = np.zeros((len(r["Q"]), 3))
    ctx.eval_points(r["Q"], own)
    e_own = np.abs(own - r["uq"]).max() / np.abs(r["uq"]).max()
    print(f"{form}: iterations {list(st.iters)}, true residual {max(st.true_rel_resid):.1e}, "
          f"{st.ms_solve:.1f} ms; psi vs oracle {e_sig:.2e}, FP64 colour vs oracle {e_u:.2e}, "
          f"the form's own evaluation {e_own:.2e} (relative)")
    assert e_sig <= (1e-8 if form == "dense64" else 2e-7)
    assert e_u <= 1e-9
    assert e_own <= (2e-6 if form == "fmm32" else 1e-10)
    # the two-sided solve afterwards takes mu from the colours again
    st2 = ctx.solve_density()
    assert st2.converged == 1
    sig2 = ctx.get_density()
    ref2 = r["sol"].sigma
    assert np.abs(sig2 - ref2).max() / np.abs(ref2).max() <= 1e-9
    ctx.close()


def test_mixed_default_dirichlet_data(dcmod, cuda_ok, ref, oracle_mod):
    from oracle import mixed as M
    r = ref
    want, _, _ = M.solve_mixed(r["d"], r["disc"], r["neu"], r["psi"])
    ctx = _ctx(dcmod, r["d"], "dense64")
    ctx.solve_mixed(r["neu"], r["psi"])
    sig = ctx.get_density()
    assert np.abs(sig - want).max() / np.abs(want).max() <= 1e-8
    ctx.close()


def test_mixed_errors(dcmod, cuda_ok, ref):
    r = ref
    ctx = _ctx(dcmod, r["d"], "fmm32")
    with pytest.raises(dcmod.DcError) as e:
        ctx.solve_mixed(np.ones(r["d"].n_panels, bool), r["psi"], r["u"])
    assert e.value.status == dcmod.DC_ERR_ARG
    bad = r["psi"].copy()
    bad[3, 1] = np.nan
    with pytest.raises(dcmod.DcError) as e:
        ctx.solve_mixed(r["neu"], bad, r["u"])
    assert e.value.status == dcmod.DC_ERR_ARG
    ctx.close()
    cw = circle_loops([(0.5, 0.5, 0.35, False)], panels_per_arc=2, g=8, s_per_panel=40)
    ctx = _ctx(dcmod, cw, "dense64")
    n = ctx.sizes().n_nodes
    with pytest.raises(dcmod.DcError) as e:
        ctx.solve_mixed(np.zeros(cw.n_panels, bool), np.zeros((n, 3)), np.ones((n, 3)))
    assert e.value.status == dcmod.DC_ERR_GEOMETRY
    ctx.close()
