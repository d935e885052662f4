"""The viewport update (Sec. 6.2, 6.4; Alg. 9) through dc_view_update
against the oracle (oracle/viewport.py) on mixed16 (16 curves, 151 panels of
g = 8, s = 40) and the viewport [0.2, 0.7]^2 at 256 x 256:

  * without subdivision (eps_coef = 0), from the oracle's density: the e of
    the rule at len_unit 1/4096 identical, the labels identical, and the
    render on the evaluation polyline within 1e-10 (FP64 forms) or 1e-5
    (FP32 form) of the oracle's direct sum on that polyline;
  * with subdivision (about three panels in the viewport above epsilon_2,
    epsilon_1 = two pixels) and the local re-solve: the same panels split
    (refined starts identical), the density within 1e-8 of the oracle's
    local LU (relative), the render within 1e-7 (FP64 forms) or 1e-5;
  * a new density drops the view: the render equals the plain one.
"""
import numpy as np
import pytest
import torch

from dc_synth import drawing_by_name

pytestmark = pytest.mark.gpu

VP = (0.2, 0.2, 0.7, 0.7)
W = H = 256
UNIT = 1.0 / 4096
OPTS = dict(p=24, leaf_size=32, gmres_tol=1e-12, gmres_restart=400, gmres_max_iter=4000)


@pytest.fixture(scope="module")
def ref(oracle_mod):
    from oracle import adaptive as A
    from oracle import viewport as V
    O = oracle_mod
    d = drawing_by_name("mixed16")
    disc = O.discretise(d)
    sol = O.solve(d, disc)
    m = V.meets_viewport(disc, VP)
    ts = np.sort(A.top_coefficient(disc, sol.sigma)[m])
    eps = float(0.5 * (ts[-4] + ts[-3]))    # between values: no test value near the threshold
    pix = np.sort(np.random.default_rng(17).choice(W * H, 3000, replace=False))
    plain = V.view_update(d, sol.sigma, VP, W, H, 0.0, 0.0, unit=UNIT)
    u_plain = V.render(plain["disc_e"], plain["sigma"], sol.mu, VP, W, H, pix)
    sub = V.view_update(d, sol.sigma, VP, W, H, eps, 2.0, unit=UNIT, max_rounds=1)
    up, um = O.boundary_values(sub["drawing"], sub["disc"])
    u_sub = V.render(sub["disc_e"], sub["sigma"], up - um, VP, W, H, pix)
    return dict(d=d, sol=sol, eps=eps, pix=pix, plain=plain, u_plain=u_plain, sub=sub, u_sub=u_sub)


def _ctx(P, d, form):
    ctx = P.Context(form=form, g=d.g, s_per_panel=d.s_per_panel, **OPTS)
    ctx.build_drawing(d)
    return ctx


def _render(ctx, pix):
    rgb = torch.empty((W * H, 3), dtype=torch.float64, device="cuda")
    ctx.render_viewport([(*VP, W, H)], rgb)
    torch.cuda.synchronize()
    return rgb.cpu().numpy()[pix]


def _labels(lab):
    return [int((lab == k).sum()) for k in (0, 1, 2)]


@pytest.mark.parametrize("form", ["dense64", "fmm64", "fmm32"])
def test_view_without_subdivision(dcmod, cuda_ok, ref, form):
    r = ref
    ctx = _ctx(dcmod, r["d"], form)
    ctx.set_density(r["sol"].sigma)
    base = _render(ctx, r["pix"])
    st = ctx.view_update((*VP, W, H), eps_coef=0.0, len_unit=UNIT)
    assert st.rounds == 0 and st.e == r["plain"]["e"] > r["d"].s_per_panel
    assert [st.n_fixed, st.n_interpolating, st.n_resolving] == _labels(r["plain"]["labels"])
    got = _render(ctx, r["pix"])
    err = np.abs(got - r["u_plain"]).max()
    moved = np.abs(base - r["u_plain"]).max()
    print(f"{form}: e = {st.e}, labels {st.n_fixed}/{st.n_interpolating}/{st.n_resolving}, build {st.ms_build:.1f} ms;"
          f" render vs oracle {err:.2e} (the solve polyline's render differs by {moved:.2e})")
    assert err <= (1e-5 if form == "fmm32" else 1e-10)
    # a new density drops the view
    ctx.set_density(r["sol"].sigma)
    assert np.array_equal(_render(ctx, r["pix"]), base)
    ctx.close()


@pytest.mark.parametrize("form", ["dense64", "fmm64", "fmm32"])
def test_view_with_subdivision(dcmod, cuda_ok, ref, form):
    r = ref
    s = r["sub"]
    ctx = _ctx(dcmod, r["d"], form)
    ctx.set_density(r["sol"].sigma)
    st = ctx.view_update((*VP, W, H), eps_coef=r["eps"], eps_len_px=2.0, len_unit=UNIT, max_rounds=1)
    assert st.rounds == 1 and st.n_split == s["n_split"] and st.e == s["e"]
    ptr, start = ctx.panels()
    assert np.array_equal(ptr, s["drawing"].panel_ptr) and np.array_equal(start, s["drawing"].panel_start)
    sig = ctx.get_density()
    e_sig = np.abs(sig - s["sigma"]).max() / np.abs(s["sigma"]).max()
    got = _render(ctx, r["pix"])
    err = np.abs(got - r["u_sub"]).max()
    print(f"{form}: {st.n_split} split, labels {st.n_fixed}/{st.n_interpolating}/{st.n_resolving} "
          f"(oracle {_labels(s['labels'])}), e = {st.e}; sigma vs oracle {e_sig:.2e}, render {err:.2e}; "
          f"ms subdivide {st.ms_subdivide:.1f} build {st.ms_build:.1f}")
    assert [st.n_fixed, st.n_interpolating, st.n_resolving] == _labels(s["labels"])
    assert e_sig <= 1e-8
    assert err <= (1e-5 if form == "fmm32" else 1e-7)
    ctx.close()


def test_view_errors(dcmod, cuda_ok, ref):
    ctx = _ctx(dcmod, ref["d"], "fmm32")
    with pytest.raises(dcmod.DcError) as e:
        ctx.view_update((*VP, W, H))
    assert e.value.status == dcmod.DC_ERR_STATE
    ctx.set_density(ref["sol"].sigma)
    with pytest.raises(dcmod.DcError) as e:
        ctx.view_update((0.5, 0.5, 0.4, 0.6, W, H))
    assert e.value.status == dcmod.DC_ERR_ARG
    with pytest.raises(dcmod.DcError) as e:
        ctx.view_update((*VP, W, H), len_unit=1e-9)
    assert e.value.status == dcmod.DC_ERR_ARG
    ctx.close()
