"""Quadtree anti-aliasing (Sec. 7) through the C ABI (options.aa_levels)
against the oracle (oracle/antialias.py), with the density set from the
oracle's LU solve so that only the render is compared:

  * mixed16 (16 curves, 6040 segments) at 256 x 256 with m = 2 in all three
    forms: the refined pixels are exactly the oracle's (count and sample
    count identical: integer decisions taken by the same IEEE operations),
    and every refined pixel's colour matches the oracle's weighted sum
    within 1e-10 (FP64 forms) or 1e-5 (FP32 form, the render's bar); pixels
    that are not refined keep the plain render's values bit for bit;
  * mixed200 (139,440 segments) at 2048 x 2048 with m = 2 in the FP32 form:
    refined-pixel count identical, 1500 sampled refined pixels within 1e-5
    and their 8-bit values identical outside the rounding band;
  * two calls give identical bytes; aa_levels outside [0, 6] is refused.
"""
import numpy as np
import pytest
import torch

from dc_synth import drawing_by_name

pytestmark = pytest.mark.gpu

VP = (0.0, 0.0, 1.0, 1.0)


def _render(ctx, w, h):
    rgb = torch.empty((w * h, 3), dtype=torch.float64, device="cuda")
    rgb8 = torch.empty((w * h, 3), dtype=torch.uint8, device="cuda")
    st = ctx.render_viewport([(*VP, w, h)], rgb, rgb8, stats=True)
    torch.cuda.synchronize()
    return rgb.cpu().numpy(), rgb8.cpu().numpy(), st


@pytest.fixture(scope="module")
def small(oracle_mod):
    from oracle import antialias as A
    O = oracle_mod
    d = drawing_by_name("mixed16")
    disc = O.discretise(d)
    sol = O.solve(d, disc)
    edge, ties = A.edge_pixels(disc, VP, 256, 256)
    u, e, t, ns = A.render_aa(disc, sol.sigma, sol.mu, VP, 256, 256, edge, 2)
    assert e.all()
    return dict(d=d, disc=disc, sol=sol, edge=edge, ties=ties, u=u, tie=t, ns=ns)


def _ctx(P, d, form, levels, **kw):
    kw.setdefault("leaf_size", 32)
    ctx = P.Context(form=form, g=d.g, s_per_panel=d.s_per_panel, p=24, aa_levels=levels, **kw)
    ctx.build_drawing(d)
    return ctx


@pytest.mark.parametrize("form", ["dense64", "fmm64", "fmm32"])
def test_antialias_matches_oracle_small(dcmod, cuda_ok, small, form):
    r = small
    assert len(r["ties"]) == 0
    ctx = _ctx(dcmod, r["d"], form, 2)
    ctx.set_density(r["sol"].sigma)
    rgb, rgb8, st = _render(ctx, 256, 256)
    plain = _ctx(dcmod, r["d"], form, 0)
    plain.set_density(r["sol"].sigma)
    prgb, prgb8, pst = _render(plain, 256, 256)
    assert pst.aa_pixels == 0
    assert st.aa_pixels == len(r["edge"]) and st.aa_samples == int(r["ns"].sum())
    err = np.abs(rgb[r["edge"]] - r["u"]).max()
    keep = np.setdiff1d(np.arange(256 * 256), r["edge"])
    print(f"{form}: {st.aa_pixels} refined pixels, {st.aa_samples} samples, {st.ms_aa:.2f} ms of "
          f"{st.ms:.2f} ms; refined colours vs oracle {err:.2e}")
    assert err <= (1e-5 if form == "fmm32" else 1e-10)
    assert np.array_equal(rgb[keep], prgb[keep]) and np.array_equal(rgb8[keep], prgb8[keep])
    again, again8, _ = _render(ctx, 256, 256)
    assert np.array_equal(again, rgb) and np.array_equal(again8, rgb8)
    ctx.close()
    plain.close()


def test_antialias_mixed200_2048(dcmod, cuda_ok, oracle_mod):
    from oracle import antialias as A
    O = oracle_mod
    d = drawing_by_name("mixed200")
    disc = O.discretise(d)
    sig = np.random.default_rng(91).standard_normal((disc.n_nodes, 3)) * 0.05
    up, um = O.boundary_values(d, disc)
    edge, ties = A.edge_pixels(disc, VP, 2048, 2048)
    pick = np.sort(np.random.default_rng(92).choice(edge, 1500, replace=False))
    u, e, t, ns = A.render_aa(disc, sig, up - um, VP, 2048, 2048, pick, 2)
    ctx = _ctx(dcmod, d, "fmm32", 2, leaf_size=64)
    ctx.set_density(sig)
    rgb, rgb8, st = _render(ctx, 2048, 2048)
    print(f"mixed200 2048^2: {st.aa_pixels} refined pixels ({len(edge)} in the oracle, {len(ties)} ties), "
          f"{st.aa_samples} samples; anti-aliasing {st.ms_aa:.2f} ms of {st.ms:.2f} ms")
    assert abs(st.aa_pixels - len(edge)) <= len(ties)
    ok = ~t
    err = np.abs(rgb[pick][ok] - u[ok]).max()
    q = 255.0 * np.clip(u[ok], 0.0, 1.0)
    band = np.abs(q - np.floor(q) - 0.5) <= 255.0 * 1e-5
    mism = int(((rgb8[pick][ok] != np.floor(q + 0.5)) & ~band).sum())
    print(f"sampled refined colours vs oracle {err:.2e}; 8-bit mismatches outside the band {mism}")
    assert err <= 1e-5 and mism == 0
    ctx.close()


def test_aa_levels_range(dcmod, cuda_ok):
    with pytest.raises(dcmod.DcError) as e:
        dcmod.Context(form="fmm32", aa_levels=7)
    assert e.value.status == dcmod.DC_ERR_ARG
