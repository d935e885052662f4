"""Adaptive subdivision with local re-solve (Sec. 6.1, 6.3; Alg. 5-7) through
the C ABI against the oracle (oracle/adaptive.py) on mixed16 (16 open and
closed curves, 151 panels of g = 8):

  * Alg. 5's test value per panel (highest Legendre coefficient of sigma)
    within 1e-8 of the largest, the same panels split, the refined panel
    starts bit-identical (dyadic arc-length fractions);
  * the re-solving labels of Eq. 40-41 identical, except panels whose
    oracle score lies within 1e-6 of the 0.9 threshold (none are expected);
  * the density after the local re-solve within 1e-8 of the oracle's LU
    solution of the same local system (relative to max |sigma|), and after
    a global re-solve within 1e-8 of the oracle's solve of the refined
    drawing.
"""
import numpy as np
import pytest

from dc_synth import drawing_by_name

pytestmark = pytest.mark.gpu

OPTS = dict(p=24, leaf_size=32, gmres_tol=1e-12, gmres_restart=400, gmres_max_iter=4000)
N_SPLIT = 12


@pytest.fixture(scope="module")
def ref16(oracle_mod):
    from oracle import adaptive as A
    O = oracle_mod
    d = drawing_by_name("mixed16")
    disc = O.discretise(d)
    sol = O.solve(d, disc)
    top = A.top_coefficient(disc, sol.sigma)
    ts = np.sort(top)
    eps = 0.5 * (ts[-N_SPLIT - 1] + ts[-N_SPLIT])
    d2, split, pmap = A.subdivide(d, disc, sol.sigma, eps, 0.0)
    disc2 = O.discretise(d2)
    AG, AF = O.hybrid_rows(disc2)
    s0 = A.warm_start(disc, sol.sigma, pmap)
    res = A.label_panels(disc2, AG, pmap)
    # each panel's largest ratio of ranges (Eq. 41's left side over the
    # right side without the 0.9), to spot borderline labels
    g, P = disc2.g, disc2.n_panels
    score = np.zeros(P)
    for a in [q for q in range(P) if pmap[q][1] != 0]:
        V = AG[:, a * g:(a + 1) * g].sum(axis=1).reshape(P, g)
        rng = V.max(axis=1) - V.min(axis=1)
        score = np.maximum(score, rng / rng[a])
    loc = A.local_resolve(d2, disc2, s0, res, AG, AF)
    glob = O.solve(d2, disc2).sigma
    return dict(d=d, eps=eps, top=top, split=split, d2=d2, res=res, score=score, loc=loc, glob=glob,
                n_old=disc.n_panels)


def _ctx(P, d, form):
    ctx = P.Context(form=form, g=d.g, s_per_panel=d.s_per_panel, **OPTS)
    ctx.build_drawing(d)
    st = ctx.solve_density()
    assert st.converged == 1
    return ctx


@pytest.mark.parametrize("form", ["dense64", "fmm64", "fmm32"])
def test_subdivide_and_local_resolve_match_oracle(dcmod, cuda_ok, ref16, form):
    r = ref16
    ctx = _ctx(dcmod, r["d"], form)
    st = ctx.subdivide(r["eps"], 0.0, "local")
    top, split, res = ctx.subdivision_info(r["n_old"])
    assert np.abs(top - r["top"]).max() <= 1e-8 * r["top"].max()
    assert st.n_split == N_SPLIT and np.array_equal(split, r["split"])
    ptr, start = ctx.panels()
    assert np.array_equal(ptr, r["d2"].panel_ptr) and np.array_equal(start, r["d2"].panel_start)
    mism = np.flatnonzero(res != r["res"])
    assert all(abs(r["score"][q] - 0.9) < 1e-6 for q in mism), mism
    sig = ctx.get_density()
    err = np.abs(sig - r["loc"]).max() / np.abs(r["loc"]).max()
    print(f"{form}: {st.n_split} split, {st.n_resolve_panels} of {st.n_panels_after} panels re-solved "
          f"({st.n_label_matvec} label applications), iterations {list(st.iters)}, local residual "
          f"{max(st.rel_resid):.1e}; sigma vs oracle {err:.2e}; ms test {st.ms_test:.1f} rebuild "
          f"{st.ms_rebuild:.1f} label {st.ms_label:.1f} solve {st.ms_solve:.1f}")
    assert len(mism) == 0
    assert st.converged == 1
    assert err <= 1e-8
    ctx.close()


@pytest.mark.parametrize("form", ["fmm32", "dense64"])
def test_subdivide_global_resolve_matches_oracle(dcmod, cuda_ok, ref16, form):
    r = ref16
    ctx = _ctx(dcmod, r["d"], form)
    st = ctx.subdivide(r["eps"], 0.0, "global")
    assert st.n_resolve_panels == st.n_panels_after
    sig = ctx.get_density()
    err = np.abs(sig - r["glob"]).max() / np.abs(r["glob"]).max()
    loc_gap = np.abs(r["loc"] - r["glob"]).max() / np.abs(r["glob"]).max()
    print(f"{form} global: sigma vs oracle {err:.2e} (local vs global re-solve in the oracle: "
          f"{loc_gap:.2e}), iterations {list(st.iters)}")
    assert err <= 1e-8
    ctx.close()


def test_subdivide_without_splits_changes_nothing(dcmod, cuda_ok, ref16):
    r = ref16
    ctx = _ctx(dcmod, r["d"], "fmm32")
    before = ctx.get_density()
    st = ctx.subdivide(1e300, 0.0, "local")
    assert st.n_split == 0 and st.n_panels_after == st.n_panels_before
    assert np.array_equal(ctx.get_density(), before)
    with pytest.raises(dcmod.DcError) as e:
        ctx.subdivide(-1.0)
    assert e.value.status == dcmod.DC_ERR_ARG
    ctx.close()
