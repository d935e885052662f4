"""Many uneven viewports in one dc_render_viewport call (all tiles in one
evaluation launch): the concatenated output equals rendering each viewport
alone, and sampled pixels match the oracle's direct sum."""
import numpy as np
import pytest

from dc_synth import drawing_by_name

pytestmark = pytest.mark.gpu


def viewports(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        w = rng.uniform(0.02, 0.6)
        h = w * rng.uniform(0.5, 2.0)
        x0 = rng.uniform(0.0, 1.0 - w)
        y0 = rng.uniform(0.0, max(1e-3, 1.0 - h))
        y1 = min(1.0, y0 + h)
        out.append((x0, y0, x0 + w, y1, int(rng.integers(4, 65)), int(rng.integers(4, 49))))
    return out


@pytest.mark.parametrize("form,tol", [("fmm32", 1e-5), ("fmm64", 1e-8)])
def test_64_uneven_viewports_in_one_call(dcmod, cuda_ok, oracle_mod, form, tol):
    import torch
    d = drawing_by_name("mixed16")
    extra = dict(p=30) if form == "fmm64" else {}
    ctx = dcmod.Context(form=form, g=d.g, s_per_panel=d.s_per_panel, leaf_size=32,
                        gmres_tol=1e-12 if form == "fmm64" else 1e-10, gmres_restart=300, **extra)
    ctx.build_drawing(d)
    ctx.solve_density()
    vps = viewports(64, seed=61)
    n = sum(v[4] * v[5] for v in vps)
    together = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
    ctx.render_viewport(vps, together)
    alone = []
    for v in vps:
        o = torch.empty((v[4] * v[5], 3), dtype=torch.float64, device="cuda")
        ctx.render_viewport([v], o)
        alone.append(o)
    torch.cuda.synchronize()
    got = together.cpu().numpy()
    np.testing.assert_array_equal(got, torch.cat(alone).cpu().numpy())
    # sampled pixels of every viewport against the oracle
    disc = oracle_mod.discretise(d)
    sig = ctx.get_density()
    up, um = oracle_mod.boundary_values(d, disc)
    rng = np.random.default_rng(62)
    off, errs = 0, []
    for v in vps:
        npx = v[4] * v[5]
        idx = rng.choice(npx, size=min(6, npx), replace=False)
        ref = oracle_mod.layer_potential(disc, oracle_mod.pixel_centres(v[:4], v[4], v[5], idx), sig, up - um)
        errs.append(np.abs(got[off + idx] - ref).max())
        off += npx
    print(f"{form}: {len(vps)} viewports, {n} pixels, max error on sampled pixels {max(errs):.2e}")
    assert max(errs) <= tol


def test_render_replays_under_cuda_graph_capture(dcmod, cuda_ok):
    """After a first call has planned the tiles, a render of the same
    viewports issues only asynchronous work on the context's stream: it can
    be captured into a CUDA graph (the FP64 passes, the FP32 copies of the
    expansions and the one evaluation launch over all viewports) and
    replayed; the replay reproduces the direct render bit for bit."""
    import torch
    d = drawing_by_name("mixed16")
    s = torch.cuda.Stream()
    ctx = dcmod.Context(stream=s.cuda_stream, form="fmm32", g=d.g, s_per_panel=d.s_per_panel, leaf_size=32,
                        gmres_tol=1e-10, gmres_restart=300)
    ctx.build_drawing(d)
    ctx.solve_density()
    vps = viewports(64, seed=62)
    n = sum(v[4] * v[5] for v in vps)
    direct = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    with torch.cuda.stream(s):
        ctx.render_viewport(vps, direct)                 # plans the tiles
    s.synchronize()
    out = torch.full((n, 3), float("nan"), dtype=torch.float32, device="cuda")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ctx.render_viewport(vps, out)
    out.fill_(float("nan"))
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()
    assert torch.equal(out, direct)
