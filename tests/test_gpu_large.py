"""The two large workloads at their full sizes, checked on samples the
oracle computes one by one (its dense LU is out of reach at these sizes):

  * batched2000: 2000 curves, 285,328 unknowns x 3 channels, 1,426,640
    segments; 64 square viewports of 256..4096 pixels at zoom 1..1e6 centred
    on curve points (about 1.9e8 pixels in one call); FP32 form, p = 24,
    GMRES tolerance 1e-10;
  * near20k: 20,000 curves of which 2,000 start 1e-4 from another, 1,409,808
    unknowns x 3 channels, 7,049,040 segments; 8192 x 8192 render of
    [0,1]^2; FP32 form, GMRES tolerance 1e-8.

Solve: the density the library returns, put into the oracle's rows of G_H
and F_H (Eq. 27) at seeded nodes, leaves a residual far below the
right-hand side (a property of the result; the FMM at p = 24 approximates
the rows to about 1e-9).  Render: with a seeded density set through the ABI
(inputs from the generator), the colours at sampled pixels of every
viewport match the oracle's direct sum (Eq. 23) within 1e-5, the viewports
at zoom 1e5..1e6 included, and the 8-bit output is identical outside the
rounding band.
"""
import numpy as np
import pytest

from dc_synth import drawing_by_name, random_node_values, viewport_set

pytestmark = pytest.mark.gpu

DOMAIN = (-0.5, -0.5, 1.5, 1.5)


def _ctx(P, d, tol):
    ctx = P.Context(form="fmm32", g=d.g, s_per_panel=d.s_per_panel, p=24, leaf_size=64, gmres_tol=tol,
                    gmres_restart=200, gmres_max_iter=3000, domain=DOMAIN)
    ctx.build_drawing(d)
    return ctx


def _solve_residual(O, d, disc, ctx, n_rows, seed):
    st = ctx.solve_density()
    sig = ctx.get_density()
    rows = np.sort(np.random.default_rng(seed).choice(disc.n_nodes, n_rows, replace=False))
    AG, AF = O.hybrid_rows(disc, rows)
    up, um = O.boundary_values(d, disc)
    b = 0.5 * (up[rows] + um[rows]) - AF @ (up - um)
    rel = np.abs(AG @ sig - b).max() / np.abs(b).max()
    return st, rel


def _sampled_pixels(vps, per_vp, seed):
    rng = np.random.default_rng(seed)
    idx, offs, o = [], [], 0
    for v in vps:
        n = v[4] * v[5]
        k = min(per_vp, n)
        idx.append(o + np.sort(rng.choice(n, k, replace=False)))
        offs.append(o)
        o += n
    return idx, offs, o


def _check_render(O, ctx, disc, vps, per_vp, seed, up, um):
    import torch
    sig = random_node_values(disc.n_nodes, seed=seed, scale=3.0)
    ctx.set_density(sig)
    idx, offs, npx = _sampled_pixels(vps, per_vp, seed + 1)
    rgb = torch.empty((npx, 3), dtype=torch.float32, device="cuda")
    rgb8 = torch.empty((npx, 3), dtype=torch.uint8, device="cuda")
    rs = ctx.render_viewport(vps, rgb, rgb8, stats=True)
    torch.cuda.synchronize()
    worst, worst_zoom, mism = 0.0, 0.0, 0
    for v, ix, o in zip(vps, idx, offs):
        pts = O.pixel_centres(v[:4], v[4], v[5], ix - o)
        ref = O.layer_potential(disc, pts, sig, up - um)
        got = rgb[torch.from_numpy(ix).cuda()].cpu().numpy().astype(np.float64)
        got8 = rgb8[torch.from_numpy(ix).cuda()].cpu().numpy().astype(np.float64)
        err = np.abs(got - ref).max()
        worst = max(worst, err)
        if 1.0 / (v[2] - v[0]) >= 1e5:
            worst_zoom = max(worst_zoom, err)
        u = 255.0 * np.clip(ref, 0.0, 1.0)
        band = np.abs(u - np.floor(u) - 0.5) <= 255.0 * 1e-5
        mism += int(((got8 != np.floor(u + 0.5)) & ~band).sum())
    return rs, npx, worst, worst_zoom, mism


def test_batched2000_solve_and_64_viewports(dcmod, cuda_ok, oracle_mod):
    O = oracle_mod
    d = drawing_by_name("batched2000")
    disc = O.discretise(d)
    ctx = _ctx(dcmod, d, 1e-10)
    st, rel = _solve_residual(O, d, disc, ctx, 48, 71)
    print(f"batched2000: iterations {list(st.iters)}, oracle-row residual {rel:.2e}")
    assert st.converged == 1 and max(st.rel_resid) <= 1e-10
    assert rel <= 1e-6
    vps = viewport_set(d, seed=20231129, n=64)
    zooms = [1.0 / (v[2] - v[0]) for v in vps]
    assert max(zooms) > 1e5
    up, um = O.boundary_values(d, disc)
    rs, npx, worst, worst_zoom, mism = _check_render(O, ctx, disc, vps, 6, 73, up, um)
    print(f"batched2000: {len(vps)} viewports, {npx} pixels, max zoom {max(zooms):.3g}; sampled colour "
          f"error {worst:.2e} (zoom >= 1e5: {worst_zoom:.2e}); 8-bit mismatches outside the band {mism}")
    assert rs.pixels == npx
    assert worst <= 1e-5 and mism == 0
    ctx.close()


def test_near20k_solve_and_8192_render(dcmod, cuda_ok, oracle_mod):
    O = oracle_mod
    d = drawing_by_name("near20k")
    disc = O.discretise(d)
    ctx = _ctx(dcmod, d, 1e-8)
    st, rel = _solve_residual(O, d, disc, ctx, 24, 81)
    print(f"near20k: iterations {list(st.iters)}, oracle-row residual {rel:.2e}")
    assert st.converged == 1 and max(st.rel_resid) <= 1e-8
    assert rel <= 1e-5
    vps = [(0.0, 0.0, 1.0, 1.0, 8192, 8192)]
    up, um = O.boundary_values(d, disc)
    rs, npx, worst, _, mism = _check_render(O, ctx, disc, vps, 160, 83, up, um)
    print(f"near20k: 8192^2 render, sampled colour error {worst:.2e}; 8-bit mismatches outside the band {mism}")
    assert worst <= 1e-5 and mism == 0
    ctx.close()
