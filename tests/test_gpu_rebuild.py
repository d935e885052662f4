"""Rebuilding one context: the overlapped build (preconditioner, node
coefficients and FP32 arrays on helper threads and side streams) and the
context's cache of device blocks, which hands the previous drawing's buffers
to the next one, must leave no trace of the earlier drawing.

  * A context that builds mixed16, then closed4 (fewer nodes: recycled
    blocks larger than needed), then mixed16 again (more: some fresh
    allocations) gives, for each drawing, the same density and the same
    rendered bytes as a fresh context that only ever built that drawing,
    bit for bit, in the FP32 FMM form and in the FP64 FMM form.
  * The density also matches the oracle's LU solve within the form's bar.
  * The build's phase timings are finite and add up to less than the total.
"""
import dataclasses

import numpy as np
import pytest
import torch

from dc_synth import drawing_by_name

pytestmark = pytest.mark.gpu

VP = [(0.0, 0.0, 1.0, 1.0, 96, 96)]


def _solve_render(ctx):
    st = ctx.solve_density()
    assert st.converged == 1
    sig = ctx.get_density()
    rgb = torch.empty((96 * 96, 3), dtype=torch.float64, device="cuda")
    rgb8 = torch.empty((96 * 96, 3), dtype=torch.uint8, device="cuda")
    ctx.render_viewport(VP, rgb, rgb8)
    torch.cuda.synchronize()
    return sig, rgb.cpu().numpy(), rgb8.cpu().numpy()


@pytest.mark.parametrize("form,tol", [("fmm32", 1e-6), ("fmm64", 1e-8)])
def test_rebuild_matches_fresh_context(dcmod, cuda_ok, oracle_mod, form, tol):
    O = oracle_mod
    names = ["mixed16", "closed4", "mixed16"]
    # one discretisation rule for all (a context's g and s are fixed)
    drawings = {n: dataclasses.replace(drawing_by_name(n), g=8, s_per_panel=40) for n in set(names)}
    opts = dict(form=form, g=8, s_per_panel=40, p=20, leaf_size=32)
    fresh = {}
    for n, d in drawings.items():
        ctx = dcmod.Context(**opts)
        ctx.build_drawing(d)
        fresh[n] = _solve_render(ctx)
        ctx.close()
    ctx = dcmod.Context(**opts)
    for n in names:
        d = drawings[n]
        ctx.build_drawing(d)
        sig, rgb, rgb8 = _solve_render(ctx)
        f_sig, f_rgb, f_rgb8 = fresh[n]
        assert np.array_equal(sig, f_sig), n
        assert np.array_equal(rgb, f_rgb) and np.array_equal(rgb8, f_rgb8), n
        disc = O.discretise(d)
        ref = O.solve(d, disc).sigma
        err = np.abs(sig - ref).max() / np.abs(ref).max()
        assert err <= tol, (n, err)
        t = ctx.build_timings()
        vals = [v for k, v in t.items() if k != "total"]
        assert all(np.isfinite(v) and v >= 0.0 for v in vals)
        assert sum(vals) <= t["total"] * 1.01 + 0.05
    ctx.close()
