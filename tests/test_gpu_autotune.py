"""The option search of the chosen form (dc_autotune through the C ABI:
leaf size x inner order x pixel tile shape) on a small drawing: every
candidate is timed and checked against the plain FP64 FMM render, the
fastest accurate one is chosen, and the JSON cache returns the same choice
for the same inputs without running again."""
import numpy as np
import pytest

from dc_synth import drawing_by_name

pytestmark = pytest.mark.gpu

VPS = [(0.0, 0.0, 1.0, 1.0, 64, 64), (0.2, 0.3, 0.5, 0.6, 40, 24)]


def test_autotune_picks_an_accurate_candidate_and_caches(dcmod, cuda_ok, tmp_path, monkeypatch):
    from paper_2311_14312_gb300 import autotune
    monkeypatch.setenv("DC_AUTOTUNE_CACHE", str(tmp_path / "at.json"))
    d = drawing_by_name("mixed16")
    kw = dict(leaf_sizes=(16, 32), p_inners=(10, 12), eval_tiles=(0, 2), repeats=1)
    best, table, cached = autotune.autotune(d, VPS, **kw)
    for r in table:
        print(r)
    assert not cached and len(table) == 8
    assert best is not None
    ok = [r for r in table if r["converged"] and r["max_err"] <= 1e-5 and r["ms"] > 0]
    chosen = min(ok, key=lambda r: r["ms"])
    assert (best["leaf_size"], best["p_inner"], best["eval_tile"]) == (
        chosen["leaf_size"], chosen["p_inner"], chosen["eval_tile"])
    best2, table2, cached2 = autotune.autotune(d, VPS, **kw)
    assert cached2 and best2 == best and table2 == table


def test_every_tile_shape_renders_the_same_pixels(dcmod, cuda_ok):
    import torch
    d = drawing_by_name("mixed16")
    outs = []
    for t in range(4):
        ctx = dcmod.Context(form="fmm32", g=d.g, s_per_panel=d.s_per_panel, leaf_size=32, eval_tile=t)
        ctx.build_drawing(d)
        ctx.solve_density()
        n = sum(v[4] * v[5] for v in VPS)
        rgb = torch.empty((n, 3), dtype=torch.float32, device="cuda")
        ctx.render_viewport(VPS, rgb)
        torch.cuda.synchronize()
        outs.append(rgb.cpu().numpy())
        ctx.close()
    for o in outs[1:]:   # the same per-pixel work in the same order (FMA contraction may differ)
        assert np.abs(o - outs[0]).max() <= 1e-6
