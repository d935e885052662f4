"""Search over the tunable options of the chosen FP32 form for one drawing and
set of viewports: leaf size b (pieces per quadtree leaf) and the inner
operator's order p_inner, timing solve + render on the device and keeping
only candidates whose pixels stay within a colour tolerance of a plain FP64
FMM reference (order 30).  Host-side search through the public ABI; every
candidate runs the library's kernels.

    from paper_2311_14312_gb300 import autotune
    best, table = autotune.autotune(drawing, [(0, 0, 1, 1, 1024, 1024)])
"""
from __future__ import annotations

import itertools


def _time_step(ctx, vps, rgb, repeats):
    import torch
    s = torch.cuda.current_stream()
    ctx.solve_density()                       # warm-up: graphs, buffers
    ctx.render_viewport(vps, rgb)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(repeats):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        ctx.solve_density()
        ctx.render_viewport(vps, rgb)
        e1.record(s)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def autotune(drawing, viewports, leaf_sizes=(32, 48, 64, 96, 128), p_inners=(10, 12, 14),
             p=24, tol=1e-5, repeats=2, gmres_tol=1e-10):
    """(best options dict, list of (options, ms or None, max colour error)).
    A candidate whose pixels differ from the reference by more than tol, or
    whose solve does not converge, is recorded with ms None."""
    import torch

    from . import Context, DcError
    n = sum(v[4] * v[5] for v in viewports)
    ref = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    rc = Context(form="fmm64", g=drawing.g, s_per_panel=drawing.s_per_panel, p=30, leaf_size=32,
                 gmres_tol=1e-12, gmres_restart=400, gmres_max_iter=4000)
    rc.build_drawing(drawing)
    rc.solve_density()
    rc.render_viewport(viewports, ref)
    rc.close()
    table = []
    rgb = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    for leaf, pi in itertools.product(leaf_sizes, p_inners):
        opts = dict(p=p, leaf_size=leaf, p_inner=min(pi, p), gmres_tol=gmres_tol, gmres_restart=200,
                    gmres_max_iter=3000)
        try:
            ctx = Context(form="fmm32", g=drawing.g, s_per_panel=drawing.s_per_panel, **opts)
            ctx.build_drawing(drawing)
            ms = _time_step(ctx, viewports, rgb, repeats)
            torch.cuda.synchronize()
            err = float((rgb - ref).abs().max().item())
            ctx.close()
        except DcError:
            table.append((opts, None, float("inf")))
            continue
        table.append((opts, ms if err <= tol else None, err))
    ok = [t for t in table if t[1] is not None]
    best = min(ok, key=lambda t: t[1])[0] if ok else None
    return best, table
