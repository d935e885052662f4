"""Small fixed workloads for profilers (ncu) and quick timing on one GPU.

    python -m paper_2311_14312_gb300.profile render --size 512
    python -m paper_2311_14312_gb300.profile matvec --reps 20
    python -m paper_2311_14312_gb300.profile solve

Each builds the 200-curve mixed drawing (27,888 nodes, 139,440 segments) in
the chosen FP32 form with order 24 and leaf size 64, solves it, then:

  render  renders [0,1]^2 at size x size twice (the second call with device
          timing) and prints the render and evaluation times;
  matvec  applies the inner FP32 operator `reps` times inside the NVTX range
          "inner" and the FP64 single layer 4 times inside the range "fp64"
          (profilers can filter on them), the FP64 double layer 4 times,
          and prints the mean device time of each;
  solve   solves again inside the NVTX range "solve" and prints the solve
          statistics, the preconditioner state and the tree sizes;
  build   builds the drawing again `reps` times (the last inside the NVTX
          range "build") and prints the wall time of each build phase.
"""
from __future__ import annotations

import argparse


def _context(p_inner=0, inner_tol=0.0, leaf_size=64, m2l_engine=0):
    from dc_synth import drawing_by_name

    from . import Context
    d = drawing_by_name("mixed200")
    ctx = Context(form="fmm32", g=d.g, s_per_panel=d.s_per_panel, p=24, leaf_size=leaf_size,
                  gmres_tol=1e-10, gmres_restart=200, gmres_max_iter=3000, p_inner=p_inner,
                  inner_tol=inner_tol, m2l_engine=m2l_engine)
    ctx.build_drawing(d)
    st = ctx.solve_density()
    return ctx, st


def _time(fn, n):
    import torch
    s = torch.cuda.current_stream()
    fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(n):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / n


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser(description="fixed workloads for profiling")
    ap.add_argument("what", choices=["render", "matvec", "solve", "build"])
    ap.add_argument("--size", type=int, default=512)
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--p-inner", type=int, default=0, help="options.p_inner (0 = default)")
    ap.add_argument("--inner-tol", type=float, default=0.0, help="options.inner_tol (0 = default)")
    ap.add_argument("--leaf-size", type=int, default=64)
    ap.add_argument("--m2l-engine", type=int, default=0, help="options.m2l_engine (0 tensor cores, 1 CUDA cores)")
    a = ap.parse_args(argv)
    ctx, st = _context(a.p_inner, a.inner_tol, a.leaf_size, a.m2l_engine)
    if a.what == "build":
        from dc_synth import drawing_by_name
        d = drawing_by_name("mixed200")
        rows = []
        for r in range(max(1, a.reps)):
            last = r == max(1, a.reps) - 1
            if last:
                torch.cuda.nvtx.range_push("build")
            ctx.build_drawing(d)
            torch.cuda.synchronize()
            if last:
                torch.cuda.nvtx.range_pop()
            rows.append(ctx.build_timings())
        for k in rows[0]:
            vals = [row[k] for row in rows]
            print(f"{k:>15s}: " + " ".join(f"{v:8.2f}" for v in vals) + " ms")
        return
    if a.what == "solve":      # a second solve, inside the NVTX range "solve": steady state
        torch.cuda.nvtx.range_push("solve")
        st = ctx.solve_density()
        torch.cuda.nvtx.range_pop()
    if a.what == "solve":
        sz = ctx.sizes()
        print(f"solve {st.ms_solve:.1f} ms (rhs {st.ms_rhs:.2f} ms) iters {list(st.iters)} "
              f"matvecs {st.n_matvec} refinement steps {st.n_refine} resid {max(st.rel_resid):.2e}")
        print("preconditioner:", ctx.precond_info())
        print(f"tree: nodes {sz.n_nodes} segments {sz.n_segments} pieces {sz.n_pieces} cells "
              f"{sz.n_cells} leaves {sz.n_leaves} depth {sz.depth}; per matvec: near pairs "
              f"{st.p2p_pairs} M2L pairs {st.m2l_pairs}")
    elif a.what == "render":
        n = a.size
        rgb = torch.empty((n * n, 3), dtype=torch.float32, device="cuda")
        rgb8 = torch.empty((n * n, 3), dtype=torch.uint8, device="cuda")
        ctx.render_viewport([(0.0, 0.0, 1.0, 1.0, n, n)], rgb, rgb8)
        torch.cuda.synchronize()
        rs = ctx.render_viewport([(0.0, 0.0, 1.0, 1.0, n, n)], rgb, rgb8, stats=True)
        print(f"render {n}x{n}: {rs.ms:.3f} ms, evaluation {rs.ms_eval:.3f} ms, "
              f"{rs.eval_flops / (rs.ms_eval * 1e9):.2f} TFLOP/s; near pairs {rs.p2p_pairs} "
              f"list-3 pairs {rs.m2p_pairs}")
    else:
        n = ctx.sizes().n_nodes
        x = torch.randn((n, 3), dtype=torch.float64, device="cuda")
        y = torch.empty_like(x)
        torch.cuda.nvtx.range_push("inner")
        t_in = _time(lambda: ctx.apply_operator(x, y, 0, True), a.reps)
        torch.cuda.nvtx.range_pop()
        torch.cuda.nvtx.range_push("fp64")
        t_g = _time(lambda: ctx.apply_operator(x, y, 0, False), 3)
        torch.cuda.nvtx.range_pop()
        t_f = _time(lambda: ctx.apply_operator(x, y, 1, False), 3)
        print(f"solve {st.ms_solve:.1f} ms iters {list(st.iters)} matvecs {st.n_matvec}")
        print(f"inner FP32 operator {t_in:.4f} ms; FP64 G_H {t_g:.4f} ms; FP64 F_H {t_f:.4f} ms")
        # the preconditioned FP32 operator against FP64 G_H applied to M v
        for name, v in (("random", x), ):
            y1 = torch.empty_like(v)
            w = torch.empty_like(v)
            y2 = torch.empty_like(v)
            ctx.apply_operator(v, y1, 0, 1)
            ctx.apply_operator(v, w, 0, 3)
            ctx.apply_operator(w, y2, 0, 0)
            rel = (torch.linalg.norm(y1 - y2, dim=0) / torch.linalg.norm(y2, dim=0)).cpu().numpy()
            print(f"G_H M (FP32 graph) vs FP64 G_H (M v) on the {name} vector: relative error per channel "
                  f"{[f'{r:.2e}' for r in rel]}; |v| {torch.linalg.norm(v).item():.3e} |M v| "
                  f"{torch.linalg.norm(w).item():.3e} |G_H M v| {torch.linalg.norm(y2).item():.3e} "
                  f"finite {bool(torch.isfinite(y1).all())}")
        # accuracy of the FP32 operator (no preconditioner) against the FP64 one
        sig = torch.from_numpy(ctx.get_density()).cuda()
        for name, v in (("random", x), ("solution", sig)):
            y64 = torch.empty_like(v)
            y32 = torch.empty_like(v)
            ctx.apply_operator(v, y64, 0, False)
            ctx.apply_operator(v, y32, 0, 2)
            rel = (torch.linalg.norm(y32 - y64, dim=0) / torch.linalg.norm(y64, dim=0)).cpu().numpy()
            print(f"FP32 operator vs FP64 on the {name} density: relative error per channel "
                  f"{[f'{r:.2e}' for r in rel]}")


if __name__ == "__main__":
    main()
