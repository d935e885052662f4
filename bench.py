#!/usr/bin/env python
"""Benchmark of the hybrid BIE diffusion-curve hot path on GB300.

One step = solve for the density (GMRES, Alg. 3) + render one viewport
(Alg. 4) of a seeded synthetic drawing: 200 cubic Bezier curves (120 open,
80 closed) with adaptive panels (27,888 Gauss-Legendre nodes x 3 colour
channels, 139,440 segments) rendered at 2048 x 2048 over the unit canvas,
in the chosen form (FP32 FMM, FP64 GMRES with iterative refinement to a
relative residual of 1e-10).  The metric is render throughput in
Mpixels/s of the whole step (solve included), with the solve time and the
render-only rate reported beside it, and the plain FP64 FMM form timed on
the same inputs.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Multi-GPU runs are independent replicas (the path does not shard here).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpixels/s render + GMRES solve ms at <=1e-5 err vs FP64 (chosen vs plain form)"
UNIT = "Mpixels/s"
WORKLOAD = "mixed200"
WIDTH = HEIGHT = 2048
VIEWPORT = (0.0, 0.0, 1.0, 1.0)
FORM_OPTS = dict(p=24, leaf_size=64, gmres_tol=1e-10, gmres_restart=200, gmres_max_iter=3000)
# nominal dense tensor rates (NVIDIA's GB300 figures without sparsity): the
# TF32 peak is the measured BF16 peak times their ratio
NOMINAL_TF32_OVER_BF16 = 1.1 / 2.25
FALLBACK_BF16_TFLOPS = 1900.0


# The large cases: the 2000-curve drawing rendered into 64 uneven viewports
# (256..4096 px, zoom 1..1e6, centred on curve points) in one call, and the
# 20k-curve drawing with near-touching pairs rendered at 8192^2.
LARGE = {
    "batched2000": dict(tol=1e-10, viewports="64 seeded viewports (seed 20231129)"),
    "near20k": dict(tol=1e-8, viewports="[0,1]^2 at 8192x8192"),
}
LARGE_DOMAIN = (-0.5, -0.5, 1.5, 1.5)


def measured_peaks() -> dict:
    """The driver-written measured peaks of this machine's GPUs, if present."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def cpu_model() -> str:
    """CPU model name from /proc/cpuinfo (x86 'model name'; Arm machines give
    implementer / part numbers only, reported as such)."""
    try:
        txt = open("/proc/cpuinfo").read()
    except Exception:
        return "unknown"
    for key in ("model name", "Model name"):
        for ln in txt.splitlines():
            if ln.startswith(key):
                return ln.split(":", 1)[1].strip()
    impl = part = None
    for ln in txt.splitlines():
        if ln.startswith("CPU implementer") and impl is None:
            impl = ln.split(":", 1)[1].strip()
        if ln.startswith("CPU part") and part is None:
            part = ln.split(":", 1)[1].strip()
    return f"Arm implementer {impl} part {part}" if impl else "unknown"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 FMM comparison")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--workload", default=WORKLOAD, choices=[WORKLOAD, *LARGE],
                    help="mixed200 (the headline) or one of the large cases, measured on their own")
    return ap.parse_args()


# ------------------------------------------------------------ helpers --
class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def traffic_for_eval_kernel():
    """DRAM bytes per launch of the eval kernel from a committed ncu
    summary, valid only while the kernel source is unchanged."""
    src = os.path.join(ROOT, "paper_2311_14312_gb300", "csrc", "fmm32.cu")
    path = os.path.join(ROOT, "profiles", "eval32_traffic.json")
    try:
        ref = json.load(open(path))
        sha = hashlib.sha1(open(src, "rb").read()).hexdigest()
        if ref.get("source_sha1") == sha and ref.get("workload") == WORKLOAD:
            return ref.get("bytes_per_launch")
    except Exception:
        pass
    return None


def whole_job_rate(t_step_ms: float, npx: int, ws: int, device: str):
    """(slowest rank's step time, whole-job Mpixels/s): every rank renders npx
    pixels per step (replicas), the job's step time is the maximum over ranks."""
    if ws > 1:
        import torch
        t = torch.tensor([t_step_ms], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_step_ms = float(t.item())
    return t_step_ms, ws * npx / (t_step_ms * 1e-3) / 1e6


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------- oracle leg --
def _oracle_setup():
    from dc_synth import drawing_by_name
    from oracle import oracle as O
    d = drawing_by_name(WORKLOAD)
    return O, d, O.discretise(d)


def oracle_render_sample(O, disc, seconds: float, seed: int = 1):
    """Oracle direct-sum render (Eq. 23, Alg. 4) of sampled pixels of the
    viewport with a seeded density (its cost does not depend on the values):
    (pixels, seconds)."""
    from dc_synth import pixel_sample, random_node_values
    sig = random_node_values(disc.n_nodes, seed=seed, scale=0.1)
    mu = random_node_values(disc.n_nodes, seed=seed + 1, scale=0.1)
    probe = pixel_sample(WIDTH, HEIGHT, 64, seed=seed)
    t0 = time.perf_counter()
    O.layer_potential(disc, O.pixel_centres(VIEWPORT, WIDTH, HEIGHT, probe), sig, mu)
    rate = len(probe) / max(time.perf_counter() - t0, 1e-6)
    count = int(max(64, min(WIDTH * HEIGHT, rate * seconds)))
    idx = pixel_sample(WIDTH, HEIGHT, count, seed=seed + 2)
    t0 = time.perf_counter()
    O.layer_potential(disc, O.pixel_centres(VIEWPORT, WIDTH, HEIGHT, idx), sig, mu)
    return count, time.perf_counter() - t0


def oracle_solve_sample(O, disc, rows: int = 512, lu_n: int = 4096):
    """Bounded sample of the oracle's solve (Alg. 3 by dense LU): dense rows
    of G_H and F_H (Eq. 19, 27) for `rows` seeded collocation nodes, and a
    LAPACK LU solve of an lu_n x lu_n system with three right-hand sides.
    Returns the full-size estimate: assembly x N / rows, LU x (N / lu_n)^3
    (LU costs 2/3 n^3 flops), in seconds, and the sample's own seconds."""
    import numpy as np
    N = disc.n_nodes
    sel = np.sort(np.random.default_rng(5).choice(N, min(rows, N), replace=False))
    t0 = time.perf_counter()
    O.hybrid_rows(disc, sel)
    t_rows = time.perf_counter() - t0
    A = np.random.default_rng(6).standard_normal((lu_n, lu_n)) + lu_n * np.eye(lu_n)
    b = np.ones((lu_n, 3))
    t0 = time.perf_counter()
    np.linalg.solve(A, b)
    t_lu = time.perf_counter() - t0
    est = t_rows * N / len(sel) + t_lu * (N / lu_n) ** 3
    return est, t_rows + t_lu


def run_reference(args):
    """The oracle as it stands on the host cores: the whole solve (dense
    assembly of G_H and F_H for all 27,888 nodes and a LAPACK LU solve of the
    three channels, Alg. 3) is timed in full once; every step renders a
    bounded sample of the 2048^2 pixels by direct summation, and the step
    time is the solve plus the full frame's render extrapolated from that
    step's sample."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    O, d, disc = _oracle_setup()
    for _ in range(args.warmup):
        oracle_render_sample(O, disc, 0.3)
    t0 = time.perf_counter()
    O.solve(d, disc)
    t_solve = time.perf_counter() - t0
    per = max(1.0, args.cpu_seconds / max(1, args.steps))
    npx = WIDTH * HEIGHT
    step_s = []
    total_px = 0
    for k in range(args.steps):
        n, dt = oracle_render_sample(O, disc, per, seed=100 + k)
        total_px += n
        step_s.append(t_solve + dt * npx / n)
    t_step = statistics.mean(step_s)
    v = npx / t_step / 1e6
    cores = O.num_threads()
    sample = (f"oracle FP64 on {cores} host threads ({cpu_model()}): dense assembly of G_H and F_H "
              f"for all {disc.n_nodes} nodes + LAPACK LU of 3 channels measured in full once "
              f"({t_solve:.1f} s); the {WIDTH}x{HEIGHT} render extrapolated per step from a direct-sum "
              f"sample ({total_px} pixels over {args.steps} steps)")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "width": WIDTH, "height": HEIGHT},
            "solve_s": t_solve,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "cpu": cpu_model(), "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------- GPU leg --
def next_rows(P, d, ctx, vp, npx):
    """The beyond-the-step rows on the bench drawing, after the timed region
    (host wall times from the library's stats, render times by CUDA events):
    f3 anti-aliasing of the 2048^2 render (m = 2), f2 the viewport update of
    a zoom-8 viewport (e rule, no subdivision) and its render, f1 one round
    of adaptive subdivision with the local re-solve (epsilon_2 at the 99.5th
    percentile of the test values)."""
    import numpy as np
    import torch

    out = {}
    sig = ctx.get_density()
    rgb = torch.empty((npx, 3), dtype=torch.float32, device="cuda")
    rgb8 = torch.empty((npx, 3), dtype=torch.uint8, device="cuda")
    # f3
    actx = P.Context(form="fmm32", g=d.g, s_per_panel=d.s_per_panel, aa_levels=2, **FORM_OPTS)
    actx.build_drawing(d)
    actx.set_density(sig)
    actx.render_viewport(vp, rgb, rgb8)
    rs = actx.render_viewport(vp, rgb, rgb8, stats=True)
    out["f3_antialias"] = {"levels": 2, "ms": rs.ms, "ms_aa": rs.ms_aa, "refined_pixels": rs.aa_pixels,
                           "samples": rs.aa_samples}
    actx.close()
    # f2
    c = d.ctrl[0].mean(axis=0)
    zv = (float(c[0] - 1 / 16), float(c[1] - 1 / 16), float(c[0] + 1 / 16), float(c[1] + 1 / 16), WIDTH, HEIGHT)
    vs = ctx.view_update(zv, eps_coef=0.0)
    ctx.render_viewport([zv], rgb, rgb8)
    rv = ctx.render_viewport([zv], rgb, rgb8, stats=True)
    ctx.view_reset()
    rp = ctx.render_viewport([zv], rgb, rgb8, stats=True)
    out["f2_view"] = {"zoom": 8, "e": vs.e, "s": d.s_per_panel, "labels_fixed_interp_resolve":
                      [vs.n_fixed, vs.n_interpolating, vs.n_resolving], "ms_build": vs.ms_build,
                      "render_ms": rv.ms, "render_ms_solve_polyline": rp.ms}
    # f1
    n0 = ctx.sizes().n_panels
    ctx.subdivide(1e300)
    top, _, _ = ctx.subdivision_info(n0)
    eps = float(np.percentile(top, 99.5))
    ss = ctx.subdivide(eps, 0.0, "local")
    out["f1_subdivide"] = {"eps_coef": eps, "n_split": ss.n_split, "panels": [ss.n_panels_before, ss.n_panels_after],
                           "resolved_panels": ss.n_resolve_panels, "iters": list(ss.iters),
                           "ms_test": ss.ms_test, "ms_rebuild": ss.ms_rebuild, "ms_label": ss.ms_label,
                           "ms_solve": ss.ms_solve}
    return out


def run_ours(args):
    import numpy as np
    import torch

    import paper_2311_14312_gb300 as P
    from dc_synth import drawing_by_name

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    d = drawing_by_name(WORKLOAD)
    ctx = P.Context(form="fmm32", g=d.g, s_per_panel=d.s_per_panel, **FORM_OPTS)
    ctx.build_drawing(d)
    npx = WIDTH * HEIGHT
    vp = [(*VIEWPORT, WIDTH, HEIGHT)]
    rgb = torch.empty((npx, 3), dtype=torch.float32, device="cuda")
    rgb8 = torch.empty((npx, 3), dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        ctx.solve_density()
        ctx.render_viewport(vp, rgb, rgb8)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    # ---- device-resident timed region (L2 flushed before every step)
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = P.kernel_launches()
    step_ms, solve_ms, render_ms = [], [], []
    barrier()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")     # profilers can filter on this range
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e2 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.solve_density()
        e1.record(stream)
        ctx.render_viewport(vp, rgb, rgb8)
        e2.record(stream)
        e2.synchronize()
        step_ms.append(e0.elapsed_time(e2))
        solve_ms.append(e0.elapsed_time(e1))
        render_ms.append(e1.elapsed_time(e2))
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier()
    launches = P.kernel_launches() - launches0
    clk = clocks.stop()
    t_step, value = whole_job_rate(statistics.mean(step_ms), npx, ws, "cuda")

    # ---- roofline of the dominant kernel (pixel evaluation), live events;
    # its peak is the FP32 FMA rate measured on this GPU
    rs = ctx.render_viewport(vp, rgb, rgb8, stats=True)
    achieved = rs.eval_flops / (rs.ms_eval * 1e-3) / 1e12 if rs.ms_eval > 0 else None
    fp32 = P.fp32_peak()
    props = torch.cuda.get_device_properties(local)
    # ---- the inner operator's tensor-core M2L (Eq. 69), live events
    mp = measured_peaks()
    bf16 = mp.get("bf16_tflops")
    tf32_peak = (bf16 if bf16 else FALLBACK_BF16_TFLOPS) * NOMINAL_TF32_OVER_BF16
    m2l = ctx.time_inner_m2l(20)
    m2l_ms = m2l["ms_main"] + m2l["ms_reduce"]
    m2l_ach = m2l["flops"] / (m2l_ms * 1e-3) / 1e12 if m2l_ms > 0 else None
    st = ctx.solve_density()
    chosen = rgb.float().cpu().numpy()

    # ---- end to end through the C ABI with host buffers
    from dc_synth import drawing_by_name as _dbn  # noqa: F401
    ctrl = np.ascontiguousarray(d.ctrl)
    pptr = np.ascontiguousarray(d.panel_ptr, dtype=np.int32)
    pst = np.ascontiguousarray(d.panel_start)
    col = np.ascontiguousarray(d.colours)
    h_rgb = torch.empty((npx, 3), dtype=torch.float32, pin_memory=True).numpy()
    h_rgb8 = torch.empty((npx, 3), dtype=torch.uint8, pin_memory=True).numpy()
    bi = ctrl.nbytes + pptr.nbytes + pst.nbytes + col.nbytes
    bo = h_rgb.nbytes + h_rgb8.nbytes
    e2e_ms = []
    for k in range(max(1, args.steps)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.build_tree(ctrl, pptr, pst, col)
        ctx.solve_density()
        ctx.render_viewport(vp, h_rgb, h_rgb8)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e = npx / (statistics.mean(e2e_ms) * 1e-3) / 1e6

    # ---- plain FP64 FMM form on the same inputs (accuracy reference too)
    plain = None
    if not args.no_plain and rank == 0:
        pctx = P.Context(form="fmm64", g=d.g, s_per_panel=d.s_per_panel, **FORM_OPTS)
        pctx.build_drawing(d)
        prgb = torch.empty((npx, 3), dtype=torch.float64, device="cuda")
        pctx.solve_density()
        pctx.render_viewport(vp, prgb)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e2 = torch.cuda.Event(enable_timing=True)
        flush.zero_()
        e0.record(stream)
        pst_ = pctx.solve_density()
        e1.record(stream)
        pctx.render_viewport(vp, prgb)
        e2.record(stream)
        e2.synchronize()
        ref = prgb.cpu().numpy()
        err = float(np.abs(chosen - ref).max())
        q_c = np.floor(255 * np.clip(chosen, 0, 1) + 0.5)
        q_r = np.floor(255 * np.clip(ref, 0, 1) + 0.5)
        v8 = 255.0 * np.clip(ref, 0, 1)
        band = np.abs(v8 - np.floor(v8) - 0.5) <= 255.0 * 1e-5
        mism = int(((q_c != q_r) & ~band).sum())
        plain = {"form": "fmm64", "solve_ms": e0.elapsed_time(e1), "render_ms": e1.elapsed_time(e2),
                 "mpix_s": npx / (e0.elapsed_time(e2) * 1e-3) / 1e6,
                 "gmres_iters": list(pst_.iters),
                 "chosen_max_abs_err_vs_plain": err, "chosen_8bit_mismatch_outside_band": mism,
                 "band_pixels": int(band.sum())}
        pctx.close()

    nxt = next_rows(P, d, ctx, vp, npx) if rank == 0 else None

    cpu = None
    if rank == 0 and ws == 1:
        O, _, disc = _oracle_setup()
        est_solve, t_solve_sample = oracle_solve_sample(O, disc)
        n, dt = oracle_render_sample(O, disc, max(2.0, args.cpu_seconds - t_solve_sample))
        t_cpu = est_solve + dt * npx / n
        cpu = {"value": npx / t_cpu / 1e6, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
               "cpu": cpu_model(),
               "sample": f"oracle FP64, extrapolated step {t_cpu:.0f} s: dense rows of G_H/F_H for 512 "
                         f"of {disc.n_nodes} nodes (x{disc.n_nodes / 512:.1f}) and LAPACK LU of a "
                         f"4096^2 system (x(N/4096)^3) for the solve ({est_solve:.0f} s), direct-sum "
                         f"render of {n} sampled pixels of {WIDTH}x{HEIGHT} ({dt:.1f} s, x{npx / n:.0f}); "
                         f"bench.py --impl reference times the whole solve"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD,
                       "drawing": "200 cubic Bezier curves (120 open, 80 closed), seeded; "
                                  f"{d.n_nodes} GL nodes x 3 channels, {d.n_segments} segments",
                       "width": WIDTH, "height": HEIGHT, "form": "fmm32", **FORM_OPTS,
                       "parallelism": f"replicas x{ws}",
                       "l2": "flushed before every timed step (256 MiB write)"},
            "solve_ms": statistics.mean(solve_ms), "render_ms": statistics.mean(render_ms),
            "render_mpix_s": npx / (statistics.mean(render_ms) * 1e-3) / 1e6,
            "gmres_iters": list(st.iters), "gmres_rel_resid": max(st.rel_resid),
            "plain_form": plain,
            "roofline": {"bound": "alu", "kernel": "eval32_kernel<0> (L2P + M2P + P2P per pixel)",
                         "achieved": achieved, "peak": fp32["tflops"], "unit": "TFLOP/s",
                         "frac": (achieved / fp32["tflops"]) if achieved else None,
                         "peak_source": f"measured: FP32 FMA chains on this GPU ({props.multi_processor_count} "
                                        f"SMs), best of 3 launches",
                         "traffic": traffic_for_eval_kernel(),
                         "eval_ms": rs.ms_eval, "eval_flops": rs.eval_flops,
                         "p2p_pairs": rs.p2p_pairs, "m2p_pairs": rs.m2p_pairs},
            "roofline_m2l": {"bound": "tensor",
                             "kernel": ("m2l_tc_kernel + m2l_tc_reduce_kernel (inner operator, p_i = 12, "
                                        "tcgen05 kind::tf32, three-term split)")
                             if m2l["engine"] == P.DC_M2L_TENSOR else "m2l_small_kernel (CUDA cores)",
                             "achieved": m2l_ach, "peak": tf32_peak, "unit": "TFLOP/s",
                             "frac": (m2l_ach / tf32_peak) if m2l_ach else None,
                             "peak_source": ("measured bf16 burst x nominal TF32/BF16 ratio 1.1/2.25"
                                             if bf16 else "fallback 1.9 PFLOP/s bf16 x 1.1/2.25"),
                             "ms": m2l_ms, "ms_main": m2l["ms_main"], "ms_reduce": m2l["ms_reduce"],
                             "algorithmic_flops": m2l["flops"], "tensor_pipe_flops": m2l["tensor_flops"],
                             "pairs": m2l["pairs"]},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo,
                    "includes": "build_tree from host arrays + solve + render to pinned host"},
            "gpu_launches": launches,
            "clocks": clk,
            "next_rows": nxt,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_large(args):
    """A large case on one GPU: every step solves (GMRES to the case's
    tolerance) and renders all of its viewports; the inputs (1.4-7 M
    segments, 0.7-4.6 GB of output) exceed L2.  The plain FP64 FMM form runs
    once on the same inputs."""
    import numpy as np
    import torch

    import paper_2311_14312_gb300 as P
    from dc_synth import drawing_by_name, viewport_set

    cfg = LARGE[args.workload]
    torch.cuda.set_device(0)
    d = drawing_by_name(args.workload)
    vps = (viewport_set(d, seed=20231129, n=64) if args.workload == "batched2000"
           else [(0.0, 0.0, 1.0, 1.0, 8192, 8192)])
    npx = sum(v[4] * v[5] for v in vps)
    opts = dict(p=24, leaf_size=64, gmres_tol=cfg["tol"], gmres_restart=200, gmres_max_iter=3000,
                domain=LARGE_DOMAIN)
    ctx = P.Context(form="fmm32", g=d.g, s_per_panel=d.s_per_panel, **opts)
    t0 = time.perf_counter()
    ctx.build_drawing(d)
    build_s = time.perf_counter() - t0
    rgb = torch.empty((npx, 3), dtype=torch.float32, device="cuda")
    rgb8 = torch.empty((npx, 3), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        ctx.solve_density()
        ctx.render_viewport(vps, rgb, rgb8)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    launches0 = P.kernel_launches()
    step_ms, solve_ms, render_ms = [], [], []
    for _ in range(args.steps):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        st = ctx.solve_density()
        e1.record(stream)
        ctx.render_viewport(vps, rgb, rgb8)
        e2.record(stream)
        e2.synchronize()
        step_ms.append(e0.elapsed_time(e2))
        solve_ms.append(e0.elapsed_time(e1))
        render_ms.append(e1.elapsed_time(e2))
    launches = P.kernel_launches() - launches0
    clk = clocks.stop()
    rs = ctx.render_viewport(vps, rgb, rgb8, stats=True)
    fp32 = P.fp32_peak()
    achieved = rs.eval_flops / (rs.ms_eval * 1e-3) / 1e12 if rs.ms_eval > 0 else None
    # the plain FP64 FMM form on the same inputs, once (its pixels: the
    # chosen form's colour differences on a sample of pixels)
    chosen = rgb[::97].float().cpu().numpy()
    ctx.close()
    pctx = P.Context(form="fmm64", g=d.g, s_per_panel=d.s_per_panel, **opts)
    pctx.build_drawing(d)
    del rgb8
    prgb = torch.empty((npx, 3), dtype=torch.float32, device="cuda")
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record(stream)
    pst = pctx.solve_density()
    e1.record(stream)
    pctx.render_viewport(vps, prgb)
    e2.record(stream)
    e2.synchronize()
    ref = prgb[::97].float().cpu().numpy()
    plain = {"form": "fmm64", "solve_ms": e0.elapsed_time(e1), "render_ms": e1.elapsed_time(e2),
             "mpix_s": npx / (e0.elapsed_time(e2) * 1e-3) / 1e6, "gmres_iters": list(pst.iters),
             "chosen_max_abs_err_vs_plain_every_97th_pixel": float(np.abs(chosen - ref).max())}
    pctx.close()
    t_step = statistics.mean(step_ms)
    line = {"metric": METRIC, "value": npx / (t_step * 1e-3) / 1e6, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "curves": d.n_curves, "nodes": d.n_nodes,
                       "segments": d.n_segments, "viewports": cfg["viewports"], "pixels": npx, "form": "fmm32",
                       **{k: v for k, v in opts.items() if k != "domain"},
                       "l2": "inputs and outputs larger than L2"},
            "build_s": build_s, "solve_ms": statistics.mean(solve_ms), "render_ms": statistics.mean(render_ms),
            "render_mpix_s": npx / (statistics.mean(render_ms) * 1e-3) / 1e6, "gmres_iters": list(st.iters),
            "gmres_rel_resid": max(st.rel_resid), "plain_form": plain,
            "roofline": {"bound": "alu", "kernel": "eval32_kernel<0> (L2P + M2P + P2P per pixel)",
                         "achieved": achieved, "peak": fp32["tflops"], "unit": "TFLOP/s",
                         "frac": (achieved / fp32["tflops"]) if achieved else None, "traffic": None,
                         "eval_ms": rs.ms_eval, "p2p_pairs": rs.p2p_pairs, "m2p_pairs": rs.m2p_pairs},
            "gpu_launches": launches, "clocks": clk}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != WORKLOAD:
        run_large(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
