"""Training of the learned warm start (no counterpart in the paper).

The network, its gradient and the Adam update run in the library's kernels
(dc_aux_mlp_loss_grad, dc_aux_mlp_adam); features and targets come from
dc_aux_panel_features of contexts that hold a solved density.  This module
only draws minibatches and loops.

    python -m paper_2311_14312_gb300.warmstart --out model.npz --drawings 64

trains on seeded synthetic drawings and writes the parameters with their
sizes; ``load`` reads them back for Context.set_warm_start_model.
"""
from __future__ import annotations

import argparse
import time

import numpy as np

from . import (Context, mlp_adam, mlp_loss_grad, mlp_param_count, mlp_workspace_floats)


def init_params(n_in: int, hidden: int, n_out: int, seed: int) -> np.ndarray:
    """He-normal weights (std sqrt(2/fan_in)), zero biases, packed as the
    library expects (W_l [out][in] then b_l per layer); the last layer is
    scaled down so that the first predictions are small."""
    rng = np.random.default_rng(seed)
    d = [n_in, hidden, hidden, hidden, n_out]
    parts = []
    for l in range(4):
        W = rng.standard_normal((d[l + 1], d[l])) * np.sqrt(2.0 / d[l])
        if l == 3:
            W *= 0.1
        parts += [W.ravel(), np.zeros(d[l + 1])]
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == mlp_param_count(n_in, hidden, n_out)
    return p


def collect(ctx: Context):
    """(features, targets) of a context that holds a density, as float32
    CUDA tensors [rows, n_features] and [rows, g]."""
    import torch
    rows, nf, no = ctx.feature_dims()
    feat = torch.empty((rows, nf), dtype=torch.float32, device="cuda")
    targ = torch.empty((rows, no), dtype=torch.float32, device="cuda")
    ctx.panel_features(feat, targ)
    return feat, targ


def train(feat, targ, hidden: int = 128, steps: int = 2000, batch: int = 1024, lr: float = 1e-3,
          seed: int = 0, log_every: int = 0):
    """Adam on the mean squared error; returns (params as a float32 CUDA
    tensor, list of (step, loss))."""
    import torch
    n_rows, n_in = feat.shape
    n_out = targ.shape[1]
    batch = min(batch, n_rows)
    params = torch.from_numpy(init_params(n_in, hidden, n_out, seed)).cuda()
    grad = torch.zeros_like(params)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    work = torch.empty(mlp_workspace_floats(n_in, hidden, n_out, batch), dtype=torch.float32,
                       device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    gen = torch.Generator(device="cpu").manual_seed(seed)
    hist = []
    perm, pos = torch.randperm(n_rows, generator=gen).cuda(), 0
    for step in range(1, steps + 1):
        if pos + batch > n_rows:
            perm, pos = torch.randperm(n_rows, generator=gen).cuda(), 0
        idx = perm[pos:pos + batch]
        pos += batch
        xb = feat.index_select(0, idx).contiguous()
        tb = targ.index_select(0, idx).contiguous()
        mlp_loss_grad(n_in, hidden, n_out, params, xb, tb, grad, loss, work)
        mlp_adam(params, grad, m, v, lr, step)
        if log_every and (step % log_every == 0 or step == steps):
            hist.append((step, float(loss.item())))
    return params, hist


def save(path: str, params, n_in: int, hidden: int, n_out: int, meta: dict | None = None):
    p = params.detach().cpu().numpy() if hasattr(params, "detach") else np.asarray(params)
    np.savez(path, params=p.astype(np.float32), n_in=n_in, hidden=hidden, n_out=n_out,
             **{k: np.asarray(v) for k, v in (meta or {}).items()})


def load(path: str):
    """(params float32 numpy, hidden, n_in, n_out)."""
    z = np.load(path)
    return z["params"], int(z["hidden"]), int(z["n_in"]), int(z["n_out"])


def _gen(args):
    """One seeded training / held-out drawing of the learned-start recipe:
    the mixed generator with a curve count uniform in [8, 64]."""
    from dc_synth.drawings import make_mixed_set
    seed, g = args
    n = 8 + int(np.random.default_rng(seed).integers(0, 57))
    return make_mixed_set(seed, n_curves=n, g=g, name=f"ws{seed}")


def drawings(seeds, g=16, workers=0):
    """The drawings of the given seeds, generated on host processes (spawned,
    so that no CUDA state is forked; the caller's main module must be
    importable, e.g. ``python -m``)."""
    import multiprocessing as mp
    import os
    workers = workers or max(1, min(16, os.cpu_count() or 1))
    if workers == 1:
        return [_gen((s, g)) for s in seeds]
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_gen, [(s, g) for s in seeds], chunksize=8)


def solve_ab(d, params, hidden, form="fmm32"):
    """The paper's x0 = 1 against the learned start on one drawing in the
    given form: iterations (summed over the refinement steps, max over
    channels), solve ms (CUDA events, after one warm-up solve), the learned
    start's residual, refinement steps, and the density difference."""
    import torch

    from . import DC_X0_LEARNED
    kw = dict(form=form, g=d.g, s_per_panel=d.s_per_panel, p=24, leaf_size=64, gmres_tol=1e-10,
              gmres_restart=200, gmres_max_iter=3000)
    out, sig = {}, {}
    for mode in ("cold", "warm"):
        ctx = Context(**kw, **({"x0_mode": DC_X0_LEARNED} if mode == "warm" else {}))
        ctx.build_drawing(d)
        if mode == "warm":
            ctx.set_warm_start_model(hidden, params)
        ctx.solve_density()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st = ctx.solve_density()
        e1.record()
        e1.synchronize()
        out[mode] = dict(iters=max(st.iters), ms=e0.elapsed_time(e1), converged=st.converged,
                         warm_resid=max(st.warm_resid) if mode == "warm" else None, n_refine=st.n_refine)
        sig[mode] = ctx.get_density()
        ctx.close()
    out["sigma_rel_diff"] = float(np.abs(sig["warm"] - sig["cold"]).max() / np.abs(sig["cold"]).max())
    return out


def config3(n_train=2000, n_held=100, hidden=256, steps=6000, batch=4096, lr=1e-3, seed=50000, g=16,
            form="fmm32", out=None, log=print):
    """Train on n_train drawings (8-64 curves each) and compare the learned
    start with x0 = 1 on n_held other drawings; returns the summary dict."""
    import json

    import torch
    t0 = time.time()
    train_d = drawings(range(seed, seed + n_train), g)
    held_d = drawings(range(seed + n_train, seed + n_train + n_held), g)
    t_gen = time.time() - t0
    feats, targs = [], []
    t0 = time.time()
    for d in train_d:
        ctx = Context(form=form, g=d.g, s_per_panel=d.s_per_panel, p=24, leaf_size=64, gmres_tol=1e-10,
                      gmres_restart=200, gmres_max_iter=3000)
        ctx.build_drawing(d)
        ctx.solve_density()
        f, t = collect(ctx)
        feats.append(f)
        targs.append(t)
        ctx.close()
    feat, targ = torch.cat(feats), torch.cat(targs)
    del feats, targs
    t_data = time.time() - t0
    log(f"{feat.shape[0]} rows from {n_train} drawings (generation {t_gen:.0f} s, solves {t_data:.0f} s)")
    t0 = time.time()
    params, hist = train(feat, targ, hidden, steps, batch, lr, seed=seed, log_every=max(1, steps // 10))
    torch.cuda.synchronize()
    t_train = time.time() - t0
    for s_, l_ in hist:
        log(f"step {s_:6d} loss {l_:.4e}")
    rows = [solve_ab(d, params, hidden, form) for d in held_d]
    ci = np.array([r["cold"]["iters"] for r in rows])
    wi = np.array([r["warm"]["iters"] for r in rows])
    cm = np.array([r["cold"]["ms"] for r in rows])
    wm = np.array([r["warm"]["ms"] for r in rows])
    summary = dict(form=form, train_drawings=n_train, heldout_drawings=n_held, rows=int(feat.shape[0]),
                   hidden=hidden, steps=steps, batch=batch, loss_first=hist[0][1], loss_last=hist[-1][1],
                   train_s=t_train, iters_cold_mean=float(ci.mean()), iters_warm_mean=float(wi.mean()),
                   ms_cold_mean=float(cm.mean()), ms_warm_mean=float(wm.mean()),
                   ms_cold_median=float(np.median(cm)), ms_warm_median=float(np.median(wm)),
                   warm_resid_median=float(np.median([r["warm"]["warm_resid"] for r in rows])),
                   refine_cold_mean=float(np.mean([r["cold"]["n_refine"] for r in rows])),
                   refine_warm_mean=float(np.mean([r["warm"]["n_refine"] for r in rows])),
                   all_converged=bool(all(r["cold"]["converged"] and r["warm"]["converged"] for r in rows)),
                   max_sigma_rel_diff=float(max(r["sigma_rel_diff"] for r in rows)))
    log(json.dumps(summary))
    if out:
        save(out, params, feat.shape[1], hidden, targ.shape[1], dict(train_drawings=n_train, seed=seed))
    return summary


def _main():
    import torch
    from dc_synth.drawings import make_mixed_set

    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--out", required=True)
    ap.add_argument("--drawings", type=int, default=32)
    ap.add_argument("--curves", type=int, default=200)
    ap.add_argument("--g", type=int, default=16)
    ap.add_argument("--seed", type=int, default=1000)
    ap.add_argument("--hidden", type=int, default=128)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--batch", type=int, default=2048)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--config3", action="store_true",
                    help="train on --drawings drawings of 8-64 curves and A/B on --heldout others")
    ap.add_argument("--heldout", type=int, default=100)
    ap.add_argument("--form", default="fmm32")
    a = ap.parse_args()
    if a.config3:
        config3(a.drawings, a.heldout, a.hidden, a.steps, a.batch, a.lr, seed=a.seed, g=a.g, form=a.form,
                out=a.out)
        return
    feats, targs = [], []
    t0 = time.time()
    for i in range(a.drawings):
        d = make_mixed_set(a.seed + i, n_curves=a.curves, g=a.g, name=f"train{i}")
        ctx = Context(form="fmm32", g=d.g, s_per_panel=d.s_per_panel, p=24, leaf_size=64,
                      gmres_tol=1e-10, gmres_restart=200, gmres_max_iter=3000)
        ctx.build_drawing(d)
        ctx.solve_density()
        f, t = collect(ctx)
        feats.append(f)
        targs.append(t)
        ctx.close()
    feat, targ = torch.cat(feats), torch.cat(targs)
    print(f"{feat.shape[0]} rows from {a.drawings} drawings in {time.time() - t0:.1f} s")
    params, hist = train(feat, targ, a.hidden, a.steps, a.batch, a.lr, seed=a.seed,
                         log_every=max(1, a.steps // 10))
    for s, l in hist:
        print(f"step {s:6d} loss {l:.4e}")
    save(a.out, params, feat.shape[1], a.hidden, targ.shape[1],
         dict(drawings=a.drawings, curves=a.curves, seed=a.seed, steps=a.steps))


if __name__ == "__main__":
    _main()
