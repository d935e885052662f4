"""Option search of the chosen FP32 form for one drawing and set of viewports
(leaf size b, inner order p_inner, pixel tile shape eval_tile), run by the
library (dc_autotune: each candidate built, timed with CUDA events over
solve + render, and checked against a plain FP64 FMM render), with the
result kept in a JSON cache keyed by the drawing, the viewports, the
candidate lists, the tolerance and the GPU's name, so a later call for the
same inputs on the same kind of GPU returns at once.

    from paper_2311_14312_gb300 import autotune
    best, table, cached = autotune.autotune(drawing, [(0, 0, 1, 1, 1024, 1024)])

The cache file is $DC_AUTOTUNE_CACHE, else ~/.cache/paper_2311_14312_gb300/
autotune.json; cache=False skips it.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np


def cache_path() -> str:
    p = os.environ.get("DC_AUTOTUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_2311_14312_gb300", "autotune.json")


def cache_key(drawing, viewports, leaf_sizes, p_inners, eval_tiles, p, tol, gmres_tol, gpu: str) -> str:
    h = hashlib.sha1()
    for a in (drawing.ctrl, drawing.colours, drawing.panel_ptr, drawing.panel_start):
        h.update(np.ascontiguousarray(a).tobytes())
    h.update(json.dumps([int(drawing.g), int(drawing.s_per_panel), [list(map(float, v[:4])) + [int(v[4]), int(v[5])]
                                                                     for v in viewports],
                         list(map(int, leaf_sizes)), list(map(int, p_inners)), list(map(int, eval_tiles)),
                         int(p), float(tol), float(gmres_tol), gpu]).encode())
    return h.hexdigest()


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def autotune(drawing, viewports, leaf_sizes=(32, 48, 64, 96, 128), p_inners=(10, 12, 14),
             eval_tiles=(0, 1, 2, 3), p=24, tol=1e-5, repeats=2, gmres_tol=1e-10, cache=True):
    """(best options dict or None, table of row dicts, True if from the cache).
    Rows that fail, do not converge or miss tol are kept with their values;
    the best is the fastest of the others."""
    import torch

    from . import Context
    gpu = torch.cuda.get_device_name() if torch.cuda.is_available() else "none"
    key = cache_key(drawing, viewports, leaf_sizes, p_inners, eval_tiles, p, tol, gmres_tol, gpu)
    path = cache_path()
    if cache:
        hit = _load(path).get(key)
        if hit is not None:
            return hit["best"], hit["table"], True
    ctx = Context(form="fmm32", g=drawing.g, s_per_panel=drawing.s_per_panel, p=p, gmres_tol=gmres_tol,
                  gmres_restart=200, gmres_max_iter=3000)
    ctx.build_drawing(drawing)
    idx, table = ctx.autotune(viewports, leaf_sizes, p_inners, eval_tiles, tol=tol, repeats=repeats)
    ctx.close()
    best = None
    if idx >= 0:
        r = table[idx]
        best = dict(p=p, leaf_size=r["leaf_size"], p_inner=r["p_inner"], eval_tile=r["eval_tile"],
                    gmres_tol=gmres_tol)
    if cache:
        os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
        data = _load(path)
        data[key] = {"best": best, "table": table, "gpu": gpu}
        tmp = f"{path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(data, f)
        os.replace(tmp, path)
    return best, table, False
