"""The quadtree's clipping of segments into pieces and its lists 1-4 on the
device (tree_gpu.cu) against the host construction over the same segments
(dc_aux_tree_compare): identical cells (levels, parents, children, grid
positions), identical pieces per leaf in the same order, identical lists
entry for entry, and piece endpoints
equal up to the last bit (the host compiler may contract a product and a sum
into one FMA); on the bench drawing, a drawing with segments along the
cells' midlines (ties at every level), and the 2000-curve drawing."""
import numpy as np
import pytest

from dc_synth import Drawing, drawing_by_name

pytestmark = pytest.mark.gpu


def grid_lines():
    """Horizontal and vertical lines on dyadic positions: every split puts
    pieces exactly on a midline."""
    segs = []
    for k in range(1, 8):
        y = k / 8
        segs.append(((0.0625, y), (0.9375, y)))
        segs.append(((y, 0.0625), (y, 0.9375)))
    ctrl = np.array([[np.asarray(p) + (np.asarray(q) - np.asarray(p)) * i / 3 for i in range(4)] for p, q in segs])
    n = len(segs)
    ptr = np.arange(n + 1, dtype=np.int32) * 4
    start = np.tile(np.arange(4) / 4, n)
    return Drawing("grid", ctrl, np.zeros(n, bool), np.random.default_rng(0).uniform(0, 1, (n, 2, 2, 3)), ptr,
                   start, g=8, s_per_panel=40)


@pytest.mark.parametrize("name", ["mixed200", "grid", "batched2000"])
def test_device_tree_equals_host_tree(dcmod, cuda_ok, name):
    d = grid_lines() if name == "grid" else drawing_by_name(name)
    dom = (-0.5, -0.5, 1.5, 1.5) if name == "batched2000" else (0.0, 0.0, 1.0, 1.0)
    for leaf in (16, 64):
        ctx = dcmod.Context(form="fmm32", g=d.g, s_per_panel=d.s_per_panel, leaf_size=leaf, domain=dom)
        ctx.build_drawing(d)
        r = ctx.tree_compare()
        bt = ctx.build_timings()
        print(f"{name} leaf {leaf}: {r}; tree phase {bt['tree_lists']:.1f} ms")
        assert r["identical"] and r["max_xy_diff"] <= 1e-15
        assert r["pieces"] >= d.n_segments
        ctx.close()
