"""Quadtree (Sec. 5.1-5.2, App. E.5) on the host: every pair of leaves is
covered by exactly one of the four routes of Alg. 8, and clipping
partitions every segment.  No GPU needed."""
import numpy as np
import pytest

from dc_synth import drawing_by_name


@pytest.mark.parametrize("name,leaf", [("closed4", 16), ("closed4", 64), ("mixed16", 16),
                                       ("mixed16", 32)])
def test_routes_cover_each_leaf_pair_once(dcmod, oracle_mod, name, leaf):
    disc = oracle_mod.discretise(drawing_by_name(name))
    r = dcmod.aux_tree_check(disc.seg_xy, leaf_size=leaf)
    assert r["bad_pairs"] == 0
    assert r["clip_rel_err"] < 1e-14
    assert r["pieces"] >= disc.n_segments
    assert r["depth"] >= 3


def test_degenerate_trees(dcmod):
    # one segment: the root is a leaf
    r = dcmod.aux_tree_check(np.array([[0.1, 0.1, 0.2, 0.3]]), leaf_size=4)
    assert (r["cells"], r["leaves"], r["depth"], r["bad_pairs"]) == (1, 1, 0, 0)
    # segments along cell midlines and through corners
    seg = np.array([[0.0, 0.5, 1.0, 0.5], [0.5, 0.0, 0.5, 1.0], [0.0, 0.0, 1.0, 1.0],
                    [0.25, 0.0, 0.25, 1.0], [0.0, 0.75, 1.0, 0.75]])
    r = dcmod.aux_tree_check(seg, leaf_size=1, max_depth=6)
    assert r["bad_pairs"] == 0 and r["clip_rel_err"] < 1e-14
    # depth limit respected
    rng = np.random.default_rng(0)
    p = rng.uniform(0.4, 0.41, (200, 2))
    r = dcmod.aux_tree_check(np.hstack([p, p + 1e-4]), leaf_size=1, max_depth=7)
    assert r["depth"] <= 7 and r["bad_pairs"] == 0


def test_rejects_bad_input(dcmod):
    with pytest.raises(dcmod.DcError):
        dcmod.aux_tree_check(np.array([[0.0, np.nan, 1.0, 1.0]]))
