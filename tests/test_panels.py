"""The library's adaptive panel rule (dc_build_tree without panels;
dc_aux_adaptive_panels, host only) against the seeded generator's own
implementation of the same rule (dc_synth): bisect in arc-length fraction
while a panel is longer than 0.2 x its distance to the nearest other curve,
on 256-point polylines.  The two are written independently (C++ grid search
against a numpy / k-d tree search) and must agree panel for panel."""
import numpy as np
import pytest

from dc_synth import drawing_by_name


@pytest.mark.parametrize("name,kw", [("mixed200", {}), ("mixed16", dict(max_level=4))])
def test_library_panels_match_generator(dcmod, name, kw):
    d = drawing_by_name(name)
    ptr, start = dcmod.aux_adaptive_panels(d.ctrl, **kw)
    assert np.array_equal(ptr, d.panel_ptr)
    assert np.array_equal(start, d.panel_start)


def test_panel_rule_arguments(dcmod):
    d = drawing_by_name("closed4")
    with pytest.raises(dcmod.DcError):
        dcmod.aux_adaptive_panels(d.ctrl, ratio=0.0)
    ptr, start = dcmod.aux_adaptive_panels(d.ctrl, ratio=1e9, max_len=10.0, min_panels=3)
    # only the minimum count applies: every curve bisected to 4 equal panels
    assert np.array_equal(np.diff(ptr), [4, 4, 4, 4])
    np.testing.assert_array_equal(start, np.tile([0.0, 0.25, 0.5, 0.75], 4))


@pytest.mark.gpu
def test_build_tree_without_panels(dcmod, cuda_ok):
    d = drawing_by_name("mixed200")
    ctx = dcmod.Context(form="fmm32", g=d.g, s_per_panel=d.s_per_panel)
    ctx.build_curves(d.ctrl, d.colours)
    ptr, start = ctx.panels()
    assert np.array_equal(ptr, d.panel_ptr) and np.array_equal(start, d.panel_start)
    assert ctx.sizes().n_nodes == d.n_nodes
    ctx.close()
