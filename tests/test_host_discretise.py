"""The library's host discretisation (dc_aux_discretise: the first step of
dc_build_tree, Sec. 4.2 and App. A-B) against the oracle's, on the CPU:
node positions and segment end points to 1e-13, node parameters to 1e-12,
boundary colours to 1e-13 and the arc / chord weights to 1e-9 relative (a
chord of 1e-5 turns a 1e-15 shift of an end point into 1e-10 of its
weight), on the three drawings the GPU tests use.  Invariants that hold
bit for bit: neighbouring panels of a curve share their end point,
consecutive segments of a panel share theirs, and a closed curve's last
segment ends where its first begins.  A curve of zero length is refused."""
import numpy as np
import pytest

from dc_synth import drawing_by_name


@pytest.mark.parametrize("name", ["closed4", "mixed16", "mixed200"])
def test_host_discretisation_matches_oracle(dcmod, oracle_mod, name):
    O = oracle_mod
    d = drawing_by_name(name)
    got = dcmod.aux_discretise(d.ctrl, d.panel_ptr, d.panel_start, d.colours, d.g, d.s_per_panel)
    disc = O.discretise(d)
    up, um = O.boundary_values(d, disc)
    np.testing.assert_allclose(got["node_xy"], disc.node_xy.reshape(-1, 2), rtol=0, atol=1e-13)
    np.testing.assert_allclose(got["seg_xy"], disc.seg_xy.reshape(-1, 4), rtol=0, atol=1e-13)
    np.testing.assert_allclose(got["node_t"], disc.node_t, rtol=0, atol=1e-12)
    np.testing.assert_allclose(got["seg_w"], disc.seg_w, rtol=1e-9, atol=0)
    np.testing.assert_allclose(got["u_plus"], up, rtol=0, atol=1e-13)
    np.testing.assert_allclose(got["u_minus"], um, rtol=0, atol=1e-13)
    s = d.s_per_panel
    seg = got["seg_xy"].reshape(-1, s, 4)
    # consecutive segments of a panel share their end point
    assert np.array_equal(seg[:, 1:, 0:2], seg[:, :-1, 2:4])
    # neighbouring panels of a curve share theirs; closed curves close
    for c in range(d.n_curves):
        p0, p1 = int(d.panel_ptr[c]), int(d.panel_ptr[c + 1])
        for p in range(p0, p1 - 1):
            assert np.array_equal(seg[p, -1, 2:4], seg[p + 1, 0, 0:2]), (c, p)
        if d.closed[c]:
            np.testing.assert_allclose(seg[p1 - 1, -1, 2:4], seg[p0, 0, 0:2], rtol=0, atol=1e-15)


def test_host_discretisation_refuses_zero_length(dcmod):
    d = drawing_by_name("closed4")
    ctrl = np.array(d.ctrl, dtype=np.float64)
    ctrl[1] = ctrl[1, 0]          # all four control points of curve 1 equal
    with pytest.raises(dcmod.DcError) as e:
        dcmod.aux_discretise(ctrl, d.panel_ptr, d.panel_start, d.colours, d.g, d.s_per_panel)
    assert e.value.status == dcmod.DC_ERR_GEOMETRY
