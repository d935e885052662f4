"""Pins of the viewport-update oracle (oracle/viewport.py; Sec. 6.2, 6.4,
Alg. 9): the e rule and the labels by hand, e = s reproducing the plain
render, the finer evaluation polyline putting the colour jump on the curve
(the purpose of Sec. 6.2's rule), and viewport-masked subdivision."""
import numpy as np

from dc_synth import Drawing, circle_loops, curve_point, curve_tangent, drawing_by_name


def lines(segs, panels=1, g=6, nseg=20):
    ctrl = np.array([[np.asarray(p) + (np.asarray(q) - np.asarray(p)) * k / 3 for k in range(4)]
                     for p, q in segs], float)
    n = len(segs)
    ptr = np.arange(n + 1, dtype=np.int32) * panels
    start = np.tile(np.arange(panels) / panels, n)
    return Drawing("lines", ctrl, np.zeros(n, bool), np.zeros((n, 2, 2, 3)), ptr, start, g=g, s_per_panel=nseg)


def test_e_rule_and_labels_by_hand(oracle_mod):
    from oracle import viewport as V
    O = oracle_mod
    d = lines([((0.1, 0.5), (0.4, 0.5)), ((0.6, 0.9), (0.9, 0.9))], panels=2)
    disc = O.discretise(d)
    vp = (0.05, 0.4, 0.5, 0.6)                      # holds the first line only
    m = V.meets_viewport(disc, vp)
    assert m.tolist() == [True, True, False, False]
    # panels of length 0.15: ceil(0.15 * 512 / 10) + 20 = ceil(7.68) + 20
    assert V.eval_segments(disc, m) == 28
    assert V.eval_segments(disc, m, unit=1.0 / 1024) == 36      # ceil(15.36) + 20
    assert V.eval_segments(disc, np.zeros(4, bool)) == 20
    # a viewport touching the second line's end point only (closed boxes)
    assert V.meets_viewport(disc, (0.9, 0.95, 1.0, 1.0)).tolist() == [False, False, False, False]
    assert V.meets_viewport(disc, (0.9, 0.9, 1.0, 1.0)).tolist() == [False, False, False, True]
    assert abs(V.pixel_size((0.0, 0.0, 2.0, 1.0), 100, 100) - 0.02) < 1e-17


def test_e_equal_s_is_the_plain_render(oracle_mod):
    from oracle import viewport as V
    O = oracle_mod
    d = drawing_by_name("mixed16")
    disc = O.discretise(d)
    sol = O.solve(d, disc)
    # a viewport that meets no panel: e = s, nothing splits
    r = V.view_update(d, sol.sigma, (2.0, 2.0, 3.0, 3.0), 64, 64, eps_coef=0.0, eps_len_px=0.0)
    assert r["e"] == d.s_per_panel and r["rounds"] == 0
    np.testing.assert_array_equal(r["disc_e"].seg_xy, disc.seg_xy)
    pix = np.arange(0, 64 * 64, 7)
    a = V.render(r["disc_e"], r["sigma"], sol.mu, (0, 0, 1, 1), 64, 64, pix)
    b = O.render(disc, sol, (0, 0, 1, 1), 64, 64, pix)
    np.testing.assert_array_equal(a, b)


def test_finer_polyline_puts_the_jump_on_the_curve(oracle_mod):
    """A disc coloured 1 inside, 0 outside (u- = 1, u+ = 0: Green's
    representation of the constant): points 2e-6 inside the curve mostly lie
    outside the s-polyline (its chords cut inside the arc by up to 1.7e-5)
    and read about 0; on the e-polyline of the rule at a fine unit (chords
    within 3e-7 of the arc) they all read about 1."""
    from oracle import viewport as V
    O = oracle_mod
    c, R = np.array([0.5, 0.5]), 0.35
    d = circle_loops([(c[0], c[1], R, True)], panels_per_arc=2, g=8, s_per_panel=40)
    d.colours[:] = 0.0
    d.colours[:, 1] = 1.0                       # the "-" (left, inside) side
    disc = O.discretise(d)
    sol = O.solve(d, disc)
    # curve points and inward normals (left of a counter-clockwise loop)
    t = np.random.default_rng(4).uniform(0.0, 1.0, 200)
    i = np.arange(200) % d.n_curves
    B = np.array([curve_point(d, int(a), float(b)) for a, b in zip(i, t)])
    T = curve_tangent(d, i, t)
    n_in = np.stack([-T[:, 1], T[:, 0]], 1) / np.linalg.norm(T, axis=1)[:, None]
    pts = B + 2e-6 * n_in
    u_s = O.layer_potential(disc, pts, sol.sigma, sol.mu)[:, 0]
    de = V.view_update(d, sol.sigma, (0, 0, 1, 1), 512, 512, 1e300, 0.0, unit=1.0 / 65536)
    assert de["e"] > 8 * d.s_per_panel
    u_e = O.layer_potential(de["disc_e"], pts, de["sigma"], sol.mu)[:, 0]
    assert np.mean(np.abs(u_s) < 0.1) > 0.5          # most read the outside colour
    assert np.all(np.abs(u_e - 1.0) < 1e-3)          # all read the inside colour


def test_view_update_splits_only_in_the_viewport(oracle_mod):
    from oracle import adaptive as A
    from oracle import viewport as V
    O = oracle_mod
    d = drawing_by_name("mixed16")
    disc = O.discretise(d)
    sol = O.solve(d, disc)
    top = A.top_coefficient(disc, sol.sigma)
    vp = (0.2, 0.2, 0.7, 0.7)
    m = V.meets_viewport(disc, vp)
    assert 10 < m.sum() < len(m)
    ts = np.sort(top[m])
    eps = float(0.5 * (ts[-4] + ts[-3]))             # three panels inside are above it
    assert (top[~m] > eps).any()                     # ... and some outside would have
    r = V.view_update(d, sol.sigma, vp, 256, 256, eps_coef=eps, eps_len_px=2.0, max_rounds=1)
    floor = 2.0 * V.pixel_size(vp, 256, 256)       # epsilon_1: two pixels
    L = A.panel_lengths(disc)
    want = int(((top > eps) & m & (L >= floor)).sum())
    assert r["rounds"] == 1 and r["n_split"] == want and 1 <= want <= 3
    # every split panel met the viewport, and panels outside keep their starts
    _, split, pmap = A.subdivide(d, disc, sol.sigma, eps, floor, mask=m)
    assert np.all(m[split])
    lab = r["labels"]
    m2 = V.meets_viewport(r["disc"], vp)
    assert np.all(lab[~m2] != 1) and np.all((lab == 0) <= ~m2)
    assert (lab == 2).sum() >= 2 * r["n_split"]
    assert r["e"] >= d.s_per_panel
