"""Pins of the anti-aliasing oracle (oracle/antialias.py; Sec. 7):

  * the segment / rectangle predicate agrees with Liang-Barsky clipping (a
    different algorithm) on random pairs away from ties;
  * on a polygon whose colour is exactly its indicator (straight edges, u-
    = 1 inside, u+ = 0 outside: Gauss's law makes the represented field 1
    inside and 0 outside), a pixel cut by an edge at a dyadic position gets
    the exact covered area once the cells align (5/8; 25/64 at a corner),
    a generic vertical edge stays within 2^-(m+1) of the covered fraction,
    and a diagonal edge within 3 2^-m, shrinking with m;
  * pixels that meet no segment keep their centre sample; the weights of
    every pixel sum to one.
A wrong child weight, a shifted sample centre or a wrong split rule breaks
the exact values or the bounds."""
import numpy as np

from dc_synth import Drawing

W = H = 128
VP = (0.0, 0.0, 1.0, 1.0)


def polygon_drawing(verts, g=8, nseg=40, panels=2):
    """Closed polygon of straight cubics (control points at thirds), counter-
    clockwise; inside colour ("-" side) 1, outside ("+" side) 0."""
    v = np.asarray(verts, float)
    n = len(v)
    ctrl = np.array([[v[i] + (v[(i + 1) % n] - v[i]) * k / 3 for k in range(4)] for i in range(n)])
    col = np.zeros((n, 2, 2, 3))
    col[:, 1] = 1.0
    ptr = np.arange(n + 1, dtype=np.int32) * panels
    start = np.tile(np.arange(panels) / panels, n)
    return Drawing("polygon", ctrl, np.zeros(n, bool), col, ptr, start, g=g, s_per_panel=nseg)


def _solve(O, d):
    disc = O.discretise(d)
    sol = O.solve(d, disc)
    return disc, sol


def liang_barsky(p, q, x0, y0, x1, y1):
    t0, t1 = 0.0, 1.0
    d = q - p
    for pk, qk in ((-d[0], p[0] - x0), (d[0], x1 - p[0]), (-d[1], p[1] - y0), (d[1], y1 - p[1])):
        if pk == 0.0:
            if qk < 0:
                return False
        else:
            t = qk / pk
            if pk < 0:
                t0 = max(t0, t)
            else:
                t1 = min(t1, t)
    return t0 <= t1


def test_predicate_matches_liang_barsky():
    from oracle import antialias as A
    rng = np.random.default_rng(11)
    seg = rng.uniform(0, 1, (4000, 4))
    seg[:1000, 2:] = seg[:1000, :2] + rng.uniform(-0.02, 0.02, (1000, 2))   # short ones
    agree = 0
    for _ in range(40):
        x0, y0 = rng.uniform(0, 0.9, 2)
        w, h = rng.uniform(0.001, 0.1, 2)
        m, t = A.meets(seg, x0, y0, x0 + w, y0 + h)
        ref = np.array([liang_barsky(s[:2], s[2:], x0, y0, x0 + w, y0 + h) for s in seg])
        assert np.array_equal(m[~t], ref[~t])
        agree += int(m.sum())
    assert agree > 100


def test_indicator_exact_at_dyadic_edges(oracle_mod):
    from oracle import antialias as A
    O = oracle_mod
    c, r = 40, 30
    a = (c + 3 / 8) / W          # left edge crosses pixel column c at 3/8
    b = (r + 3 / 8) / H          # bottom edge crosses pixel row r at 3/8
    d = polygon_drawing([(a, b), (0.8, b), (0.8, 0.75), (a, 0.75)])
    disc, sol = _solve(O, d)
    mid = (r + 20) * W + c       # left edge only
    corner = r * W + c           # both edges
    for m in (3, 4):
        u, edge, tie, ns = A.render_aa(disc, sol.sigma, sol.mu, VP, W, H, [mid, corner], m)
        assert edge.all()
        np.testing.assert_allclose(u[0], 5 / 8, atol=1e-10)
        np.testing.assert_allclose(u[1], 25 / 64, atol=1e-10)
    u, *_ = A.render_aa(disc, sol.sigma, sol.mu, VP, W, H, [mid], 1)
    np.testing.assert_allclose(u[0], 0.5, atol=1e-10)      # halves: centre 1/4 out, 3/4 in
    # closed sets: an edge on a pixel boundary makes both pixels edge pixels
    e = (c + 10) / W
    d3 = polygon_drawing([(e, 0.2), (0.8, 0.2), (0.8, 0.8), (e, 0.8)])
    disc3, sol3 = _solve(O, d3)
    row = 50 * W
    u, edge, tie, ns = A.render_aa(disc3, sol3.sigma, sol3.mu, VP, W, H, [row + c + 9, row + c + 10], 2)
    assert edge.all() and np.all(ns == 10)
    np.testing.assert_allclose(u[0], 0.0, atol=1e-10)
    np.testing.assert_allclose(u[1], 1.0, atol=1e-10)


def test_indicator_bounds_generic_edges(oracle_mod):
    from oracle import antialias as A
    O = oracle_mod
    c, r = 50, 60
    a = (c + 0.3) / W
    d = polygon_drawing([(a, 0.2), (0.8, 0.2), (0.8, 0.8), (a, 0.8)])
    disc, sol = _solve(O, d)
    errs = []
    for m in range(1, 6):
        u, *_ = A.render_aa(disc, sol.sigma, sol.mu, VP, W, H, [r * W + c], m)
        errs.append(np.abs(u[0] - 0.7).max())
        assert errs[-1] <= 2.0 ** -(m + 1) + 1e-10
    assert errs[-1] < errs[0]
    # a diamond: the edge x + y = s cuts a corner triangle off pixel (c, r)
    s = (c + r + 0.37) / W
    cx = 0.5
    # bottom, right, top, left; the closing edge (left -> bottom) lies on
    # x + y = s and the inside is above it
    d2 = polygon_drawing([(cx, s - cx), (cx + 0.3, s - cx + 0.3), (cx, s - cx + 0.6), (cx - 0.3, s - cx + 0.3)])
    disc2, sol2 = _solve(O, d2)
    t = 0.37
    frac = 1.0 - t * t / 2.0     # the pixel's part with x + y >= s
    px = r * W + c
    prev = None
    for m in range(1, 6):
        u, edge, tie, _ = A.render_aa(disc2, sol2.sigma, sol2.mu, VP, W, H, [px], m)
        e = np.abs(u[0] - frac).max()
        assert edge[0] and e <= 3.0 * 2.0 ** -m
        prev = e
    assert prev < 0.05


def test_plain_pixels_and_weights(oracle_mod):
    from oracle import antialias as A
    O = oracle_mod
    d = polygon_drawing([(0.3, 0.3), (0.7, 0.3), (0.7, 0.7), (0.3, 0.7)])
    disc, sol = _solve(O, d)
    pix = np.arange(0, W * H, 97)
    u, edge, tie, ns = A.render_aa(disc, sol.sigma, sol.mu, VP, W, H, pix, 3)
    plain = O.layer_potential(disc, O.pixel_centres(VP, W, H, pix), sol.sigma, sol.mu)
    assert edge.sum() > 0 and (~edge).sum() > 0
    np.testing.assert_array_equal(u[~edge], plain[~edge])
    assert np.all(ns[~edge] == 1) and np.all(ns[edge] >= 4)
    seg = np.ascontiguousarray(disc.seg_xy)
    for p in pix[edge][:10]:
        _, wts, _, _ = A.pixel_samples(seg, VP, W, H, p, 3)
        assert abs(wts.sum() - 1.0) < 1e-15
