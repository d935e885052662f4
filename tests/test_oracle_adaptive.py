"""Pins of the adaptive-subdivision oracle (oracle/adaptive.py; Sec. 6.1,
6.3, Alg. 5-7) against numpy's Legendre series, hand values, geometry and
invariants of the local system."""
import numpy as np
from numpy.polynomial import legendre as npleg

from dc_synth import Drawing, drawing_by_name


def line_drawing(a=(0.2, 0.4), b=(0.8, 0.4), starts=(0.0,), g=6, nseg=30):
    a, b = np.asarray(a, float), np.asarray(b, float)
    ctrl = np.array([[a + (b - a) * k / 3 for k in range(4)]])
    return Drawing("line", ctrl, np.zeros(1, bool), np.zeros((1, 2, 2, 3)),
                   np.array([0, len(starts)], np.int32), np.asarray(starts, float), g=g, s_per_panel=nseg)


def test_top_coefficient_is_the_highest_legendre_coefficient(oracle_mod):
    """Node values of a known Legendre series (numpy's legval at numpy's
    Gauss-Legendre nodes): Alg. 5's test value is |c_{g-1}| of the largest
    channel."""
    from oracle import adaptive as A
    d = drawing_by_name("closed4")
    disc = oracle_mod.discretise(d)
    g = disc.g
    x, _ = npleg.leggauss(g)
    rng = np.random.default_rng(3)
    coef = rng.standard_normal((disc.n_panels, g, 3))
    sig = np.stack([np.stack([npleg.legval(x, coef[p, :, c]) for c in range(3)], 1)
                    for p in range(disc.n_panels)]).reshape(-1, 3)
    top = A.top_coefficient(disc, sig)
    np.testing.assert_allclose(top, np.abs(coef[:, g - 1, :]).max(axis=1), rtol=1e-9)


def test_subdivide_hand_values(oracle_mod):
    """Panels [0, 1/2) and [1/2, 1) of one curve; only the second splits:
    the refined starts are 0, 1/2, 3/4 (halves in arc-length fraction)."""
    from oracle import adaptive as A
    d = line_drawing(starts=(0.0, 0.5), g=4, nseg=20)
    disc = oracle_mod.discretise(d)
    g = disc.g
    x, _ = npleg.leggauss(g)
    sig = np.zeros((2 * g, 3))
    sig[g:, 0] = npleg.legval(x, [0, 0, 0, 5.0])      # panel 1: top coefficient 5
    sig[:g, 1] = npleg.legval(x, [1.0, 0, 0, 0.5])    # panel 0: top coefficient 0.5
    d2, split, pmap = A.subdivide(d, disc, sig, eps_coef=1.0, eps_len=0.0)
    assert split.tolist() == [False, True]
    np.testing.assert_array_equal(d2.panel_start, [0.0, 0.5, 0.75])
    np.testing.assert_array_equal(d2.panel_ptr, [0, 3])
    assert pmap.tolist() == [[0, 0], [1, 1], [1, 2]]
    # the length floor epsilon_1 keeps a short panel whole
    L = A.panel_lengths(disc)
    np.testing.assert_allclose(L, [0.3, 0.3], rtol=1e-13)
    _, split2, _ = A.subdivide(d, disc, sig, eps_coef=1.0, eps_len=0.31)
    assert not split2.any()


def test_warm_start_reproduces_polynomial_densities(oracle_mod):
    """A density that is a polynomial of degree < g in arc length is
    reproduced exactly at the nodes of the halves (Sec. 6.1 warm start); on a
    straight line the node position is linear in arc length, so the expected
    value comes from the new node's position."""
    from oracle import adaptive as A
    d = line_drawing(starts=(0.0,), g=5, nseg=25)
    disc = oracle_mod.discretise(d)
    a, b = np.array([0.2, 0.4]), np.array([0.8, 0.4])

    def f(P):      # polynomial of degree 4 in the arc-length coordinate
        s = (P[:, 0] - a[0]) / (b[0] - a[0]) * 2.0 - 1.0
        return np.stack([1 + s ** 4, s - 2 * s ** 3, 0.5 * s ** 2], 1)

    sig = f(disc.node_xy)
    d2, split, pmap = A.subdivide(d, disc, sig, eps_coef=0.0, eps_len=0.0)
    assert split.all()
    disc2 = oracle_mod.discretise(d2)
    s0 = A.warm_start(disc, sig, pmap)
    np.testing.assert_allclose(s0, f(disc2.node_xy), atol=1e-12)


def test_labels_near_and_far(oracle_mod):
    """Eq. 40-41: with one panel split, its halves and a close parallel curve
    are re-solved; a curve far away is not (the range of G_H 1_alpha over a
    distant panel is small, by the mean-value argument of Sec. 6.3)."""
    from oracle import adaptive as A
    segs = [((0.3, 0.5), (0.5, 0.5)), ((0.3, 0.51), (0.5, 0.51)), ((0.3, 0.95), (0.5, 0.95))]
    ctrl = np.array([[np.asarray(p) + (np.asarray(q) - np.asarray(p)) * k / 3 for k in range(4)]
                     for p, q in segs])
    d = Drawing("three", ctrl, np.zeros(3, bool), np.zeros((3, 2, 2, 3)),
                np.array([0, 1, 2, 3], np.int32), np.zeros(3), g=4, s_per_panel=20)
    disc = oracle_mod.discretise(d)
    sig = np.zeros((disc.n_nodes, 3))
    sig[:4, 0] = npleg.legval(npleg.leggauss(4)[0], [0, 0, 0, 1.0])
    d2, split, pmap = A.subdivide(d, disc, sig, eps_coef=0.5, eps_len=0.0)
    assert split.tolist() == [True, False, False]
    disc2 = oracle_mod.discretise(d2)
    AG, _ = oracle_mod.hybrid_rows(disc2)
    res = A.label_panels(disc2, AG, pmap)
    assert res.tolist() == [True, True, True, False]


def test_local_resolve_invariants(oracle_mod):
    """Sec. 6.3's local system: (1) started from the global solution of the
    refined discretisation it returns that solution; (2) with every panel
    re-solving it is the global solve; (3) on mixed16 the local solution's
    colours are closer to the global re-solve's than the unsolved warm
    start's."""
    from oracle import adaptive as A
    d = drawing_by_name("mixed16")
    disc = oracle_mod.discretise(d)
    sol = oracle_mod.solve(d, disc)
    top = np.sort(A.top_coefficient(disc, sol.sigma))
    eps = 0.5 * (top[-13] + top[-12])
    d2, split, pmap = A.subdivide(d, disc, sol.sigma, eps, 0.0)
    assert split.sum() == 12
    disc2 = oracle_mod.discretise(d2)
    AG, AF = oracle_mod.hybrid_rows(disc2)
    glob = oracle_mod.solve(d2, disc2).sigma
    s0 = A.warm_start(disc, sol.sigma, pmap)
    res = A.label_panels(disc2, AG, pmap)
    assert 12 * 2 <= res.sum() < disc2.n_panels
    back = A.local_resolve(d2, disc2, glob, res, AG, AF)
    assert np.abs(back - glob).max() <= 1e-12 * np.abs(glob).max()
    allp = A.local_resolve(d2, disc2, s0, np.ones(disc2.n_panels, bool), AG, AF)
    assert np.abs(allp - glob).max() <= 1e-12 * np.abs(glob).max()
    loc = A.local_resolve(d2, disc2, s0, res, AG, AF)
    P = np.random.default_rng(0).uniform(0, 1, (1500, 2))
    up, um = oracle_mod.boundary_values(d2, disc2)
    ug = oracle_mod.layer_potential(disc2, P, glob, up - um)
    e_loc = np.abs(oracle_mod.layer_potential(disc2, P, loc, up - um) - ug).max()
    e_warm = np.abs(oracle_mod.layer_potential(disc2, P, s0, up - um) - ug).max()
    assert e_loc < 0.5 * e_warm
