"""Pins of the FP64 oracle against things other than itself.

Each test ties one oracle function to the paper or to mathematics: library
routines for textbook special cases (Gauss-Legendre rules, Legendre values,
adaptive quadrature of the integrands), closed forms (Eq. 52), the jump
relations (App. C), Gauss's lemma for a straight-edged polygon, exact
harmonic interiors and Green's representation formula for closed curves,
brute-force assembly of tiny systems, rigid-motion invariance, and agreement
of two solution routes (LU and GMRES).  A plausible mistake in the oracle
(a dropped term, a wrong sign or normal, a transposed interpolation matrix,
a wrong index) fails at least one of them.
"""
import numpy as np
import pytest
from scipy import integrate

from dc_synth import Drawing, drawing_by_name

KAPPA = 0.5522847498307936   # quarter-circle cubic handle length


# ------------------------------------------------------------ helpers ----
def circle_drawing(R=0.3, c=(0.5, 0.5), panels=4, g=8, nseg=40):
    """Four cubic quarter arcs, counter-clockwise (right-hand normal points
    outward, so the "+" side is the outside)."""
    ctrl = []
    for q in range(4):
        a0, a1 = q * np.pi / 2, (q + 1) * np.pi / 2
        p0 = np.array([np.cos(a0), np.sin(a0)])
        p3 = np.array([np.cos(a1), np.sin(a1)])
        t0 = np.array([-np.sin(a0), np.cos(a0)])
        t3 = np.array([-np.sin(a1), np.cos(a1)])
        ctrl.append(np.array(c) + R * np.array([p0, p0 + KAPPA * t0, p3 - KAPPA * t3, p3]))
    ptr = np.arange(5, dtype=np.int32) * panels
    start = np.tile(np.arange(panels) / panels, 4)
    return Drawing("circle", np.array(ctrl), np.zeros(4, bool), np.zeros((4, 2, 2, 3)),
                   ptr, start, g=g, s_per_panel=nseg)


def square_drawing(lo=0.2, hi=0.7, panels=3, g=4, nseg=20):
    """Counter-clockwise square of four straight cubics (control points
    evenly spaced on each edge, so arc length equals chord length)."""
    corners = np.array([[lo, lo], [hi, lo], [hi, hi], [lo, hi]])
    ctrl = []
    for i in range(4):
        a, b = corners[i], corners[(i + 1) % 4]
        ctrl.append(np.array([a + (b - a) * k / 3.0 for k in range(4)]))
    ptr = np.arange(5, dtype=np.int32) * panels
    start = np.tile(np.arange(panels) / panels, 4)
    return Drawing("square", np.array(ctrl), np.zeros(4, bool), np.zeros((4, 2, 2, 3)),
                   ptr, start, g=g, s_per_panel=nseg)


def bezier_normal(c, t):
    u = 1 - t
    d = 3 * (u * u * (c[1] - c[0]) + 2 * t * u * (c[2] - c[1]) + t * t * (c[3] - c[2]))
    d = d / np.linalg.norm(d)
    return np.array([d[1], -d[0]])


def G_point(p, q):
    return -np.log(np.hypot(p[0] - q[0], p[1] - q[1])) / (2 * np.pi)


def F_point(p, q, n):
    d = np.asarray(p) - np.asarray(q)
    return -(d @ n) / (2 * np.pi * (d @ d))


# -------------------------------------------------- Legendre (Eq. 8-11) --
@pytest.mark.parametrize("n", [1, 2, 3, 4, 7, 8, 16, 20, 33])
def test_gauss_legendre_matches_library(oracle_mod, n):
    x, w = oracle_mod.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(x, xr, rtol=0, atol=2e-15)
    np.testing.assert_allclose(w, wr, rtol=1e-13, atol=1e-15)


def test_legendre_values_match_library(oracle_mod):
    for x in [-1.0, -0.3, 0.0, 0.71, 1.0]:
        P = oracle_mod.legendre_values(12, x)
        ref = [np.polynomial.legendre.legval(x, np.eye(12)[k]) for k in range(12)]
        np.testing.assert_allclose(P, ref, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("g,nseg", [(4, 20), (8, 40), (16, 80), (3, 10)])
def test_interpolation_reproduces_polynomials(oracle_mod, g, nseg):
    """Pbar Pring^-1 maps node values of any degree < g polynomial to its
    values at the arc-length midpoints exactly (Eq. 10-11)."""
    lam = oracle_mod.interpolation_matrix(g, nseg)
    x, _ = oracle_mod.gauss_legendre(g)
    xbar = -1 + (2 * np.arange(nseg) + 1) / nseg
    rng = np.random.default_rng(1)
    for deg in range(g):
        coef = rng.standard_normal(deg + 1)
        np.testing.assert_allclose(lam @ np.polyval(coef, x), np.polyval(coef, xbar),
                                   atol=1e-12 * max(1, np.abs(coef).sum()))
    # Lagrange basis: row sums are 1, matrix is not its own transpose
    np.testing.assert_allclose(lam.sum(1), 1.0, atol=1e-13)


# ------------------------------------------------------ Bezier (App. B) --
def test_arclength_matches_adaptive_quadrature(oracle_mod):
    d = drawing_by_name("closed4")
    for c in d.ctrl:
        def speed(t):
            u = 1 - t
            dd = 3 * (u * u * (c[1] - c[0]) + 2 * t * u * (c[2] - c[1]) + t * t * (c[3] - c[2]))
            return np.hypot(*dd)
        for t in [0.3, 0.77, 1.0]:
            ref, err = integrate.quad(speed, 0, t, epsabs=1e-15, epsrel=1e-14, limit=200)
            assert abs(oracle_mod.arclen(c, t) - ref) <= 1e-13 * max(ref, 1e-3)


def test_arclength_of_uniform_line_is_linear(oracle_mod):
    a, b = np.array([0.1, 0.2]), np.array([0.8, 0.5])
    c = np.array([a + (b - a) * k / 3 for k in range(4)])   # B(t) = a + t (b - a)
    L = np.linalg.norm(b - a)
    assert abs(oracle_mod.arclen(c, 1.0) - L) < 1e-15
    for s in [0.0, 0.1, 0.37, 0.5, 0.7]:
        assert abs(oracle_mod.t_of_s(c, s * L, L) - s) < 1e-14


def test_t_of_s_inverts_arclength(oracle_mod):
    d = drawing_by_name("closed4")
    for c in d.ctrl:
        L = oracle_mod.arclen(c, 1.0)
        for frac in [0.013, 0.25, 0.5, 0.9, 0.999]:
            t = oracle_mod.t_of_s(c, frac * L, L)
            assert abs(oracle_mod.arclen(c, t) - frac * L) <= 2e-15 * L


# ------------------------------------------------ closed forms (App. D) --
def _quad_GF(p1, p2, q):
    p1, p2, q = map(np.asarray, (p1, p2, q))
    d = p2 - p1
    c = np.linalg.norm(d)
    n = np.array([d[1], -d[0]]) / c
    gi = integrate.quad(lambda s: G_point(p1 + s * d / c, q), 0, c,
                        epsabs=1e-15, epsrel=1e-13, limit=400)[0]
    fi = integrate.quad(lambda s: F_point(p1 + s * d / c, q, n), 0, c,
                        epsabs=1e-15, epsrel=1e-13, limit=400)[0]
    return gi, fi


def test_segment_integrals_match_quadrature(oracle_mod):
    rng = np.random.default_rng(2)
    for _ in range(40):
        p1, p2 = rng.uniform(0, 1, 2), rng.uniform(0, 1, 2)
        dist = 10 ** rng.uniform(-3, 0.3)
        mid = 0.5 * (p1 + p2)
        q = mid + dist * rng.standard_normal(2)
        G, F = oracle_mod.segment_GF(p1, p2, q)
        gr, fr = _quad_GF(p1, p2, q)
        assert abs(G - gr) < 1e-12
        assert abs(F - fr) < 1e-11


def test_singular_G_is_eq52_and_F_vanishes(oracle_mod):
    """Target on the segment: int G = (c - e1 log e1 - e2 log e2)/2pi (Eq. 52)
    against quadrature with the log singularity marked; int F = 0 (Eq. 53)."""
    p1, p2 = np.array([0.1, 0.3]), np.array([0.6, 0.5])
    d = p2 - p1
    c = np.linalg.norm(d)
    for ts in [0.5, 0.2, 0.93]:
        q = p1 + ts * d
        G, F = oracle_mod.segment_GF(p1, p2, q, singular=True)
        ref = integrate.quad(lambda s: G_point(p1 + s * d / c, q), 0, c,
                             points=[ts * c], epsabs=1e-15, epsrel=1e-13, limit=400)[0]
        assert abs(G - ref) < 1e-13
        assert F == 0.0
        e1, e2 = ts * c, (1 - ts) * c
        assert abs(G - (c - e1 * np.log(e1) - e2 * np.log(e2)) / (2 * np.pi)) < 1e-15


def test_jump_relations(oracle_mod):
    """Approaching the segment interior from the side the normal points to,
    int F -> +1/2; from the other side -> -1/2; int G is continuous
    (App. C and Eq. 21)."""
    p1, p2 = np.array([0.0, 0.0]), np.array([1.0, 0.0])
    n = np.array([0.0, -1.0])                  # right-hand normal of +x travel
    q0 = np.array([0.4, 0.0])
    Gs, _ = oracle_mod.segment_GF(p1, p2, q0, singular=True)
    for delta in [1e-7, 1e-9]:
        Gp, Fp = oracle_mod.segment_GF(p1, p2, q0 + delta * n)
        Gm, Fm = oracle_mod.segment_GF(p1, p2, q0 - delta * n)
        assert abs(Fp - 0.5) < 1e-6 and abs(Fm + 0.5) < 1e-6
        assert abs(Gp - Gs) < 1e-6 and abs(Gm - Gs) < 1e-6


# ------------------------------------------------ whole-operator pins ----
def test_gauss_lemma_straight_polygon(oracle_mod):
    """Constant mu = 1 on a counter-clockwise polygon: the double layer is -1
    inside, 0 outside, and its principal value at boundary nodes is -1/2.
    Arc length = chord length on straight edges, so this is exact."""
    d = square_drawing()
    disc = oracle_mod.discretise(d)
    np.testing.assert_allclose(disc.seg_w, 1.0, atol=1e-13)
    N = disc.n_nodes
    zero, one = np.zeros((N, 3)), np.ones((N, 3))
    inside = np.array([[0.45, 0.45], [0.21, 0.6], [0.69, 0.21]])
    outside = np.array([[0.1, 0.1], [0.95, 0.5], [0.45, 0.71], [3.0, -2.0]])
    u_in = oracle_mod.layer_potential(disc, inside, zero, one)
    u_out = oracle_mod.layer_potential(disc, outside, zero, one)
    np.testing.assert_allclose(u_in, -1.0, atol=1e-13)
    np.testing.assert_allclose(u_out, 0.0, atol=1e-13)
    _, AF = oracle_mod.hybrid_rows(disc)
    np.testing.assert_allclose(AF @ np.ones(N), -0.5, atol=1e-13)


def test_brute_force_tiny_system(oracle_mod):
    """One straight curve, one panel, g = 2, nseg = 3: every entry of G_H and
    F_H from quadrature of the integrand against the Lagrange basis."""
    a, b = np.array([0.2, 0.1]), np.array([0.9, 0.6])
    ctrl = np.array([[a + (b - a) * k / 3 for k in range(4)]])
    d = Drawing("tiny", ctrl, np.zeros(1, bool), np.zeros((1, 2, 2, 3)),
                np.array([0, 1], np.int32), np.array([0.0]), g=2, s_per_panel=3)
    disc = oracle_mod.discretise(d)
    AG, AF = oracle_mod.hybrid_rows(disc)
    L = np.linalg.norm(b - a)
    xg = np.array([-1, 1]) / np.sqrt(3.0)
    nodes = a + np.outer((xg + 1) / 2, b - a)
    np.testing.assert_allclose(disc.node_xy, nodes, atol=1e-15)
    def lag(m, x):          # Lagrange basis at the two nodes
        o = 1 - m
        return (x - xg[o]) / (xg[m] - xg[o])
    for i in range(2):
        for m in range(2):
            ref = 0.0
            for k in range(3):
                xbar = -1 + (2 * k + 1) / 3
                lo, hi = k * L / 3, (k + 1) * L / 3
                s_node = (xg[i] + 1) / 2 * L
                pts = [s_node] if lo < s_node < hi else None
                gk = integrate.quad(lambda s: G_point(a + s * (b - a) / L, nodes[i]), lo, hi,
                                    points=pts, epsabs=1e-15, epsrel=1e-13, limit=200)[0]
                ref += gk * lag(m, xbar)
            assert abs(AG[i, m] - ref) < 1e-13
    np.testing.assert_allclose(AF, 0.0, atol=1e-15)   # collinear: F vanishes


def _harmonic(P, centre=(0.5, 0.5), x0=(1.2, 0.9)):
    return (P[:, 0] - centre[0]) ** 2 - (P[:, 1] - centre[1]) ** 2 + \
        0.3 * np.log(np.hypot(P[:, 0] - x0[0], P[:, 1] - x0[1]))


def _harmonic_grad(P, centre=(0.5, 0.5), x0=(1.2, 0.9)):
    d = P - np.asarray(x0)
    r2 = (d ** 2).sum(1)
    return np.stack([2 * (P[:, 0] - centre[0]) + 0.3 * d[:, 0] / r2,
                     -2 * (P[:, 1] - centre[1]) + 0.3 * d[:, 1] / r2], 1)


def _interior_points(n=150, seed=0):
    rng = np.random.default_rng(seed)
    ang = rng.uniform(0, 2 * np.pi, n)
    rad = 0.25 * np.sqrt(rng.uniform(0, 1, n))
    return np.stack([0.5 + rad * np.cos(ang), 0.5 + rad * np.sin(ang)], 1)


def test_harmonic_interior_converges(oracle_mod):
    """u+ = u- = f with f harmonic (Re z^2 plus an outside point source, the
    paper's own test of Sec. 4 figure): the interior field is f exactly, so
    the discrete error must be small and shrink with refinement."""
    P = _interior_points()
    errs = []
    for panels in (4, 8):
        d = circle_drawing(panels=panels, g=16, nseg=80)
        disc = oracle_mod.discretise(d)
        U = np.repeat(_harmonic(disc.node_xy)[:, None], 3, 1)
        sol = oracle_mod.solve_values(disc, U, U)
        u = oracle_mod.layer_potential(disc, P, sol.sigma, sol.mu)
        errs.append(np.abs(u[:, 0] - _harmonic(P)).max())
    assert errs[0] < 2e-7
    assert errs[1] < 0.5 * errs[0]


def test_green_representation_two_sided(oracle_mod):
    """u+ = 0 outside, u- = f inside: Green's third identity gives the field
    f inside, 0 outside, and sigma = df/dn (outward), mu = -f.  Pins the
    right-hand side b = (u+ + u-)/2 - F_H mu and the sign of the F term."""
    d = circle_drawing(panels=4, g=16, nseg=80)
    disc = oracle_mod.discretise(d)
    fN = _harmonic(disc.node_xy)
    U = np.repeat(fN[:, None], 3, 1)
    sol = oracle_mod.solve_values(disc, np.zeros_like(U), U)
    P = _interior_points()
    ang = np.linspace(0, 2 * np.pi, 60, endpoint=False)
    Q = np.stack([0.5 + 0.45 * np.cos(ang), 0.5 + 0.45 * np.sin(ang)], 1)
    uin = oracle_mod.layer_potential(disc, P, sol.sigma, sol.mu)
    uout = oracle_mod.layer_potential(disc, Q, sol.sigma, sol.mu)
    assert np.abs(uin[:, 0] - _harmonic(P)).max() < 5e-7
    assert np.abs(uout[:, 0]).max() < 5e-7
    n = np.array([bezier_normal(d.ctrl[ci], t) for ci, t in zip(disc.node_curve, disc.node_t)])
    dfdn = (_harmonic_grad(disc.node_xy) * n).sum(1)
    assert np.abs(sol.sigma[:, 0] - dfdn).max() < 2e-4 * np.abs(dfdn).max()


def test_lu_and_gmres_agree(oracle_mod):
    d = drawing_by_name("closed4")
    disc = oracle_mod.discretise(d)
    sol = oracle_mod.solve(d, disc, keep_matrix=True)
    for ch in range(3):
        x, it, rr = oracle_mod.gmres(lambda v: sol.AG @ v, sol.b[:, ch],
                                     np.ones(disc.n_nodes), 1e-13, restart=1024)
        assert rr <= 1e-13
        assert np.abs(x - sol.sigma[:, ch]).max() <= 1e-10 * np.abs(sol.sigma[:, ch]).max()


def test_rigid_motion_invariance(oracle_mod):
    """Rotating and translating the drawing moves the field with it: the
    densities are unchanged and pixel values follow the points."""
    d = drawing_by_name("mixed16")
    ang, shift = 0.7, np.array([0.31, -0.17])
    R = np.array([[np.cos(ang), -np.sin(ang)], [np.sin(ang), np.cos(ang)]])
    d2 = Drawing("moved", d.ctrl @ R.T + shift, d.closed, d.colours, d.panel_ptr,
                 d.panel_start, g=d.g, s_per_panel=d.s_per_panel)
    disc, disc2 = oracle_mod.discretise(d), oracle_mod.discretise(d2)
    s1, s2 = oracle_mod.solve(d, disc), oracle_mod.solve(d2, disc2)
    scale = np.abs(s1.sigma).max()
    assert np.abs(s1.sigma - s2.sigma).max() <= 1e-9 * scale
    P = np.random.default_rng(3).uniform(0, 1, (64, 2))
    u1 = oracle_mod.layer_potential(disc, P, s1.sigma, s1.mu)
    u2 = oracle_mod.layer_potential(disc2, P @ R.T + shift, s2.sigma, s2.mu)
    np.testing.assert_allclose(u1, u2, atol=1e-9)


def test_quantise_rule(oracle_mod):
    u = np.array([-0.1, 0.0, 0.5 / 255, 0.49999 / 255, 0.5, 1.0, 1.7])
    np.testing.assert_array_equal(oracle_mod.quantise(u), [0, 0, 1, 0, 128, 255, 255])


def test_arc_length_weighting(oracle_mod):
    """App. A: each segment integral is weighted so the total integration
    length is the curve's true arc length, whatever the segment count.  A
    unit density on a half circle seen from far away gives L G(x, c) to
    leading order, with L = pi R; on 2 segments the chord sum is 10% short."""
    R = 0.3
    half = circle_drawing(R=R, panels=1, g=2, nseg=2)
    ctrl = half.ctrl[:2]
    x = np.array([1e4, 3e3])
    vals = []
    for nseg in (2, 3, 40):
        d = Drawing("half", ctrl, np.zeros(2, bool), np.zeros((2, 2, 2, 3)),
                    np.array([0, 1, 2], np.int32), np.array([0.0, 0.0]),
                    g=2, s_per_panel=nseg)
        disc = oracle_mod.discretise(d)
        np.testing.assert_allclose(disc.curve_len.sum(), np.pi * R, rtol=3e-4)  # cubic arcs
        ones = np.ones((disc.n_nodes, 3))
        u = oracle_mod.layer_potential(disc, x[None], ones, 0 * ones)[0, 0]
        vals.append(u)
        lead = disc.curve_len.sum() * G_point(x, (0.5, 0.5))
        assert abs(u - lead) < 1e-4 * abs(lead)
        # the row assembly weights segments the same way as the direct sum
        AG, _ = oracle_mod.hybrid_rows(disc)
        un = oracle_mod.layer_potential(disc, disc.node_xy, ones, 0 * ones,
                                        disc.node_seg, disc.node_seg2)[:, 0]
        np.testing.assert_allclose(AG.sum(1), un, rtol=1e-13, atol=1e-15)
    assert abs(vals[0] - vals[2]) < 1e-4 * abs(vals[2])


def test_layer_potential_brute_force_curved(oracle_mod):
    """Tiny curved case computed independently here: vertices at equal arc
    length (scipy quad + brentq), Lagrange interpolation of the node values
    to segment midpoints, both kernels integrated over each chord by
    quadrature and weighted by arc / chord (App. A)."""
    from scipy.optimize import brentq
    c = circle_drawing(R=0.3, panels=1).ctrl[1]          # one quarter arc
    g, nseg = 3, 4
    d = Drawing("arc", c[None], np.zeros(1, bool), np.zeros((1, 2, 2, 3)),
                np.array([0, 1], np.int32), np.array([0.0]), g=g, s_per_panel=nseg)
    disc = oracle_mod.discretise(d)

    def B(t):
        u = 1 - t
        return u ** 3 * c[0] + 3 * t * u * u * c[1] + 3 * t * t * u * c[2] + t ** 3 * c[3]

    def speed(t):
        u = 1 - t
        return np.hypot(*(3 * (u * u * (c[1] - c[0]) + 2 * t * u * (c[2] - c[1]) + t * t * (c[3] - c[2]))))

    def L(t):
        return integrate.quad(speed, 0, t, epsabs=1e-15, epsrel=1e-14)[0]

    Ltot = L(1.0)
    ts = [0.0] + [brentq(lambda t: L(t) - k * Ltot / nseg, 0, 1, xtol=1e-15)
                  for k in range(1, nseg)] + [1.0]
    V = np.array([B(t) for t in ts])
    np.testing.assert_allclose(disc.seg_xy[:, :2], V[:-1], atol=1e-13)
    xg, _ = np.polynomial.legendre.leggauss(g)
    xbar = -1 + (2 * np.arange(nseg) + 1) / nseg
    lag = np.array([[np.prod([(xb - xg[o]) / (xg[m] - xg[o]) for o in range(g) if o != m])
                     for m in range(g)] for xb in xbar])
    rng = np.random.default_rng(5)
    sig, mu = rng.standard_normal((g, 3)), rng.standard_normal((g, 3))
    targets = np.array([[0.5, 0.5], [0.7, 0.95], [0.2, 0.9], [0.45, 0.83]])
    u = oracle_mod.layer_potential(disc, targets, sig, mu)
    for i, q in enumerate(targets):
        ref = np.zeros(3)
        for k in range(nseg):
            p1, p2 = V[k], V[k + 1]
            chord = np.linalg.norm(p2 - p1)
            w = (Ltot / nseg) / chord
            gk, fk = _quad_GF(p1, p2, q)
            ref += w * (gk * (lag[k] @ sig) + fk * (lag[k] @ mu))
        np.testing.assert_allclose(u[i], ref, atol=1e-11)
    # the F rows of the hybrid operator weight segments like the direct sum
    _, AF = oracle_mod.hybrid_rows(disc)
    ones = np.ones((disc.n_nodes, 3))
    un = oracle_mod.layer_potential(disc, disc.node_xy, 0 * ones, ones,
                                    disc.node_seg, disc.node_seg2)[:, 0]
    np.testing.assert_allclose(AF.sum(1), un, rtol=1e-12, atol=1e-15)


# ----------------------------------------- boundary colours and pixels ----
def test_boundary_colours_straight_line_hand_values(oracle_mod):
    """One straight cubic with evenly spaced control points (t equals the
    arc-length fraction), one panel of g = 3 nodes: the middle node sits at
    t = 1/2, so u+ and u- there are the means of each side's end colours,
    worked out by hand.  A swapped side or end changes these numbers."""
    a, b = np.array([0.2, 0.5]), np.array([0.8, 0.5])
    ctrl = np.array([[a + (b - a) * k / 3 for k in range(4)]])
    col = np.zeros((1, 2, 2, 3))
    col[0, 0, 0] = [0.2, 0.4, 0.6]      # "+" side (right of travel), t = 0
    col[0, 0, 1] = [0.6, 0.0, 1.0]      # "+" side, t = 1
    col[0, 1, 0] = [1.0, 0.9, 0.1]      # "-" side, t = 0
    col[0, 1, 1] = [0.0, 0.3, 0.7]      # "-" side, t = 1
    d = Drawing("line", ctrl, np.zeros(1, bool), col, np.array([0, 1], np.int32),
                np.array([0.0]), g=3, s_per_panel=15)
    disc = oracle_mod.discretise(d)
    up, um = oracle_mod.boundary_values(d, disc)
    np.testing.assert_allclose(disc.node_xy[1], [0.5, 0.5], atol=1e-15)
    np.testing.assert_allclose(up[1], [0.4, 0.2, 0.8], atol=1e-14)
    np.testing.assert_allclose(um[1], [0.5, 0.6, 0.4], atol=1e-14)
    # first node: Gauss-Legendre root -sqrt(3/5) maps to t = (1 - sqrt(3/5)) / 2
    t0 = (1.0 - np.sqrt(0.6)) / 2.0
    np.testing.assert_allclose(up[0], [0.2 + 0.4 * t0, 0.4 - 0.4 * t0, 0.6 + 0.4 * t0], atol=1e-14)


def _linear_field(P):
    A = np.array([[0.8, -0.3, 0.1], [0.2, 0.5, 0.05], [-0.4, 0.9, 0.6]])
    return np.atleast_2d(P) @ A[:, :2].T + A[:, 2]


def test_boundary_colours_side_and_end_by_harmonic_interior(oracle_mod):
    """A counter-clockwise square (straight edges, so the polyline is exact)
    whose inside ("-", left of travel) colours are a linear function f at the
    corners: linear in t along each edge, this is f itself on the boundary,
    so the interior field is f (Dirichlet problem, Sec. 3), converging with
    refinement.  The outside ("+") colour is an unrelated constant 0.9.
    Reading the sides or the ends the other way round leaves O(0.1) errors."""
    corners = np.array([[0.2, 0.2], [0.7, 0.2], [0.7, 0.7], [0.2, 0.7]])
    P = np.random.default_rng(1).uniform(0.3, 0.6, (100, 2))
    errs = []
    for panels, g, nseg in ((4, 8, 40), (8, 16, 80)):
        d = square_drawing(panels=panels, g=g, nseg=nseg)
        col = np.full((4, 2, 2, 3), 0.9)
        for i in range(4):
            col[i, 1, 0] = _linear_field(corners[i])[0]
            col[i, 1, 1] = _linear_field(corners[(i + 1) % 4])[0]
        d.colours = col
        disc = oracle_mod.discretise(d)
        sol = oracle_mod.solve(d, disc)
        u = oracle_mod.layer_potential(disc, P, sol.sigma, sol.mu)
        errs.append(np.abs(u - _linear_field(P)).max())
    assert errs[0] < 3e-6 and errs[1] < 1e-8, errs


def test_pixel_centres_hand_values(oracle_mod):
    """Pixel (r, c) of a w x h grid over [x0, x1] x [y0, y1] has its centre at
    (x0 + (c + 1/2) dx, y0 + (r + 1/2) dy), rows counted from y0 (Alg. 4's
    pixel grid, row 0 at the bottom)."""
    np.testing.assert_allclose(oracle_mod.pixel_centres((0, 0, 1, 1), 2, 1),
                               [[0.25, 0.5], [0.75, 0.5]], atol=0)
    np.testing.assert_allclose(oracle_mod.pixel_centres((0, 0, 1, 1), 1, 2),
                               [[0.5, 0.25], [0.5, 0.75]], atol=0)
    # 3 x 2 grid over [1, 4] x [2, 6]: dx = 1, dy = 2
    np.testing.assert_allclose(oracle_mod.pixel_centres((1, 2, 4, 6), 3, 2, [0, 2, 4, 5]),
                               [[1.5, 3.0], [3.5, 3.0], [2.5, 5.0], [3.5, 5.0]], atol=0)
