"""Pins of the mixed Dirichlet / Neumann oracle (oracle/mixed.py; Sec. 4.3)
against closed-form harmonic functions, Green's identity and the
two-sided problem:

  * a disc with a hole (outer loop counter-clockwise, hole clockwise; four
    cubic quarter arcs each), Dirichlet data on half of the outer loop and
    Neumann data on the rest: the represented u matches the harmonic
    function inside, u on the Neumann panels matches its boundary values,
    psi on the Dirichlet panels its normal derivative, and the error falls
    at second order in the segment length (the polyline's sag);
  * outside the region the representation vanishes (Green's identity);
  * with every panel Dirichlet the block system is the two-sided problem of
    Eq. 27 with u+ = 0 outside and u- = u inside (mu = -u);
  * the constant channel is reproduced inside (Gauss's law for the double
    layer).
A dropped 1/2, a sign error in F_H, swapped masks or a wrong normal make
the interior error O(1)."""
import numpy as np
import pytest

from dc_synth import circle_loops, harmonic

HOLE = (0.45, 0.52)
LOOPS = [(0.5, 0.5, 0.35, True), (HOLE[0], HOLE[1], 0.12, False)]


def _case(O, ppa, g, s):
    d = circle_loops(LOOPS, panels_per_arc=ppa, g=g, s_per_panel=s)
    disc = O.discretise(d)
    u, psi = harmonic.boundary_data(d, disc.node_xy, disc.node_curve, disc.node_t, HOLE)
    arc = np.repeat(np.arange(d.n_curves), ppa)
    neu = arc >= 2               # outer arcs 2, 3 and the whole hole: Neumann
    return d, disc, u, psi, neu


def _points(seed=1, n=4000):
    Q = np.random.default_rng(seed).uniform(0.0, 1.0, (n, 2))
    r = np.hypot(*(Q - 0.5).T)
    h = np.hypot(*(Q - np.asarray(HOLE)).T)
    return Q, (r < 0.33) & (h > 0.14), (r > 0.37) | (h < 0.10)


def _errors(O, ppa, g, s):
    from oracle import mixed as M
    d, disc, u, psi, neu = _case(O, ppa, g, s)
    sig, mu, x = M.solve_mixed(d, disc, neu, psi, u)
    nm = np.repeat(neu, g)
    Q, inside, outside = _points()
    up = O.layer_potential(disc, Q, sig, mu)
    ue, _ = harmonic.fields(Q, HOLE)
    return dict(
        interior=np.abs(up[inside] - ue[inside]).max(0),
        outside=np.abs(up[outside]).max(0),
        u_neu=np.abs(x[nm] - u[nm]).max(0),
        psi_dir=np.abs(x[~nm, :2] - psi[~nm, :2]).max(0) / np.abs(psi[~nm, :2]).max(0),
        sig=sig, mu=mu, u=u, psi=psi, nm=nm)


@pytest.fixture(scope="module")
def errs(oracle_mod):
    return {k: _errors(oracle_mod, *k) for k in [(4, 16, 80), (8, 16, 80)]}


def test_region_orientation(oracle_mod):
    from oracle import mixed as M
    d, disc, *_ = _case(oracle_mod, 4, 8, 40)
    area = M.signed_areas(d, disc).sum()
    assert abs(area - np.pi * (0.35 ** 2 - 0.12 ** 2)) < 1e-4


def test_harmonic_solution_inside(errs):
    e = errs[(8, 16, 80)]
    assert e["interior"].max() < 2.5e-6
    assert e["u_neu"].max() < 3e-6
    assert e["psi_dir"].max() < 1e-4
    assert e["interior"][2] < 5e-7          # the constant channel


def test_second_order_convergence(errs):
    c, f = errs[(4, 16, 80)], errs[(8, 16, 80)]
    for k in ("interior", "u_neu"):
        assert np.all(c[k] / f[k] > 3.0), (k, c[k], f[k])


def test_representation_vanishes_outside(errs):
    e = errs[(8, 16, 80)]
    assert e["outside"].max() < 1e-6


def test_mu_is_minus_u_and_sigma_is_psi(errs):
    e = errs[(8, 16, 80)]
    nm = e["nm"]
    np.testing.assert_array_equal(e["mu"][~nm], -e["u"][~nm])     # Dirichlet: given u
    np.testing.assert_array_equal(e["sig"][nm], e["psi"][nm])     # Neumann: given psi


def test_all_dirichlet_is_the_two_sided_problem(oracle_mod):
    from oracle import mixed as M
    O = oracle_mod
    d, disc, u, psi, _ = _case(O, 2, 8, 40)
    sig, mu, _ = M.solve_mixed(d, disc, np.zeros(d.n_panels, bool), psi, u)
    ref = O.solve_values(disc, np.zeros_like(u), u)
    assert np.abs(sig - ref.sigma).max() <= 1e-10 * np.abs(ref.sigma).max()
    np.testing.assert_array_equal(mu, ref.mu)


def test_default_dirichlet_data_are_the_inside_colours(oracle_mod):
    from oracle import mixed as M
    O = oracle_mod
    d, disc, _, psi, neu = _case(O, 2, 8, 40)
    um = O.boundary_values(d, disc)[1]
    a = M.solve_mixed(d, disc, neu, psi)
    b = M.solve_mixed(d, disc, neu, psi, um)
    np.testing.assert_array_equal(a[0], b[0])
