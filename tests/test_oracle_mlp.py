"""Pins of the warm-start oracle (oracle/mlp.py): the network gradient
against FP64 finite differences, GELU against closed values, BF16 rounding
against hand-worked ties, the features' invariance under rigid motions and
scaling of the drawing, and the nearest-panel lists on a hand-checked
layout.  CPU only."""
import dataclasses

import numpy as np
import pytest

from dc_synth import drawing_by_name, random_node_values


@pytest.fixture(scope="module")
def M():
    from oracle import mlp
    return mlp


def test_gelu_closed_values(M):
    assert M.gelu(0.0) == 0.0
    # Phi(1) of the standard normal distribution
    assert abs(M.gelu(1.0) - 0.8413447460685429) < 1e-15
    x = np.linspace(-6, 6, 97)
    # x Phi(x) - (-x) Phi(-x) = x since Phi(x) + Phi(-x) = 1
    np.testing.assert_allclose(M.gelu(x) - M.gelu(-x), x, atol=1e-14)
    h = 1e-6
    fd = (M.gelu(x + h) - M.gelu(x - h)) / (2 * h)
    np.testing.assert_allclose(M.gelu_grad(x), fd, atol=1e-9)


def test_bf16_rounding_ties_to_even(M):
    one = 1.0
    cases = {
        one: one,
        one + 2.0**-8: one,                         # tie, 1.0 has an even mantissa
        one + 3 * 2.0**-8: one + 2.0**-6,           # tie, rounds up to the even neighbour
        one + 2.0**-8 + 2.0**-20: one + 2.0**-7,    # above the tie
        -(one + 2.0**-9): -one,
        3.0e38: 2.9975e38,                          # largest finite magnitudes stay finite
    }
    for x, want in cases.items():
        got = float(M.bf16_round(np.array([x], dtype=np.float32))[0])
        if abs(want) > 1e30:
            assert np.isfinite(got) and abs(got - x) / x < 2.0**-8
        else:
            assert got == want, (x, got, want)


@pytest.mark.parametrize("rows", [1, 11])
def test_gradient_matches_finite_differences(M, rows):
    n_in, H, n_out = 5, 7, 3
    rng = np.random.default_rng(3)
    n = M.param_count(n_in, H, n_out)
    assert n == (7 * 5 + 7) + 2 * (7 * 7 + 7) + (3 * 7 + 3)
    p = rng.standard_normal(n) * 0.5
    x = rng.standard_normal((rows, n_in))
    t = rng.standard_normal((rows, n_out))
    loss, g = M.loss_grad(p, x, t, n_in, H, n_out, round_bf16=False)
    h = 1e-6
    fd = np.empty(n)
    for i in range(n):
        e = np.zeros(n)
        e[i] = h
        lp, _ = M.loss_grad(p + e, x, t, n_in, H, n_out, round_bf16=False)
        lm, _ = M.loss_grad(p - e, x, t, n_in, H, n_out, round_bf16=False)
        fd[i] = (lp - lm) / (2 * h)
    assert np.abs(g - fd).max() <= 1e-8 * max(1.0, np.abs(fd).max())
    y, _ = M.forward(p, x, n_in, H, n_out, round_bf16=False)
    assert abs(loss - np.mean((y - t) ** 2)) < 1e-15 * max(1.0, loss)


def test_adam_first_step_moves_by_lr(M):
    # after one step with bias correction, every parameter with a nonzero
    # gradient moves by lr * sign(g) (up to eps)
    rng = np.random.default_rng(4)
    p = rng.standard_normal(20)
    g = rng.standard_normal(20)
    m = np.zeros(20)
    v = np.zeros(20)
    q = M.adam_step(p.copy(), g, m, v, lr=1e-3, beta1=0.9, beta2=0.999, eps=0.0, step=1)
    np.testing.assert_allclose(p - q, 1e-3 * np.sign(g), rtol=1e-12)


def _transform(d, angle, shift, scale):
    c, s = np.cos(angle), np.sin(angle)
    R = np.array([[c, -s], [s, c]])
    ctrl = scale * np.einsum("ij,nkj->nki", R, d.ctrl) + np.asarray(shift)
    return dataclasses.replace(d, ctrl=ctrl)


def test_features_invariant_under_rotation_translation_scaling(M, oracle_mod):
    d = drawing_by_name("mixed16")
    disc = oracle_mod.discretise(d)
    up, um = oracle_mod.boundary_values(d, disc)
    f0, _ = M.panel_features(disc, up, um)
    d2 = _transform(d, 0.7, (0.31, -0.12), 0.45)
    disc2 = oracle_mod.discretise(d2)
    up2, um2 = oracle_mod.boundary_values(d2, disc2)
    f1, _ = M.panel_features(disc2, up2, um2)
    assert f0.shape == (3 * d.n_panels, M.n_features(d.g))
    np.testing.assert_allclose(f1, f0, atol=1e-9)
    # a reflection flips the orientation of the normals: features change
    d3 = dataclasses.replace(d, ctrl=d.ctrl * np.array([-1.0, 1.0]) + np.array([1.0, 0.0]))
    disc3 = oracle_mod.discretise(d3)
    up3, um3 = oracle_mod.boundary_values(d3, disc3)
    f3, _ = M.panel_features(disc3, up3, um3)
    assert np.abs(f3 - f0).max() > 0.1


def test_feature_layout_and_targets(M, oracle_mod):
    d = drawing_by_name("mixed16")
    disc = oracle_mod.discretise(d)
    up, um = oracle_mod.boundary_values(d, disc)
    sig = random_node_values(disc.n_nodes, seed=8)
    f, t = M.panel_features(disc, up, um, sig)
    g = d.g
    j, c = 5, 2
    r = 3 * j + c
    np.testing.assert_array_equal(f[r, 4 * g:5 * g], up[j * g:(j + 1) * g, c])
    np.testing.assert_array_equal(f[r, 5 * g:6 * g], um[j * g:(j + 1) * g, c])
    # own nodes: unit normals, centred positions spanning about one arc length
    own = f[r, :4 * g].reshape(g, 4)
    np.testing.assert_allclose(np.hypot(own[:, 2], own[:, 3]), 1.0, atol=1e-12)
    np.testing.assert_allclose(own[:, :2].mean(axis=0), 0.0, atol=1e-12)
    assert 0.5 < own[-1, 0] - own[0, 0] <= 1.0 and abs(own[-1, 1] - own[0, 1]) < 1e-12
    _, _, plen = M.panel_frames(disc)
    np.testing.assert_allclose(t[r], sig[j * g:(j + 1) * g, c] * plen[j], rtol=1e-15)
    # arc lengths of the panels add up to the curve lengths (App. A weighting)
    np.testing.assert_allclose(plen.sum(), disc.curve_len.sum(), rtol=1e-12)


def test_nearest_panels_hand_layout(M):
    cen = np.array([[0.0, 0.0], [1.0, 0.0], [3.0, 0.0], [6.0, 0.0], [10.0, 0.0], [0.0, 0.5]])
    nb = M.nearest_panels(cen, k=3)
    np.testing.assert_array_equal(nb[0], [5, 1, 2])
    np.testing.assert_array_equal(nb[3], [2, 4, 1])
    np.testing.assert_array_equal(nb[4], [3, 2, 1])
    few = M.nearest_panels(cen[:3], k=4)
    np.testing.assert_array_equal(few[0], [1, 2, -1, -1])
