"""Pins of the learned warm start's oracle (oracle/net.py) to facts outside it:
brute-force convolution loops, central finite differences of its own loss,
closed forms of the Adam update, hand-computed BF16 roundings, and the
identity between the features and a dense solve with the isogeometric mass
matrix."""
import itertools

import numpy as np
import pytest

import oracle
import oracle.net as net
import workloads as W


def _rand_theta(rng, scale=0.3):
    return rng.uniform(-scale, scale, net.NPARAM)


def test_param_count():
    assert net.NPARAM == 16 * 3 * 27 + 16 + 16 * 27 + 1 == 1745


def test_tap_offsets_cover_the_cube_once():
    offs = {net.tap_offset(t) for t in range(27)}
    assert offs == set(itertools.product((-1, 0, 1), repeat=3))
    assert net.tap_offset(0) == (-1, -1, -1) and net.tap_offset(13) == (0, 0, 0)
    assert net.tap_offset(1) == (0, -1, -1)  # i1 runs fastest


@pytest.mark.parametrize("v,expect", [
    (1.0, 1.0),
    (1.0 + 2.0 ** -8, 1.0),                           # tie, even mantissa kept
    (1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -6),            # tie, rounds up to even
    (1.0 + 2.0 ** -8 + 2.0 ** -20, 1.0 + 2.0 ** -7),  # above the tie
    (-(1.0 + 3 * 2.0 ** -8), -(1.0 + 2.0 ** -6)),
    (1.0 / 3.0, 0.333984375),
    (3.0, 3.0),
    (0.0, 0.0),
])
def test_bf16_round_to_nearest_even(v, expect):
    assert net.bf16_round(np.array([v]))[0] == expect


def test_conv_matches_brute_force_loops():
    rng = np.random.default_rng(0)
    n3, n2, n1 = 3, 4, 5
    ci, co = 2, 3
    x = rng.standard_normal((ci, n3, n2, n1))
    Wt = rng.standard_normal((co, ci, 27))
    b = rng.standard_normal(co)
    y = net.conv3d(x, Wt, b)
    ref = np.zeros_like(y)
    for o in range(co):
        for i3 in range(n3):
            for i2 in range(n2):
                for i1 in range(n1):
                    s = b[o]
                    for c in range(ci):
                        for e3 in range(3):
                            for e2 in range(3):
                                for e1 in range(3):
                                    j1, j2, j3 = i1 + e1 - 1, i2 + e2 - 1, i3 + e3 - 1
                                    if 0 <= j1 < n1 and 0 <= j2 < n2 and 0 <= j3 < n3:
                                        s += Wt[o, c, e1 + 3 * e2 + 9 * e3] * x[c, j3, j2, j1]
                    ref[o, i3, i2, i1] = s
    assert np.allclose(y, ref, rtol=0, atol=1e-12)


def test_corner_delta_sees_only_inner_taps():
    # a unit impulse at grid point (0,0,0): output at p picks W[..., tap with p + off = 0]
    Wt = np.arange(27, dtype=float).reshape(1, 1, 27) + 1.0
    x = np.zeros((1, 4, 4, 4))
    x[0, 0, 0, 0] = 1.0
    y = net.conv3d(x, Wt, np.zeros(1))[0]
    for i3, i2, i1 in itertools.product(range(4), repeat=3):
        off = (-i1, -i2, -i3)
        want = Wt[0, 0, (off[0] + 1) + 3 * (off[1] + 1) + 9 * (off[2] + 1)] if max(i1, i2, i3) <= 1 else 0.0
        assert y[i3, i2, i1] == want


def test_forward_is_positively_homogeneous_without_biases():
    rng = np.random.default_rng(1)
    W1, _, W2, _ = net.split_params(_rand_theta(rng))
    theta = net.join_params(W1, np.zeros(16), W2, np.zeros(1))
    x = rng.standard_normal((3, 4, 3, 5))
    _, _, y1 = net.forward(x, theta, round_act=False)
    _, _, y2 = net.forward(2.5 * x, theta, round_act=False)
    assert np.allclose(y2, 2.5 * y1, rtol=1e-13, atol=1e-13)
    _, _, y3 = net.forward(-x, theta, round_act=False)
    assert not np.allclose(y3, -y1)  # ReLU: not odd


def test_backward_matches_central_differences():
    rng = np.random.default_rng(2)
    shape = (3, 4, 5)
    x = rng.standard_normal((3,) + shape)
    theta = _rand_theta(rng)
    dy = rng.standard_normal(shape)
    g = net.backward(x, theta, dy, round_act=False)

    def L(th):
        return float(np.sum(dy * net.forward(x, th, round_act=False)[2]))

    idx = np.concatenate([rng.choice(net.N_W1, 60, replace=False),
                          net.N_W1 + np.arange(net.N_B1),
                          net.N_W1 + net.N_B1 + rng.choice(net.N_W2, 40, replace=False),
                          [net.NPARAM - 1]])
    h = 1e-6
    for i in idx:
        tp = theta.copy(); tp[i] += h
        tm = theta.copy(); tm[i] -= h
        fd = (L(tp) - L(tm)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_loss_gradient_is_residual_over_n():
    rng = np.random.default_rng(3)
    y = rng.standard_normal((2, 3, 4))
    t = rng.standard_normal((2, 3, 4))
    L, dy = net.loss_and_dy(y, t)
    h = 1e-6
    for i in range(5):
        yp = y.copy(); yp.flat[i] += h
        ym = y.copy(); ym.flat[i] -= h
        fd = (net.loss_and_dy(yp, t)[0] - net.loss_and_dy(ym, t)[0]) / (2 * h)
        assert abs(fd - dy.flat[i]) < 1e-8


def test_adam_first_step_is_signed_learning_rate():
    rng = np.random.default_rng(4)
    th = rng.standard_normal(50)
    g = rng.standard_normal(50)
    lr = 1e-3
    th1, _, _ = net.adam(th, g, np.zeros(50), np.zeros(50), 1, lr)
    assert np.allclose(th1, th - lr * g / (np.abs(g) + net.ADAM_EPS), rtol=0, atol=1e-15)


def test_adam_constant_gradient_moves_linearly():
    # with bias correction, a constant gradient gives m_hat = g and v_hat = g^2 at every step
    g = np.array([0.5, -2.0, 1e-3])
    th = np.zeros(3)
    m = np.zeros(3)
    v = np.zeros(3)
    lr = 0.01
    for s in range(1, 26):
        th, m, v = net.adam(th, g, m, v, s, lr)
    assert np.allclose(th, -25 * lr * g / (np.abs(g) + net.ADAM_EPS), rtol=1e-12, atol=0)


def test_features_are_the_scaled_residual_of_the_extrapolated_guess():
    # with exact solves M Z^m = b^m, c0 = D^{-1}(b^n - M E) and the target is
    # M^{-1}(b^n - 2 b^{n-1} + b^{n-2}) / s0
    w = W.small(d=3, nel=3, p=2, amp=0.1)
    P = oracle.Patch(w.p, w.knots, w.ctrl())
    Mb, _ = P.assemble()
    M = P.band_to_dense(Mb)
    D = np.diag(M).copy()
    assert np.allclose(D, P.mass_diagonal(), rtol=1e-13)
    shape = tuple(reversed(P.n))
    rng = np.random.default_rng(5)
    b, b1, b2 = rng.standard_normal((3, P.N))
    z, z1, z2 = (np.linalg.solve(M, v) for v in (b, b1, b2))
    x, s0, s1, E = net.features(b, b1, b2, D, z1, z2, shape)
    c0 = (b - M @ E) / D
    assert np.isclose(s0, np.sqrt(np.mean(c0 ** 2)), rtol=1e-10)
    assert np.isclose(s1, np.sqrt(np.mean(z1 ** 2)), rtol=1e-14)
    assert np.allclose(x[0].ravel(), c0 / s0, rtol=2.0 ** -8, atol=0)
    assert np.allclose(x[1].ravel(), z1 / s1, rtol=2.0 ** -8, atol=0)
    assert np.allclose(x[2].ravel(), z2 / s1, rtol=2.0 ** -8, atol=0)
    t = net.target(z, E, s0, shape)
    assert np.allclose(t.ravel(), np.linalg.solve(M, b - 2 * b1 + b2) / s0, rtol=1e-9, atol=1e-12)
    # the guess built from the exact target is the exact solution
    assert np.allclose(net.guess(E, s0, t), z, rtol=1e-12, atol=1e-12)


def test_features_guard_zero_scales():
    shape = (2, 2, 2)
    zero = np.zeros(8)
    x, s0, s1, E = net.features(zero, zero, zero, np.ones(8), zero, zero, shape)
    assert s0 == 1.0 and s1 == 1.0 and not x.any() and not E.any()


def test_backward_with_given_hidden_layer_equals_recomputed():
    rng = np.random.default_rng(6)
    x = net.bf16_round(rng.standard_normal((3, 3, 4, 5)))
    theta = net.bf16_round(_rand_theta(rng))
    dy = rng.standard_normal((3, 4, 5))
    _, a, _ = net.forward(x, theta)
    assert np.array_equal(net.backward(x, theta, dy), net.backward(x, theta, dy, act=a))
