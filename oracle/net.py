"""Plain FP64 oracle of the learned PCG warm start: a two-layer 3-D convolutional
network on the control-point grid, its gradients, the Adam update, and the
features and target built from the method's own solves.

TEST INFRASTRUCTURE ONLY (same rule as the rest of `oracle/`): the CUDA path
never imports it.

The warm start is not part of the paper. Its only link to the method is the
solve it feeds: the k mass systems M Z_j = b_j of every time step (Sec. 4,
eq. ho1), solved by PCG (Sec. 5.5). What is fixed here:

  * Network: y = conv2(R(relu(conv1(x)))), conv1: 3 -> 16 channels, conv2:
    16 -> 1, 3x3x3 taps, zero padding ("same" size), with biases. R rounds to
    BF16 (round to nearest even); inputs and weights are BF16 values, sums FP32
    on the device and FP64 here.
  * Layout: a field on the n1 x n2 x n3 interior grid is a flat co-lexicographic
    vector (i1 fastest), here reshaped to (n3, n2, n1). Tap t = e1 + 3 e2 + 9 e3,
    e in {0,1,2}, reads the neighbour at offset (e1-1, e2-1, e3-1) along
    (i1, i2, i3): y[o, p] = b[o] + sum_c sum_t W[o, c, t] x[c, p + off(t)].
  * Parameter vector (NPARAM = 1745 floats): W1 [16][3][27], b1 [16],
    W2 [16][27] (one output channel), b2 [1].
  * Features of the solve of stage j at step n from the right-hand sides b^n,
    b^{n-1}, b^{n-2} and the solutions Z^{n-1}, Z^{n-2} of the same stage:
        E  = 2 Z^{n-1} - Z^{n-2}                      (extrapolated guess)
        c0 = D^{-1} (b^n - 2 b^{n-1} + b^{n-2})        (D = diag M)
        s0 = rms(c0), s1 = rms(Z^{n-1})                (1 where the rms is 0)
        x  = R32(c0 / s0, Z^{n-1} / s1, Z^{n-2} / s1)  (FP64 -> FP32 -> BF16)
    Because M Z^m = b^m for every m, b^n - 2 b^{n-1} + b^{n-2} = b^n - M E: c0
    is the Jacobi-scaled residual of the extrapolated guess, obtained without
    a product with M.
  * Guess x0 = E + s0 y; training target t = (Z^n - E) / s0, which equals
    M^{-1}(b^n - 2 b^{n-1} + b^{n-2}) / s0 up to the solver tolerance.
  * Loss of one sample: L = sum_p (y_p - t_p)^2 / (2 N); dL/dy = (y - t) / N.
  * Adam (Kingma and Ba, 2015), beta1 = 0.9, beta2 = 0.999, eps = 1e-8.

Parity status: pinned by tests/test_oracle_net.py (brute-force convolution,
finite-difference gradients, the Adam closed forms, BF16 rounding cases, and
the target identity against a dense solve).
"""
from __future__ import annotations

import numpy as np

C_IN = 3
C_HID = 16
NTAP = 27
N_W1 = C_HID * C_IN * NTAP
N_B1 = C_HID
N_W2 = C_HID * NTAP
N_B2 = 1
NPARAM = N_W1 + N_B1 + N_W2 + N_B2

ADAM_B1 = 0.9
ADAM_B2 = 0.999
ADAM_EPS = 1e-8


def tap_offset(t: int):
    """Offset (d1, d2, d3) along (i1, i2, i3) of tap t."""
    return (t % 3 - 1, (t // 3) % 3 - 1, t // 9 - 1)


def bf16_round(a):
    """Round to the nearest BF16 value, ties to even, via FP32 (FP64 -> FP32 by
    numpy's round-to-nearest, then the upper 16 bits of the FP32 pattern)."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def split_params(theta):
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.shape == (NPARAM,)
    o = 0
    W1 = theta[o:o + N_W1].reshape(C_HID, C_IN, NTAP); o += N_W1
    b1 = theta[o:o + N_B1]; o += N_B1
    W2 = theta[o:o + N_W2].reshape(1, C_HID, NTAP); o += N_W2
    b2 = theta[o:o + N_B2]
    return W1, b1, W2, b2


def join_params(W1, b1, W2, b2):
    return np.concatenate([np.ravel(W1), np.ravel(b1), np.ravel(W2), np.ravel(b2)])


def shift(x, off):
    """s[..., i3, i2, i1] = x[..., i3+d3, i2+d2, i1+d1], zero outside the grid."""
    d1, d2, d3 = off
    n3, n2, n1 = x.shape[-3:]
    pad = [(0, 0)] * (x.ndim - 3) + [(1, 1)] * 3
    xp = np.pad(x, pad)
    return xp[..., 1 + d3:1 + d3 + n3, 1 + d2:1 + d2 + n2, 1 + d1:1 + d1 + n1]


def conv3d(x, W, b):
    """y[o] = b[o] + sum_c sum_t W[o, c, t] shift(x[c], off(t)); x (C, n3, n2, n1)."""
    y = np.zeros((W.shape[0],) + x.shape[1:])
    for t in range(NTAP):
        y += np.einsum("oc,c...->o...", W[:, :, t], shift(x, tap_offset(t)))
    return y + b[:, None, None, None]


def forward(x, theta, round_act=True):
    """Returns (h, a, y) for one sample x of shape (3, n3, n2, n1)."""
    W1, b1, W2, b2 = split_params(theta)
    h = conv3d(x, W1, b1)
    a = np.maximum(h, 0.0)
    if round_act:
        a = bf16_round(a)
    y = conv3d(a, W2, b2)[0]
    return h, a, y


def backward(x, theta, dy, round_act=True, act=None):
    """Gradient of sum_p dy_p y_p with respect to theta (the BF16 rounding of the
    activations passes gradients through unchanged). With `act` given, that hidden
    layer is used instead of recomputing it and the ReLU derivative is [act > 0]
    (equal to [h > 0] for a layer computed from h): a check of another
    implementation's backward can then take the ReLU decision on its own values."""
    W1, b1, W2, b2 = split_params(theta)
    if act is None:
        h, a, _ = forward(x, theta, round_act)
    else:
        a = np.asarray(act, dtype=np.float64)
        h = a
    gW2 = np.empty_like(W2)
    da = np.zeros_like(a)
    for t in range(NTAP):
        off = tap_offset(t)
        gW2[0, :, t] = np.einsum("ijk,cijk->c", dy, shift(a, off))
        da += W2[0, :, t][:, None, None, None] * shift(dy[None], tuple(-o for o in off))
    gb2 = np.array([dy.sum()])
    dh = da * (h > 0)
    gW1 = np.empty_like(W1)
    for t in range(NTAP):
        gW1[:, :, t] = np.einsum("oijk,cijk->oc", dh, shift(x, tap_offset(t)))
    gb1 = dh.sum(axis=(1, 2, 3))
    return join_params(gW1, gb1, gW2, gb2)


def loss_and_dy(y, t):
    n = y.size
    d = y - t
    return float(np.sum(d * d) / (2.0 * n)), d / n


def adam(theta, g, m, v, step, lr):
    """One Adam update (step counts from 1); returns new (theta, m, v)."""
    m = ADAM_B1 * m + (1.0 - ADAM_B1) * g
    v = ADAM_B2 * v + (1.0 - ADAM_B2) * g * g
    mh = m / (1.0 - ADAM_B1 ** step)
    vh = v / (1.0 - ADAM_B2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + ADAM_EPS), m, v


def _rms(a):
    s = float(np.sqrt(np.mean(a * a)))
    return s if s > 0.0 else 1.0


def features(b, b1, b2, D, z1, z2, shape):
    """Network input x (3, n3, n2, n1), scales (s0, s1) and extrapolation E for
    one solve; vectors are flat co-lexicographic FP64."""
    E = 2.0 * z1 - z2
    c0 = (b - 2.0 * b1 + b2) / D
    s0 = _rms(c0)
    s1 = _rms(z1)
    x = np.stack([c0 / s0, z1 / s1, z2 / s1]).reshape((3,) + tuple(shape))
    return bf16_round(x), s0, s1, E


def target(z, E, s0, shape):
    return ((z - E) / s0).reshape(tuple(shape))


def guess(E, s0, y):
    return E + s0 * np.ravel(y)
