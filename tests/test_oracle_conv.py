"""Pins of the warm-start network's float64 reference: every backward is checked against
central finite differences of its forward on tiny shapes, and the forward convolution
against a direct sum over the padded input."""

import numpy as np
import pytest

from oracle import conv


def _fd(f, x, eps=1e-6):
    g = np.zeros_like(x)
    it = np.nditer(x, flags=["multi_index"])
    for _ in it:
        i = it.multi_index
        xp = x.copy()
        xm = x.copy()
        xp[i] += eps
        xm[i] -= eps
        g[i] = (f(xp) - f(xm)) / (2 * eps)
    return g


def test_conv_forward_direct_sum():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((1, 4, 5, 2))
    w = rng.standard_normal((3, 3, 3, 2))
    b = rng.standard_normal(3)
    y = conv.conv3x3(x, w, b)
    for (yy, xx, o) in [(0, 0, 0), (2, 3, 1), (3, 4, 2), (1, 2, 0)]:
        s = b[o]
        for ky in range(3):
            for kx in range(3):
                sy, sx = yy + ky - 1, xx + kx - 1
                if 0 <= sy < 4 and 0 <= sx < 5:
                    s += np.dot(x[0, sy, sx, :], w[o, ky, kx, :])
        assert abs(y[0, yy, xx, o] - s) < 1e-12


def test_conv_grads_finite_differences():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 4, 2))
    w = rng.standard_normal((3, 3, 3, 2))
    b = rng.standard_normal(3)
    dy = rng.standard_normal((2, 3, 4, 3))

    def loss_x(xx):
        return np.sum(conv.conv3x3(xx, w, b) * dy)

    def loss_w(ww):
        return np.sum(conv.conv3x3(x, ww, b) * dy)

    def loss_b(bb):
        return np.sum(conv.conv3x3(x, w, bb) * dy)

    assert np.max(np.abs(conv.conv3x3_dgrad(dy, w) - _fd(loss_x, x))) < 1e-7
    assert np.max(np.abs(conv.conv3x3_wgrad(x, dy) - _fd(loss_w, w))) < 1e-7
    assert np.max(np.abs(conv.bias_grad(dy) - _fd(loss_b, b))) < 1e-7


def test_pool_upsample_grads():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((1, 4, 6, 2))
    dy = rng.standard_normal((1, 2, 3, 2))
    g = _fd(lambda xx: np.sum(conv.avgpool2(xx) * dy), x)
    assert np.max(np.abs(conv.avgpool2_bwd(dy) - g)) < 1e-8
    dz = rng.standard_normal((1, 8, 12, 2))
    g2 = _fd(lambda xx: np.sum(conv.upsample2(xx) * dz), x)
    assert np.max(np.abs(conv.upsample2_bwd(dz) - g2)) < 1e-8


def test_phase_loss_properties_and_grad():
    rng = np.random.default_rng(3)
    B, H, W = 2, 3, 4
    out = rng.standard_normal((B, H, W, 2))
    z = np.exp(1j * rng.uniform(0, 2 * np.pi, (B, H, W)))
    wts = rng.random((B, H, W))
    L = conv.phase_loss(out, z, wts)
    assert 0.0 <= L <= 1.0
    # a prediction equal to the label up to a global offset has zero loss
    off = np.exp(0.7j) * z
    perfect = np.stack([off.real * 3.0, off.imag * 3.0], axis=-1)
    assert conv.phase_loss(perfect, z, wts) < 1e-12
    g = conv.phase_loss_grad(out, z, wts)
    fd = _fd(lambda o: conv.phase_loss(o, z, wts), out)
    assert np.max(np.abs(g - fd)) < 1e-7
