"""Pins of the float64 reference of the warm start's last steps: the bilinear resample of
the network's (u, v) output onto the GS grid with the phase taken from it, the input's
area average, and the Adam update. Expected values are worked by hand
(tests/golden/warmstart_resample_adam.json) or follow from properties of the definitions."""

import json
import os

import numpy as np

from oracle import conv


def _golden(golden_dir):
    with open(os.path.join(golden_dir, "warmstart_resample_adam.json")) as f:
        return json.load(f)


def test_resample_hand_worked_2x2_to_4x4(golden_dir):
    g = _golden(golden_dir)["resample_2x2_to_4x4"]
    assert np.allclose(conv.bilinear_resample(g["u_in"], 4, 4), g["u_out"], atol=1e-15)
    assert np.allclose(conv.bilinear_resample(g["v_in"], 4, 4), g["v_out"], atol=1e-15)
    uv = np.stack([np.array(g["u_in"], float), np.array(g["v_in"], float)], axis=-1)
    ph = conv.phase_of_uv(uv, 4, 4)
    # phase = atan2(v, u): u >= 1 and 0 <= v <= 1 keep it in [0, pi/4]
    assert np.allclose(ph, np.arctan2(g["v_out"], g["u_out"]), atol=1e-15)
    assert ph.min() >= 0 and ph.max() <= np.pi / 4


def test_resample_hand_worked_non_integer_scale(golden_dir):
    g = _golden(golden_dir)["resample_1x3_to_1x5"]
    assert np.allclose(conv.bilinear_resample(g["u_in"], 1, 5), g["u_out"], atol=1e-14)


def test_resample_identity_and_linear_exactness():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((6, 10))
    assert np.array_equal(conv.bilinear_resample(x, 6, 10), x)
    uv = rng.standard_normal((6, 10, 2))
    assert np.allclose(conv.phase_of_uv(uv, 6, 10), np.arctan2(uv[..., 1], uv[..., 0]), atol=0)
    # a linear field a + b*y + c*x is reproduced at every interior sample position
    H, W, Ho, Wo = 8, 8, 24, 20
    yy, xx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    lin = 0.5 + 1.5 * yy - 0.75 * xx
    out = conv.bilinear_resample(lin, Ho, Wo)
    sy = (np.arange(Ho) + 0.5) * H / Ho - 0.5
    sx = (np.arange(Wo) + 0.5) * W / Wo - 0.5
    iy = (sy >= 0) & (sy <= H - 1)
    ix = (sx >= 0) & (sx <= W - 1)
    ref = 0.5 + 1.5 * sy[:, None] - 0.75 * sx[None, :]
    assert np.allclose(out[np.ix_(iy, ix)], ref[np.ix_(iy, ix)], atol=1e-12)
    # transposed shapes transpose the result
    assert np.allclose(conv.bilinear_resample(x.T, 15, 9), conv.bilinear_resample(x, 9, 15).T, atol=1e-15)


def test_resample_integer_upsample_partition_of_unity():
    # 4x upsampling: every output is a convex combination of its neighbours (weights sum
    # to one), so a constant stays constant and outputs stay within the input range
    rng = np.random.default_rng(4)
    x = rng.uniform(-1, 1, (8, 8))
    out = conv.bilinear_resample(x, 32, 32)
    assert np.allclose(conv.bilinear_resample(np.full((8, 8), 2.5), 32, 32), 2.5, atol=1e-15)
    assert out.min() >= x.min() - 1e-15 and out.max() <= x.max() + 1e-15
    # a global phase rotation of (u, v) shifts the output phase by the same angle
    uv = rng.standard_normal((8, 8, 2))
    a = 0.7
    rot = np.stack([np.cos(a) * uv[..., 0] - np.sin(a) * uv[..., 1],
                    np.sin(a) * uv[..., 0] + np.cos(a) * uv[..., 1]], axis=-1)
    d = conv.phase_of_uv(rot, 20, 20) - conv.phase_of_uv(uv, 20, 20) - a
    assert np.allclose(np.angle(np.exp(1j * d)), 0, atol=1e-12)


def test_area_average_blocks():
    t = np.arange(16, dtype=float).reshape(4, 4)
    assert np.array_equal(conv.area_average(t, 2), [[2.5, 4.5], [10.5, 12.5]])
    assert np.array_equal(conv.area_average(t, 4), t)


def test_adam_hand_worked_two_steps(golden_dir):
    g = _golden(golden_dir)["adam_two_steps"]
    hp = dict(lr=g["lr"], beta1=g["beta1"], beta2=g["beta2"], eps=g["eps"])
    w = np.array(g["w0"])
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    w, m, v = conv.adam_step(w, g["g1"], m, v, 1, **hp)
    assert np.allclose(w, g["w1"], atol=1e-14)
    w, m, v = conv.adam_step(w, g["g2"], m, v, 2, **hp)
    assert np.allclose(w, g["w2"], atol=1e-14)
    assert np.allclose(m, g["m2"], atol=1e-14) and np.allclose(v, g["v2"], atol=1e-14)


def test_adam_first_step_and_scale_invariance():
    rng = np.random.default_rng(5)
    w0 = rng.standard_normal(50)
    g = rng.standard_normal(50)
    z = np.zeros(50)
    # bias correction makes the first step exactly lr * g / (|g| + eps)
    w1, _, _ = conv.adam_step(w0, g, z, z, 1, 1e-3, eps=0.0)
    assert np.allclose(w0 - w1, 1e-3 * np.sign(g), atol=1e-15)
    # with eps = 0 the update does not change when every gradient is scaled by c > 0
    g2 = rng.standard_normal(50)
    a1, m1, v1 = conv.adam_step(w0, g, z, z, 1, 1e-3, eps=0.0)
    a2, _, _ = conv.adam_step(a1, g2, m1, v1, 2, 1e-3, eps=0.0)
    b1, n1, u1 = conv.adam_step(w0, 7.0 * g, z, z, 1, 1e-3, eps=0.0)
    b2, _, _ = conv.adam_step(b1, 7.0 * g2, n1, u1, 2, 1e-3, eps=0.0)
    assert np.allclose(a2, b2, atol=1e-13)
    # a zero gradient from zero moments leaves the weights in place
    w, m, v = conv.adam_step(w0, z, z, z, 3, 1e-3)
    assert np.array_equal(w, w0) and not m.any() and not v.any()
