"""Pins of the oracle's Fresnel-propagation OSPR (paper Section 2 names Fresnel propagation
as the near-field alternative to the Fourier far field of Eq. 1 / Eq. 2).

Model (the reading in the oracle's docstring): replay intensity |DFT(h * Q)|^2 with
Q(y, x) = exp(i*pi*kappa*((x - W/2)^2 + (y - H/2)^2)); back-propagation conj(Q) * IDFT(E).
What would catch a dropped chirp, a chirp of the wrong sign or a transposed raster:
  * kappa = 0 reduces to the Fourier OSPR oracle, which has its own pins;
  * an explicit double sum over the pixels with the quadratic phase written into the
    kernel (no FFT) equals the oracle's replay on 4x8 and 8x4 rasters;
  * a lens: the back-propagated image of a point at the replay origin is conj(Q), and
    the hologram conj(Q) focuses all energy P into the origin;
  * unitarity: every sub-frame's replay energy equals P;
  * a real hologram's Fourier replay is centrosymmetric (twin image); its Fresnel replay
    is not, so a chirp missing from the replay breaks this pin.
"""

import numpy as np
import pytest

from oracle import lut, ospr
from synthetic import blob_target


def _fresnel_replay_by_sum(h, kappa):
    """|R(u, v)|^2 from R(u, v) = P^-1/2 sum_{y,x} h(y,x) exp(i*pi*kappa*(x~^2 + y~^2))
    exp(-2*pi*i*(u*y/H + v*x/W)), evaluated term by term."""
    H, W = h.shape
    out = np.zeros((H, W))
    for u in range(H):
        for v in range(W):
            acc = 0.0 + 0.0j
            for y in range(H):
                for x in range(W):
                    q = np.pi * kappa * ((x - W / 2) ** 2 + (y - H / 2) ** 2)
                    ang = q - 2.0 * np.pi * (u * y / H + v * x / W)
                    acc += h[y, x] * complex(np.cos(ang), np.sin(ang))
            out[u, v] = abs(acc) ** 2 / (H * W)
    return out


@pytest.mark.parametrize("H,W,kappa", [(4, 8, 0.137), (8, 4, 0.61)])
def test_replay_equals_explicit_sum(H, W, kappa):
    rng = np.random.default_rng(H * 10 + W)
    h = np.where(rng.random((H, W)) < 0.5, 1.0, -1.0)
    np.testing.assert_allclose(ospr.replay_intensity_fresnel(h, kappa), _fresnel_replay_by_sum(h, kappa),
                               rtol=1e-10, atol=1e-10)


def test_kappa_zero_is_the_fourier_oracle():
    T = blob_target(32, 64, 1000)
    table = lut.lut_codes(7, 1031)
    b0, I0, _ = ospr.ospr(T, 5, table, 1031, 7)
    b1, I1, _ = ospr.ospr_fresnel(T, 5, table, 1031, 7, 0.0)
    assert np.array_equal(b0, b1)
    np.testing.assert_allclose(I1, I0, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("kappa", [0.01, 0.25])
def test_lens(kappa):
    H, W = 16, 32
    Q = ospr.fresnel_chirp(H, W, kappa)
    # a point at the replay origin back-propagates to the lens conj(Q) (scaled by P^-1/2)
    E = np.zeros((H, W), dtype=complex)
    E[0, 0] = np.sqrt(H * W)
    np.testing.assert_allclose(ospr.back_propagate_fresnel(E, kappa), np.conj(Q), atol=1e-12)
    # and the lens focuses all of its energy into the origin
    I = ospr.replay_intensity_fresnel(np.conj(Q), kappa)
    assert I[0, 0] == pytest.approx(H * W, rel=1e-12)
    assert np.abs(I.reshape(-1)[1:]).max() < 1e-9


def test_energy_and_symmetry():
    H, W = 32, 32
    T = blob_target(H, W, 1001)
    table = lut.lut_codes(11, 4099)
    for kappa, symmetric in [(0.0, True), (0.003, False)]:
        bits, I, _ = ospr.ospr_fresnel(T, 3, table, 4099, 11, kappa)
        for s in range(3):
            h = ospr.unpack_bits(bits[s], H * W).reshape(H, W)
            assert ospr.replay_intensity_fresnel(h, kappa).sum() == pytest.approx(H * W, rel=1e-12)
        twin = np.roll(np.flip(I), shift=(1, 1), axis=(0, 1))
        gap = np.abs(I - twin).max() / I.max()
        assert (gap < 1e-12) == symmetric, (kappa, gap)


def test_bits_follow_the_binarised_field():
    T = blob_target(16, 16, 1002)
    table = lut.lut_codes(3, 257)
    bits, I, extra = ospr.ospr_fresnel(T, 2, table, 257, 3, 0.02, keep_fields=True)
    for s in range(2):
        assert np.array_equal(ospr.unpack_bits(bits[s], 256), np.where(extra["re_h"][s].reshape(-1) >= 0, 1.0, -1.0))
    np.testing.assert_allclose(ospr.replay_from_bits_fresnel(bits, 16, 16, 0.02), I, rtol=1e-12)
