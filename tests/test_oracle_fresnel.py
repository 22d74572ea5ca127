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
GS under Fresnel propagation: kappa = 0 is the far-field GS oracle; one iteration equals
the explicit sums (inverse and forward, term by term); the error never increases.
"""

import numpy as np
import pytest

from oracle import gs, lut, ospr
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


def _inverse_fresnel_by_sum(E, kappa):
    """conj(Q(y,x)) * P^-1/2 sum_{u,v} E(u,v) exp(+2*pi*i*(u*y/H + v*x/W)), term by term."""
    H, W = E.shape
    out = np.zeros((H, W), dtype=complex)
    for y in range(H):
        for x in range(W):
            acc = 0.0 + 0.0j
            for u in range(H):
                for v in range(W):
                    ang = 2.0 * np.pi * (u * y / H + v * x / W)
                    acc += E[u, v] * complex(np.cos(ang), np.sin(ang))
            q = np.pi * kappa * ((x - W / 2) ** 2 + (y - H / 2) ** 2)
            out[y, x] = acc * complex(np.cos(q), -np.sin(q)) / np.sqrt(H * W)
    return out


def test_gs_kappa_zero_is_the_far_field_oracle():
    T = blob_target(32, 32, 1000)
    table = lut.lut_codes(7, 1031)
    q0, I0, e0, _ = gs.gs(T, 4, table, 1031, 7)
    q1, I1, e1, _ = gs.gs_fresnel(T, 4, table, 1031, 7, 0.0)
    assert np.array_equal(q0, q1)
    np.testing.assert_allclose(e1, e0, rtol=1e-12)
    np.testing.assert_allclose(I1, I0, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("levels", [256, 2])
def test_gs_step_equals_explicit_sums(levels):
    H, W, kappa = 4, 8, 0.093
    rng = np.random.default_rng(5)
    T = rng.random((H, W)) + 0.1
    Ts = gs.energy_scaled_target(T)
    E = Ts * np.exp(1j * 2 * np.pi * rng.random((H, W)))
    q, R, eps, En = gs.gs_step_fresnel(E, Ts, kappa, levels)
    Hf = _inverse_fresnel_by_sum(E, kappa)
    q_ref = gs.quantise_phase(Hf, levels)
    assert np.array_equal(q, q_ref)
    h = gs.hologram_of_codes(q_ref, levels)
    I_ref = _fresnel_replay_by_sum(h, kappa)
    np.testing.assert_allclose(np.abs(R) ** 2, I_ref, rtol=1e-10, atol=1e-10)
    assert eps == pytest.approx(float(np.sum((np.sqrt(I_ref) - Ts) ** 2)), rel=1e-10)


@pytest.mark.parametrize("levels", [256, 2])
def test_gs_fresnel_error_never_increases(levels):
    T = blob_target(32, 64, 1003)
    table = lut.lut_codes(5, 4099)
    _, _, eps, _ = gs.gs_fresnel(T, 12, table, 4099, 5, 0.004, levels=levels)
    assert np.all(np.diff(eps) <= 1e-9 * eps[0]), eps
