"""Pins of the oracle's unitary DFT (paper Section 2, Eq. 1 and Eq. 2).

The radix-2 FFT is checked against the brute-force double sum of Eq. 1 / Eq. 2, against
numpy's library FFT (an independent implementation), and against closed forms:
Parseval (unitarity), the transform of an impulse, and the inverse identity.
"""

import numpy as np
import pytest

from oracle import fft
from synthetic import random_field

SHAPES = [(1, 1), (1, 2), (2, 1), (2, 2), (4, 8), (8, 4), (16, 16), (8, 64), (32, 32)]


@pytest.mark.parametrize("shape", SHAPES)
def test_fft2_matches_bruteforce_eq1(shape):
    f = random_field(*shape, seed=11)
    assert np.max(np.abs(fft.fft2(f) - fft.dft2_brute(f))) < 1e-12


@pytest.mark.parametrize("shape", SHAPES)
def test_ifft2_matches_bruteforce_eq2(shape):
    F = random_field(*shape, seed=12)
    assert np.max(np.abs(fft.ifft2(F) - fft.idft2_brute(F))) < 1e-12


def test_bruteforce_sign_convention_eq1():
    # Eq. 1 has exp(-2 pi i ...): a pure tone exp(+2 pi i x u0/N) lands on bin u0.
    n = 8
    x = np.arange(n)
    f = np.exp(2j * np.pi * 3 * x / n)[:, None] * np.ones((1, 4))
    F = fft.dft2_brute(f)
    peak = np.unravel_index(np.argmax(np.abs(F)), F.shape)
    assert peak == (3, 0)
    assert abs(F[3, 0] - np.sqrt(n * 4)) < 1e-12


@pytest.mark.parametrize("shape", [(64, 128), (128, 64), (256, 256)])
def test_fft2_matches_numpy_library(shape):
    f = random_field(*shape, seed=13)
    assert np.max(np.abs(fft.fft2(f) - np.fft.fft2(f, norm="ortho"))) < 1e-11
    assert np.max(np.abs(fft.ifft2(f) - np.fft.ifft2(f, norm="ortho"))) < 1e-11


@pytest.mark.parametrize("shape", [(64, 64), (32, 256)])
def test_parseval_unitary(shape):
    f = random_field(*shape, seed=14)
    e0 = np.sum(np.abs(f) ** 2)
    assert abs(np.sum(np.abs(fft.fft2(f)) ** 2) - e0) < 1e-10 * e0
    assert abs(np.sum(np.abs(fft.ifft2(f)) ** 2) - e0) < 1e-10 * e0


def test_impulse_gives_plane_wave():
    H, W = 16, 32
    f = np.zeros((H, W), dtype=complex)
    f[3, 5] = 1.0
    F = fft.fft2(f)
    u = np.arange(H)[:, None]
    v = np.arange(W)[None, :]
    expect = np.exp(-2j * np.pi * (u * 3 / H + v * 5 / W)) / np.sqrt(H * W)
    assert np.max(np.abs(F - expect)) < 1e-14
    f0 = np.zeros((H, W))
    f0[0, 0] = 1.0
    assert np.max(np.abs(fft.fft2(f0) - 1.0 / np.sqrt(H * W))) < 1e-15


def test_inverse_identity():
    f = random_field(128, 64, seed=15)
    assert np.max(np.abs(fft.ifft2(fft.fft2(f)) - f)) < 1e-12
    assert np.max(np.abs(fft.fft2(fft.ifft2(f)) - f)) < 1e-12


def test_real_input_is_hermitian():
    f = random_field(32, 16, seed=16).real
    F = fft.fft2(f)
    Fm = np.roll(np.flip(F), shift=(1, 1), axis=(0, 1))     # F[-u mod H, -v mod W]
    assert np.max(np.abs(F - np.conj(Fm))) < 1e-13


def test_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        fft.fft2(np.zeros((6, 8)))
