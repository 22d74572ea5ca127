"""Pins of the oracle's Gerchberg-Saxton (paper Section 2, Section 3, Section 8).

  * error reduction: both per-plane steps are nearest-point projections (the quantised
    phase is the nearest allowed unit-modulus value; T_s*exp(i arg R) is the nearest
    field of the target amplitude) and the transforms are unitary, so
    eps_k = sum (|R_k| - T_s)^2 never increases;
  * global-phase equivariance: a table of length 1 puts the same phase c0 on every
    pixel; every later field is the flat-start field times exp(2 pi i c0/256), so the
    codes differ by exactly c0 (mod 256) and the errors are equal;
  * levels = 2 is the binary device: exp(i*pi*q) = sign(Re H) away from Re H = 0;
  * the energy-matched target carries P units of energy.
"""

import numpy as np
import pytest

from oracle import fft, gs, lut, ospr
from synthetic import blob_target, noise_target


def test_energy_scaled_target():
    T = blob_target(32, 32, 1000)
    Ts = gs.energy_scaled_target(T)
    assert abs(np.sum(Ts ** 2) - 32 * 32) < 1e-9
    assert np.allclose(Ts / Ts.max(), T / T.max(), rtol=1e-6, atol=1e-7)


def test_quantiser_cases():
    H = np.array([1 + 0j, -1 + 0j, 1j, -1j, 0j, np.exp(1j * (np.pi / 256) * 0.999),
                  np.exp(1j * (np.pi / 256) * 1.001), np.exp(-1j * (np.pi / 256) * 1.001)])
    q = gs.quantise_phase(H, 256)
    assert list(q) == [0, 128, 64, 192, 0, 0, 1, 255]
    q2 = gs.quantise_phase(np.array([1 + 0j, -1 + 0j, 0.1 + 1j, -0.1 + 1j]), 2)
    assert list(q2) == [0, 1, 0, 1]


@pytest.mark.parametrize("levels", [256, 2])
@pytest.mark.parametrize("kind", ["blob", "noise"])
def test_error_non_increasing(levels, kind):
    H = W = 64
    T = blob_target(H, W, 1004) if kind == "blob" else noise_target(H, W, 2004)
    L = 1031
    table = lut.lut_codes(3, L)
    q, I, eps, E = gs.gs(T, 25, table, L, 3, levels=levels)
    assert eps.shape == (25,)
    d = np.diff(eps)
    assert np.all(d <= 1e-12 * eps[0]), d.max()
    assert eps[-1] < eps[0]


def test_global_phase_equivariance():
    H = W = 32
    T = blob_target(H, W, 1005)
    c0 = 77
    q1, I1, e1, _ = gs.gs(T, 6, np.array([c0]), 1, 0)
    q0, I0, e0, _ = gs.gs(T, 6, None, 0, 0)
    # compare away from quantiser ties: check the fraction that agree
    agree = np.mean((q0 + c0) % 256 == q1)
    assert agree > 0.999
    assert np.allclose(e1, e0, rtol=1e-9)
    assert np.max(np.abs(I1 - I0)) < 1e-8 * I0.max()


def test_binary_levels_match_sign_of_real_part():
    H = W = 32
    T = blob_target(H, W, 1006)
    table = lut.lut_codes(4, 521)
    E = gs.initial_field(T, table, 521, 4)
    Hf = fft.ifft2(E)
    q = gs.quantise_phase(Hf, 2)
    h = gs.hologram_of_codes(q, 2)
    away = np.abs(Hf.real) > 1e-9 * np.abs(Hf).max()
    assert np.allclose(h.real[away], ospr.binarise(Hf.real)[away])
    assert np.max(np.abs(h.imag)) < 1e-15


def test_first_iteration_by_hand():
    # one iteration written out step by step on a 4x8 case with explicit DFT matrices
    H, W = 4, 8
    T = blob_target(H, W, 1007)
    table = lut.lut_codes(8, 11)
    q, I, eps, E1 = gs.gs(T, 1, table, 11, 8)
    Ts = T * np.sqrt(H * W / np.sum(T.astype(float) ** 2))
    c = table[np.arange(H * W) % 11].reshape(H, W)
    E0 = Ts * np.exp(2j * np.pi * c / 256)
    k_r, k_c = np.arange(H), np.arange(W)
    Fr = np.exp(-2j * np.pi * np.outer(k_r, k_r) / H)
    Fc = np.exp(-2j * np.pi * np.outer(k_c, k_c) / W)
    Hf = np.conj(Fr) @ E0 @ np.conj(Fc).T / np.sqrt(H * W)
    qq = np.mod(np.floor(256 * np.angle(Hf) / (2 * np.pi) + 0.5), 256).astype(int)
    assert np.array_equal(qq, q)
    R = Fr @ np.exp(2j * np.pi * qq / 256) @ Fc.T / np.sqrt(H * W)
    assert np.max(np.abs(np.abs(R) ** 2 - I)) < 1e-12
    assert abs(np.sum((np.abs(R) - Ts) ** 2) - eps[0]) < 1e-10
    assert np.max(np.abs(E1 - Ts * np.exp(1j * np.angle(R)))) < 1e-12


def test_lut_levels_independent_of_hologram_levels():
    # the initial phase comes from 8-bit table codes whatever the hologram's levels are
    H = W = 32
    T = blob_target(H, W, 1012)
    table = lut.lut_codes(6, 101)
    E256 = gs.initial_field(T, table, 101, 6)
    q2, _, e2, _ = gs.gs(T, 1, table, 101, 6, levels=2)
    q2b, _, e2b, _ = gs.gs(T, 1, None, 0, 0, levels=2, init_field=E256)
    assert np.array_equal(q2, q2b) and np.allclose(e2, e2b, rtol=1e-14)


def test_caller_phase_start_equals_lut_phase():
    H = W = 16
    T = blob_target(H, W, 1008)
    table = lut.lut_codes(2, 97)
    theta = lut.phase_of_codes(table[np.arange(H * W) % 97]).reshape(H, W)
    a = gs.gs(T, 3, table, 97, 2)
    b = gs.gs(T, 3, None, 0, 0, init_phase=theta)
    assert np.array_equal(a[0], b[0])
    assert np.allclose(a[2], b[2], rtol=1e-12)


def test_resume_from_state():
    H = W = 16
    T = blob_target(H, W, 1009)
    table = lut.lut_codes(2, 97)
    q6, I6, e6, _ = gs.gs(T, 6, table, 97, 2)
    q3, _, e3, E3 = gs.gs(T, 3, table, 97, 2)
    q33, I33, e33, _ = gs.gs(T, 3, None, 0, 0, init_field=E3)
    assert np.array_equal(q33, q6)
    assert np.allclose(np.concatenate([e3, e33]), e6, rtol=1e-12)
