"""Pins of the oracle's replay error (paper Section 5.2, Eq. 3)."""

import json
import os
from fractions import Fraction

import numpy as np

from oracle import error


def test_hand_worked_2x2(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "replay_error_2x2.json")))
    a, m, n = error.replay_error(np.array(g["I"], float), np.array(g["T"], float))
    assert abs(a - float(Fraction(*g["alpha"]))) < 1e-15
    assert abs(m - float(Fraction(*g["mse"]))) < 1e-15
    assert abs(n - float(Fraction(*g["nmse"]))) < 1e-15


def test_exact_replay_has_zero_error():
    rng = np.random.default_rng(3)
    T = rng.random((16, 16))
    kappa = 3.7
    a, m, n = error.replay_error(kappa * T ** 2, T)
    assert abs(a - 1 / kappa) < 1e-14
    assert m < 1e-28 and n < 1e-28


def test_scale_invariance():
    rng = np.random.default_rng(4)
    T = rng.random((16, 8))
    I = rng.random((16, 8))
    a1, m1, n1 = error.replay_error(I, T)
    a2, m2, n2 = error.replay_error(5.0 * I, T)
    assert abs(n1 - n2) < 1e-14 * n1
    assert abs(m1 - m2) < 1e-14 * m1
    assert abs(a2 * 5.0 - a1) < 1e-14 * a1


def test_mask_restricts_sums():
    rng = np.random.default_rng(5)
    T = rng.random((8, 8))
    I = rng.random((8, 8))
    mask = np.zeros((8, 8), np.uint8)
    mask[:4] = 1
    full = error.replay_error(I[:4], T[:4])
    masked = error.replay_error(I, T, mask)
    assert np.allclose(full, masked, rtol=1e-15)


def test_paper_normalisation():
    assert error.paper_nmse([2.0, 4.0], [3.0, 3.0]) == 1.0
