"""Pins of the oracle's phase LUT and draw rule (paper Sections 4, 5 and 5.1, Fig. 3)."""

import json
import os

import numpy as np
import pytest

from oracle import lut


def _read_vectors(golden_dir):
    seed = None
    vals = []
    with open(os.path.join(golden_dir, "splitmix64_seed1234567.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("seed"):
                seed = int(line.split()[1])
            else:
                vals.append(int(line))
    return seed, vals


def test_splitmix64_published_vectors(golden_dir):
    seed, vals = _read_vectors(golden_dir)
    out = lut.splitmix64(seed, np.arange(len(vals), dtype=np.uint64))
    assert [int(v) for v in out] == vals


def test_codes_are_top_bits(golden_dir):
    seed, vals = _read_vectors(golden_dir)
    c256 = lut.lut_codes(seed, len(vals), 256)
    assert [int(c) for c in c256] == [v >> 56 for v in vals]
    c2 = lut.lut_codes(seed, len(vals), 2)
    assert [int(c) for c in c2] == [v >> 63 for v in vals]


def test_paper_lut_size_arithmetic(golden_dir):
    # Section 5.2: a table for 256x256 pixels x 24 sub-frames needs "over 12 Mb";
    # with one 8-bit code per entry that is 12,582,912 bits.
    facts = json.load(open(os.path.join(golden_dir, "paper_facts.json")))
    f = facts["lut_bits_for_full_independence"]
    bits = f["H"] * f["W"] * f["N_SF"] * lut.code_bits(256)
    assert bits >= f["value_bits_at_least"]
    assert bits == 12582912
    # 7-bit codes would fall short of the quoted size
    assert f["H"] * f["W"] * f["N_SF"] * 7 < f["value_bits_at_least"]


def test_codes_range_and_uniformity():
    c = lut.lut_codes(7, 1 << 16, 256)
    assert c.min() >= 0 and c.max() <= 255
    counts = np.bincount(c, minlength=256)
    expected = c.size / 256
    chi2 = np.sum((counts - expected) ** 2 / expected)
    assert chi2 < 400           # 255 dof: mean 255, sd ~22.6


def test_cyclic_draw_with_continuation():
    # Fig. 3: successive sub-frames continue through the pool where the last one stopped
    L, P, seed = 37, 16, 3
    table = lut.lut_codes(seed, L)
    draws = np.concatenate([lut.subframe_codes(table, L, seed, 5, s, P, P) for s in range(4)])
    expect = table[(5 + np.arange(4 * P)) % L]
    assert np.array_equal(draws, expect)
    # periodicity: c_{i+L} = c_i
    a = lut.subframe_codes(table, L, seed, 0, 0, P, 3 * L)
    assert np.array_equal(a[:L], a[L:2 * L])


def test_unrepeated_equals_long_table():
    # Section 5.1: a table at least as long as every draw of the run equals the generator
    H, W, N, seed = 8, 8, 3, 99
    P = H * W
    L = N * P
    table = lut.lut_codes(seed, L)
    for s in range(N):
        a = lut.subframe_codes(table, L, seed, 0, s, P, P)
        b = lut.subframe_codes(None, lut.UNREPEATED, seed, 0, s, P, P)
        assert np.array_equal(a, b)


def test_flat_phase_for_zero_length():
    c = lut.subframe_codes(None, 0, 1, 0, 2, 16, 16)
    assert np.all(c == 0)
    assert np.all(lut.phase_of_codes(c) == 0.0)


def test_phase_of_codes():
    assert lut.phase_of_codes(128, 256) == pytest.approx(np.pi, abs=1e-15)
    assert lut.phase_of_codes(1, 2) == pytest.approx(np.pi, abs=1e-15)
    assert lut.phase_of_codes(64, 256) == pytest.approx(np.pi / 2, abs=1e-15)


def test_rejects_bad_levels():
    with pytest.raises(ValueError):
        lut.lut_codes(1, 4, 3)
    with pytest.raises(ValueError):
        lut.lut_codes(1, 4, 512)
