"""Pins of the oracle's OSPR (paper Sections 2, 3, 5.1, 5.2).

Closed forms and invariants that a dropped term, a wrong sign or index, or a transposed
operand in the oracle would break:
  * a real binary hologram replays a twin image: I(u, v) = I(-u, -v)  (Section 6 shows
    only the top portion of the replay field for this reason);
  * unitarity: every sub-frame's replay energy equals the pixel count P;
  * L dividing the sub-frame stride gives every sub-frame the same phases, so the
    N-sub-frame average equals one sub-frame (the factorisation effect behind the
    prime-length rule of Section 8 and the L = 256 spike of Section 5.2);
  * L >= N*P makes the table equal to the generator (Section 5.1 hard limit);
  * adding half a turn to every code negates the field, so every bit inverts and the
    replay is unchanged;
  * on 4x4 and 8x8 the whole chain equals an explicit matrix DFT of the same steps.
"""

import numpy as np
import pytest

from oracle import lut, ospr
from synthetic import blob_target


def _twin(I):
    return np.roll(np.flip(I), shift=(1, 1), axis=(0, 1))    # I[-u mod H, -v mod W]


def _run(H, W, N, L, seed=7, start=0, levels=256):
    T = blob_target(H, W, 1000)
    table = lut.lut_codes(seed, L, levels) if L > 0 else None
    return T, ospr.ospr(T, N, table, L, seed, start=start, levels=levels, keep_fields=True)


def test_pack_unpack_roundtrip():
    rng = np.random.default_rng(1)
    h = np.where(rng.random(100) < 0.5, 1.0, -1.0)
    w = ospr.pack_bits(h)
    assert w.dtype == np.uint32 and w.size == 4
    assert np.array_equal(ospr.unpack_bits(w, 100), h)
    # bit j of word k is pixel 32k + j, set for -1
    h2 = np.ones(64)
    h2[33] = -1.0
    assert list(ospr.pack_bits(h2)) == [0, 2]


def test_binarise_tie_is_plus_one():
    assert list(ospr.binarise(np.array([0.0, -0.0, 1e-300, -1e-300]))) == [1, 1, 1, -1]


def test_twin_symmetry_and_energy():
    H, W, N = 32, 64, 3
    T, (bits, I, _) = _run(H, W, N, 1009)
    assert np.max(np.abs(I - _twin(I))) < 1e-9 * I.max()
    # each sub-frame carries energy P, so the average does too
    assert abs(I.sum() - H * W) < 1e-9 * H * W
    for s in range(N):
        Is = ospr.replay_intensity(ospr.unpack_bits(bits[s], H * W).reshape(H, W))
        assert abs(Is.sum() - H * W) < 1e-9 * H * W


def test_length_dividing_stride_repeats_subframes():
    H, W, N = 32, 32, 4
    T, (bits, I, _) = _run(H, W, N, 256)          # 256 divides P = 1024
    for s in range(1, N):
        assert np.array_equal(bits[s], bits[0])
    I1 = ospr.replay_from_bits(bits[:1], H, W)
    assert np.max(np.abs(I - I1)) < 1e-12 * I.max()
    # a prime length does not repeat
    T, (bits_p, _, _) = _run(H, W, N, 257)
    assert not np.array_equal(bits_p[1], bits_p[0])


def test_long_table_equals_generator():
    H, W, N = 16, 16, 3
    T = blob_target(H, W, 1001)
    P = H * W
    table = lut.lut_codes(5, N * P)
    b_lut, I_lut, _ = ospr.ospr(T, N, table, N * P, 5)
    b_gen, I_gen, _ = ospr.ospr(T, N, None, lut.UNREPEATED, 5)
    assert np.array_equal(b_lut, b_gen)
    assert np.array_equal(I_lut, I_gen)
    # a table of one sub-frame (L = P) matches the generator for sub-frame 0 only; later
    # sub-frames wrap onto the same draws, so they repeat sub-frame 0 (Section 5.1: the
    # equivalence needs N*P entries, not P)
    tableP = lut.lut_codes(5, P)
    b_p, _, _ = ospr.ospr(T, N, tableP, P, 5)
    assert np.array_equal(b_p[0], b_gen[0])
    for s in range(1, N):
        assert np.array_equal(b_p[s], b_p[0])
        assert not np.array_equal(b_p[s], b_gen[s])


def test_half_turn_inverts_bits_keeps_replay():
    H, W, N, L = 16, 32, 2, 101
    T = blob_target(H, W, 1002)
    table = lut.lut_codes(9, L)
    b0, I0, ex0 = ospr.ospr(T, N, table, L, 9, keep_fields=True)
    b1, I1, _ = ospr.ospr(T, N, (table + 128) % 256, L, 9)
    nonzero = np.all([np.all(np.abs(r) > 1e-12) for r in ex0["re_h"]])
    assert nonzero
    assert np.array_equal(b1, ~b0 & np.uint32(0xFFFFFFFF))
    assert np.max(np.abs(I1 - I0)) < 1e-12 * I0.max()


def _explicit_dft_matrix(n, sign):
    k = np.arange(n)
    return np.exp(sign * 2j * np.pi * np.outer(k, k) / n) / np.sqrt(n)


@pytest.mark.parametrize("H,W,N,L", [(4, 4, 1, 5), (4, 4, 3, 7), (8, 8, 2, 13), (8, 4, 3, 0)])
def test_chain_equals_explicit_matrix_dft(H, W, N, L):
    T = blob_target(H, W, 1003)
    seed = 21
    table = lut.lut_codes(seed, L) if L > 0 else None
    bits, I, ex = ospr.ospr(T, N, table, L, seed, keep_fields=True)
    Fr_inv, Fc_inv = _explicit_dft_matrix(H, +1), _explicit_dft_matrix(W, +1)
    Fr, Fc = _explicit_dft_matrix(H, -1), _explicit_dft_matrix(W, -1)
    P = H * W
    acc = np.zeros((H, W))
    for s in range(N):
        p = np.arange(P)
        if L > 0:
            c = table[(s * P + p) % L]
        else:
            c = np.zeros(P, dtype=int)
        E = T * np.exp(2j * np.pi * c.reshape(H, W) / 256)
        Hs = Fr_inv @ E @ Fc_inv.T
        assert np.max(np.abs(Hs.real - ex["re_h"][s])) < 1e-12
        h = np.where(Hs.real >= 0, 1.0, -1.0)
        assert np.array_equal(ospr.unpack_bits(bits[s], P).reshape(H, W), h)
        R = Fr @ h @ Fc.T
        acc += np.abs(R) ** 2
    assert np.max(np.abs(acc / N - I)) < 1e-12


def test_flat_phase_single_subframe_of_constant_target():
    # T = 1 everywhere with flat phase: IDFT is sqrt(P) at the origin and 0 elsewhere, so
    # Re H >= 0 everywhere -> h = +1 -> all energy in the DC bin: I[0,0] = P.
    H, W = 8, 16
    T = np.ones((H, W))
    bits, I, _ = ospr.ospr(T, 1, None, 0, 0)
    assert np.all(bits == 0)
    assert abs(I[0, 0] - H * W) < 1e-9
    assert np.sum(I) - I[0, 0] < 1e-9
