"""Pins of the m-sequence code oracle (Section 7's PRNG alternative): the register, the
output recurrence and the jump-ahead agree; a small primitive register gives a full-period,
balanced m-sequence; x^31 + x^3 + 1 is primitive; codes pack bits most significant first."""

import numpy as np

from oracle import lfsr


def test_small_register_is_an_m_sequence():
    poly = (1 << 7) | (1 << 1) | 1            # x^7 + x + 1, primitive
    b = lfsr.bits_by_stepping(1, 3 * 127, poly)
    assert np.array_equal(b[:127], b[127:254]) and np.array_equal(b[:127], b[254:])
    assert b[:127].sum() == 64                 # 2^(n-1) ones, 2^(n-1) - 1 zeros
    # no shorter period: the 127 cyclic shifts are distinct
    shifts = {tuple(np.roll(b[:127], t)) for t in range(127)}
    assert len(shifts) == 127
    # every nonzero 7-bit window occurs exactly once per period
    w = [int("".join(map(str, np.roll(b[:127], -t)[:7])), 2) for t in range(127)]
    assert sorted(w) == list(range(1, 128))


def test_three_constructions_agree():
    for poly in (lfsr.POLY31, (1 << 7) | (1 << 1) | 1, (1 << 17) | (1 << 3) | 1):
        for s0 in (1, 0x1234567 & ((1 << lfsr.degree(poly)) - 1) or 1):
            a = lfsr.bits_by_stepping(s0, 3000, poly)
            assert np.array_equal(a, lfsr.bits_by_recurrence(s0, 3000, poly))
            s = s0
            for k in range(3000):
                if k in (0, 1, 30, 31, 997, 2999):
                    assert lfsr.jump(s0, k, poly) == s
                s = lfsr.step(s, poly)
    # far jumps: stepping from a jumped state continues the same sequence
    s = lfsr.jump(5, 123456)
    b = lfsr.bits_by_stepping(s, 64)
    assert np.array_equal(b, lfsr.bits_by_recurrence(5, 123456 + 64)[123456:])


def test_degree_31_polynomial_is_primitive():
    # 2^31 - 1 is a Mersenne prime, so x has order 2^31 - 1 exactly when x^(2^31-1) = 1
    assert lfsr.order_of_x(lfsr.POLY31, [2 ** 31 - 1])
    assert not lfsr.order_of_x((1 << 31) | (1 << 2) | 1, [2 ** 31 - 1])  # x^31+x^2+1: not primitive


def test_codes_pack_bits_msb_first():
    b = lfsr.bits_by_stepping(77, 8 * 20)
    c = lfsr.codes(77, 0, 20)
    for i in range(20):
        assert c[i] == int("".join(str(x) for x in b[8 * i:8 * i + 8]), 2)
    # continuation: codes from a later start equal the tail of a longer run
    assert np.array_equal(lfsr.codes(77, 7, 13), c[7:20])
    c2 = lfsr.codes(77, 3, 5, levels=4)
    b2 = lfsr.bits_by_stepping(77, 2 * 8)
    assert list(c2) == [2 * b2[2 * i] + b2[2 * i + 1] for i in range(3, 8)]
