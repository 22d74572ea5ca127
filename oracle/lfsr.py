"""M-sequence phase codes: the PRNG alternative that Section 7 weighs against the LUT
(a fast m-sequence generator feeding a sine/cosine table).

Test infrastructure only (see the package docstring).

Reading (the paper names the technique, not a construction): a Galois linear feedback
shift register over GF(2) with a primitive feedback polynomial p(x) of degree n. Its state
after k steps is s_k = s_0 * x^k mod p(x) for a nonzero seed state s_0 (bit j of an
integer holds the coefficient of x^j); output bit k is the coefficient of x^(n-1) in s_k.
Because p is primitive the bits form an m-sequence of period 2^n - 1. Phase code i, for
levels = 2^m, packs bits m*i .. m*i + m - 1 most significant first; its phase is
2*pi*code/levels as for the LUT (the sine/cosine table of Section 7). The default
polynomial is x^31 + x^3 + 1 (primitive: see ``order_of_x``).

Three independent ways to the same bits are kept so that each pins the others:
``step`` (the register itself), ``bits_by_recurrence`` (the output sequence's own linear
recurrence b_{k+n} = sum of b_{k+j} over the non-leading terms x^j of p) and ``jump``
(s_0 * x^k mod p by square-and-multiply).
"""

import numpy as np

POLY31 = (1 << 31) | (1 << 3) | 1      # x^31 + x^3 + 1
DEGREE31 = 31


def degree(poly):
    return int(poly).bit_length() - 1


def step(s, poly):
    """One Galois step: s -> x*s mod p."""
    n = degree(poly)
    s <<= 1
    if (s >> n) & 1:
        s ^= poly
    return s


def output_bit(s, poly):
    return (s >> (degree(poly) - 1)) & 1


def bits_by_stepping(s0, count, poly=POLY31):
    """Output bits 0 .. count-1 of the register started at s0 (one step per bit)."""
    out = np.empty(count, dtype=np.uint8)
    s = int(s0)
    for k in range(count):
        out[k] = output_bit(s, poly)
        s = step(s, poly)
    return out


def bits_by_recurrence(s0, count, poly=POLY31):
    """The same bits from the sequence's linear recurrence: the first n bits by stepping,
    then b_{k+n} = XOR of b_{k+j} over the terms x^j (j < n) of p, since
    x^n = sum of those x^j modulo p. Blocks of n - (largest such j) bits depend only on
    bits already known."""
    n = degree(poly)
    taps = [j for j in range(n) if (poly >> j) & 1]
    m = n - max(taps)
    b = np.zeros(count + n, dtype=np.uint8)
    b[:n] = bits_by_stepping(s0, n, poly)
    k = 0
    while k + n < count:
        w = min(m, count - n - k)
        acc = np.zeros(w, dtype=np.uint8)
        for j in taps:
            acc ^= b[k + j:k + j + w]
        b[k + n:k + n + w] = acc
        k += w
    return b[:count]


def mulmod(a, b, poly):
    """a * b mod p over GF(2) (carry-less product, then reduction)."""
    n = degree(poly)
    r = 0
    a = int(a)
    b = int(b)
    while b:
        if b & 1:
            r ^= a
        b >>= 1
        a <<= 1
        if (a >> n) & 1:
            a ^= poly
    return r


def jump(s0, k, poly=POLY31):
    """s_0 * x^k mod p by square-and-multiply."""
    r = int(s0)
    x_pow = 2                              # the polynomial x
    while k:
        if k & 1:
            r = mulmod(r, x_pow, poly)
        x_pow = mulmod(x_pow, x_pow, poly)
        k >>= 1
    return r


def order_of_x(poly, n_divisors):
    """Checks that x has order exactly 2^n - 1 modulo p, given the prime divisors of 2^n - 1
    (for n = 31, 2^31 - 1 is prime): x^(2^n - 1) = 1 and x^((2^n - 1)/q) != 1 for every
    prime q dividing it. True means p is primitive."""
    n = degree(poly)
    e = (1 << n) - 1
    if jump(1, e, poly) != 1:
        return False
    return all(jump(1, e // q, poly) != 1 for q in n_divisors)


def codes(s0, start, count, levels=256, poly=POLY31):
    """Codes start .. start+count-1: code i packs bits m*i .. m*i+m-1, MSB first."""
    m = int(levels).bit_length() - 1
    if levels < 2 or levels > 256 or (1 << m) != levels:
        raise ValueError("levels must be a power of two in [2, 256]")
    s = jump(s0, m * int(start), poly)
    b = bits_by_recurrence(s, m * int(count), poly).astype(np.int64).reshape(count, m)
    weights = 1 << np.arange(m - 1, -1, -1)
    return (b * weights).sum(axis=1)
