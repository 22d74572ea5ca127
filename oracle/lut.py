"""The phase lookup table ("pool") and its cyclic draw rule (paper Sections 4 and 5, Fig. 3).

Test infrastructure only (see the package docstring).

Section 4: random numbers are generated once, at compile time, into a table of N_LUT
entries that algorithms then draw from sequentially. Section 5 (Fig. 3): the pool is
cycled through, and successive sub-frames and frames continue where the previous one
stopped. Section 5.2: a table for 256x256 pixels and 24 sub-frames would need "over
12 Mb", i.e. 256*256*24 entries of 8 bits, so each entry is an 8-bit phase code.

Readings of what the paper leaves open:
  * generator: SplitMix64 (Steele, Lea and Flood, OOPSLA 2014). Its k-th output (k from
    0) is mix(seed + (k+1)*0x9E3779B97F4A7C15); being counter based, draw i of the
    "unrepeated" case (no table) is simply output i, so an infinitely long table and the
    unrepeated generator give the same codes.
  * code: the top log2(levels) bits of the 64-bit output; levels = 256 by default;
    the phase of code c is theta = 2*pi*c/levels.
  * draw index for sub-frame s, pixel p = r*W + c (row-major, column fastest):
    i = start + s*stride + p with stride = H*W (continuation, Fig. 3). With a table of
    length L the code is table[i mod L]. L = 0 means no randomisation (flat phase,
    theta = 0), the edge-enhanced case of Section 3.
"""

import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)

UNREPEATED = -1   # L value meaning "no table: draw i uses generator output i directly"


def splitmix64(seed, k):
    """k-th SplitMix64 output (k = 0, 1, ...) for the stream started at ``seed``.

    z = seed + (k + 1) * gamma (mod 2^64); z ^= z >> 30; z *= M1; z ^= z >> 27; z *= M2;
    z ^= z >> 31.  Arithmetic is modulo 2^64 (numpy uint64 wraps).
    """
    k = np.asarray(k, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (k + np.uint64(1)) * GOLDEN_GAMMA
        z = (z ^ (z >> np.uint64(30))) * _MIX1
        z = (z ^ (z >> np.uint64(27))) * _MIX2
        z = z ^ (z >> np.uint64(31))
    return z


def code_bits(levels):
    if levels < 2 or levels > 256 or (levels & (levels - 1)) != 0:
        raise ValueError("levels must be a power of two in [2, 256]")
    return levels.bit_length() - 1


def codes_from_draws(seed, i, levels=256):
    """Phase code of generator draw(s) i: the top log2(levels) bits of SplitMix64."""
    b = code_bits(levels)
    return (splitmix64(seed, i) >> np.uint64(64 - b)).astype(np.int64)


def lut_codes(seed, L, levels=256):
    """The table itself: entry k holds the code of generator draw k, k in [0, L)."""
    if L < 0:
        raise ValueError("a table needs L >= 0")
    return codes_from_draws(seed, np.arange(L, dtype=np.uint64), levels)


def draw_indices(start, s, stride, P):
    """Draw index of every pixel of sub-frame s: i_p = start + s*stride + p, p in [0, P)."""
    base = int(start) + int(s) * int(stride)
    return base + np.arange(P, dtype=np.int64)


def subframe_codes(table, L, seed, start, s, stride, P, levels=256):
    """Codes c_p for sub-frame s (Fig. 3 draw rule).

    L > 0: table[(start + s*stride + p) mod L]; L = 0: all zeros (flat phase);
    L = UNREPEATED: codes_from_draws(seed, start + s*stride + p).
    """
    i = draw_indices(start, s, stride, P)
    if L == 0:
        return np.zeros(P, dtype=np.int64)
    if L == UNREPEATED:
        return codes_from_draws(seed, i.astype(np.uint64), levels)
    table = np.asarray(table, dtype=np.int64)
    if table.shape != (L,):
        raise ValueError("table length must equal L")
    return table[np.mod(i, L)]


def phase_of_codes(c, levels=256):
    """theta = 2*pi*c/levels in float64."""
    return 2.0 * np.pi * np.asarray(c, dtype=np.float64) / float(levels)
