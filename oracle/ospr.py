"""One-Step Phase-Retrieval with binary sub-frames (paper Sections 2 and 3), float64.

Test infrastructure only (see the package docstring).

Section 2: a hologram is found by back-propagating the target replay field to the
diffraction plane, H = IDFT(R) (Eq. 2), and then moving every pixel to the nearest value
the SLM allows. OSPR (Section 2, Section 3) repeats this for N sub-frames, each with an
independent random phase on the target, and the eye averages the sub-frames' replay
intensities, which lowers the error. Here the SLM is binary phase (Section 5.2, the
ferroelectric device of Section 6): allowed values are +1 and -1.

Per sub-frame s (readings: sign(0) = +1; bit = 1 means -1; bits packed LSB-first):
    E    = T * exp(i*theta_s)          theta_s from the LUT draw rule (lut.subframe_codes)
    Hs   = IDFT(E)                     Eq. 2, unitary
    h_s  = +1 where Re Hs >= 0 else -1
    R_s  = DFT(h_s)                    Eq. 1, unitary
    I   += |R_s|^2 / N

Fresnel propagation (Section 2 names it as the near-field alternative to the Fourier far
field without giving a model). Reading: the single-transform discrete Fresnel model, the
replay of hologram h being R = Q2 * DFT(h * Q) with the quadratic phase
    Q(y, x) = exp(i*pi*kappa*((x - W/2)^2 + (y - H/2)^2)),   kappa = pitch^2 / (wavelength * z),
and Q2 a phase-only factor of the replay plane that an intensity replay cannot see. The
random target phase is taken relative to Q2, so back-propagation is Hs = conj(Q) * IDFT(E)
and the replay intensity is |DFT(h * Q)|^2. kappa = 0 is the Fourier case above.
"""

import numpy as np

from . import fft as _fft
from . import lut as _lut


def binarise(re_h):
    """h = +1 where Re H >= 0, else -1 (nearest of the two binary phase values)."""
    return np.where(np.asarray(re_h) >= 0.0, 1.0, -1.0)


def pack_bits(h):
    """Pack a +-1 raster into uint32 words: bit j of word w is pixel 32*w + j, 1 means -1."""
    flat = (np.asarray(h).reshape(-1) < 0).astype(np.uint64)
    P = flat.size
    nw = (P + 31) // 32
    padded = np.zeros(nw * 32, dtype=np.uint64)
    padded[:P] = flat
    weights = np.left_shift(np.uint64(1), np.arange(32, dtype=np.uint64))
    words = (padded.reshape(nw, 32) * weights).sum(axis=1)
    return words.astype(np.uint32)


def unpack_bits(words, P):
    """Inverse of pack_bits: uint32 words -> +-1 float64 raster of P pixels."""
    w = np.asarray(words, dtype=np.uint64)
    bits = (w[:, None] >> np.arange(32, dtype=np.uint64)) & np.uint64(1)
    bits = bits.reshape(-1)[:P]
    return np.where(bits == 1, -1.0, 1.0)


def subframe_field(target, codes, levels=256):
    """E = T * exp(i*theta): the randomised target of one sub-frame."""
    T = np.asarray(target, dtype=np.float64)
    theta = _lut.phase_of_codes(codes, levels).reshape(T.shape)
    return T * np.exp(1j * theta)


def back_propagate(E):
    """Hs = IDFT(E), Eq. 2."""
    return _fft.ifft2(E)


def replay_intensity(h):
    """|DFT(h)|^2 of one hologram (Eq. 1)."""
    R = _fft.fft2(h)
    return np.abs(R) ** 2


def replay_from_bits(bits, H, W):
    """Time-averaged replay (1/N) sum_s |DFT(h_s)|^2 of N packed binary sub-frames.

    ``bits`` has shape [N, ceil(H*W/32)].
    """
    bits = np.asarray(bits)
    N = bits.shape[0]
    I = np.zeros((H, W), dtype=np.float64)
    for s in range(N):
        h = unpack_bits(bits[s], H * W).reshape(H, W)
        I += replay_intensity(h)
    return I / N


def ospr(target, N, table, L, seed, start=0, stride=None, levels=256, keep_fields=False):
    """Run N OSPR sub-frames and return (bits [N, P/32] uint32, I [H, W] float64, extra).

    ``extra`` holds per-sub-frame Re Hs (float64) when keep_fields is set, so that a test
    can see how close to zero a pixel whose binarisation disagrees was.
    """
    T = np.asarray(target, dtype=np.float64)
    H, W = T.shape
    P = H * W
    if stride is None:
        stride = P
    bits = np.zeros((N, (P + 31) // 32), dtype=np.uint32)
    I = np.zeros((H, W), dtype=np.float64)
    re_fields = []
    for s in range(N):
        c = _lut.subframe_codes(table, L, seed, start, s, stride, P, levels)
        E = subframe_field(T, c, levels)
        Hs = back_propagate(E)
        h = binarise(Hs.real)
        bits[s] = pack_bits(h)
        I += replay_intensity(h)
        if keep_fields:
            re_fields.append(Hs.real.copy())
    I /= N
    extra = {"re_h": re_fields} if keep_fields else {}
    return bits, I, extra


# ------------------------------------------------------------------ Fresnel ----
def fresnel_chirp(H, W, kappa):
    """Q(y, x) = exp(i*pi*kappa*((x - W/2)^2 + (y - H/2)^2)), float64 complex [H, W]."""
    y = np.arange(H, dtype=np.float64) - H / 2
    x = np.arange(W, dtype=np.float64) - W / 2
    a = kappa * (y[:, None] ** 2 + x[None, :] ** 2)
    return np.exp(1j * np.pi * a)


def back_propagate_fresnel(E, kappa):
    """Hs = conj(Q) * IDFT(E): the diffraction-plane field whose Fresnel replay is E."""
    H, W = np.asarray(E).shape
    return np.conj(fresnel_chirp(H, W, kappa)) * _fft.ifft2(E)


def replay_intensity_fresnel(h, kappa):
    """|DFT(h * Q)|^2 of one hologram under Fresnel propagation."""
    h = np.asarray(h)
    H, W = h.shape
    return np.abs(_fft.fft2(h * fresnel_chirp(H, W, kappa))) ** 2


def replay_from_bits_fresnel(bits, H, W, kappa):
    """(1/N) sum_s |DFT(h_s * Q)|^2 of N packed binary sub-frames."""
    bits = np.asarray(bits)
    N = bits.shape[0]
    I = np.zeros((H, W), dtype=np.float64)
    for s in range(N):
        I += replay_intensity_fresnel(unpack_bits(bits[s], H * W).reshape(H, W), kappa)
    return I / N


def ospr_fresnel(target, N, table, L, seed, kappa, start=0, stride=None, levels=256, keep_fields=False):
    """OSPR with Fresnel propagation: (bits [N, P/32] uint32, I [H, W] float64, extra).

    Per sub-frame: E = T*exp(i*theta_s) (the same draw rule as ``ospr``),
    Hs = conj(Q) * IDFT(E), h_s = sign(Re Hs) with sign(0) = +1, I += |DFT(h_s * Q)|^2 / N.
    """
    T = np.asarray(target, dtype=np.float64)
    H, W = T.shape
    P = H * W
    if stride is None:
        stride = P
    bits = np.zeros((N, (P + 31) // 32), dtype=np.uint32)
    I = np.zeros((H, W), dtype=np.float64)
    re_fields = []
    for s in range(N):
        c = _lut.subframe_codes(table, L, seed, start, s, stride, P, levels)
        Hs = back_propagate_fresnel(subframe_field(T, c, levels), kappa)
        h = binarise(Hs.real)
        bits[s] = pack_bits(h)
        I += replay_intensity_fresnel(h, kappa)
        if keep_fields:
            re_fields.append(Hs.real.copy())
    I /= N
    extra = {"re_h": re_fields} if keep_fields else {}
    return bits, I, extra
