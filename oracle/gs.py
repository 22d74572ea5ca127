"""Gerchberg-Saxton with a phase-quantised hologram (paper Section 2), float64.

Test infrastructure only (see the package docstring).

Section 2: GS alternates between the replay plane and the diffraction plane. In the
diffraction plane the hologram is moved to the nearest value the SLM allows; in the
replay plane the amplitude is reset to the target while the phase found so far is kept.
Section 3: the initial replay-plane phase is random (here: from the LUT draw rule with
s = 0), which diffuses the light and avoids edge enhancement. Section 8 notes that only
the prime-length and longer-than-the-image-dimension rules apply to GS.

Readings (the flowchart of Fig. 2 is missing from the text):
  * T_s = T * sqrt(P / sum T^2): the target scaled to the energy of a unit-modulus
    hologram of P pixels, so that both planes hold the same energy (Parseval).
  * phase quantiser with ``levels`` levels: q = floor(levels*arg(H)/(2*pi) + 1/2) mod
    levels, arg from atan2 in (-pi, pi]; the hologram pixel is exp(i*2*pi*q/levels).
    levels = 2 is the binary-phase device (values +1, -1).
  * arg(0) := 0, both for H and for R.
  * error of iteration k: eps_k = sum_p (|R_k| - T_s)^2.
Iteration k = 1..K:
    H = IDFT(E);  q = quantise(arg H);  h = exp(i*2*pi*q/levels);  R = DFT(h);
    eps_k = sum (|R| - T_s)^2;  E = T_s * exp(i*arg R)
Returns the codes q and intensity |R|^2 of the last iteration and all eps_k.

Fresnel propagation (``gs_fresnel``): the same iteration with the propagation pair of
the Fresnel model in ospr.py, H = conj(Q) * IDFT(E) and R = DFT(h * Q); both are unitary,
so the projection argument behind the non-increasing error carries over.
"""

import numpy as np

from . import fft as _fft
from . import lut as _lut
from .ospr import fresnel_chirp


def energy_scaled_target(target):
    T = np.asarray(target, dtype=np.float64)
    P = T.size
    return T * np.sqrt(P / np.sum(T * T))


def quantise_phase(Hf, levels=256):
    """q = floor(levels*arg(H)/(2 pi) + 1/2) mod levels, arg(0) = 0."""
    ang = np.arctan2(Hf.imag, Hf.real)          # atan2(0, 0) = 0
    q = np.floor(levels * ang / (2.0 * np.pi) + 0.5).astype(np.int64)
    return np.mod(q, levels)


def hologram_of_codes(q, levels=256):
    return np.exp(1j * 2.0 * np.pi * np.asarray(q, dtype=np.float64) / levels)


def amplitude_constraint(R, Ts):
    """E = T_s * exp(i*arg R), with arg 0 = 0 (so E = T_s where R = 0)."""
    ang = np.arctan2(R.imag, R.real)
    return Ts * np.exp(1j * ang)


def initial_field(target, table, L, seed, start=0, lut_levels=256, init_phase=None):
    """E_0 = T_s * exp(i*theta): LUT phases drawn for s = 0, or a caller-given phase.

    The table holds phase codes of ``lut_levels`` levels (8-bit codes, Section 5.2); they
    are independent of the levels the hologram is quantised to.
    """
    Ts = energy_scaled_target(target)
    H, W = Ts.shape
    if init_phase is not None:
        theta = np.asarray(init_phase, dtype=np.float64).reshape(H, W)
    else:
        c = _lut.subframe_codes(table, L, seed, start, 0, H * W, H * W, lut_levels)
        theta = _lut.phase_of_codes(c, lut_levels).reshape(H, W)
    return Ts * np.exp(1j * theta)


def replay_phase(E):
    """The replay-plane phase of a GS state E (the warm start's training label): arg E in
    (-pi, pi], with arg 0 := 0 as everywhere in GS."""
    E = np.asarray(E, dtype=np.complex128)
    ang = np.arctan2(E.imag, E.real)
    return np.where((E.real == 0) & (E.imag == 0), 0.0, ang)


def gs_step(E, Ts, levels=256):
    """One GS iteration from replay-plane field E. Returns (q, R, eps, E_next)."""
    Hf = _fft.ifft2(E)
    q = quantise_phase(Hf, levels)
    h = hologram_of_codes(q, levels)
    R = _fft.fft2(h)
    eps = float(np.sum((np.abs(R) - Ts) ** 2))
    return q, R, eps, amplitude_constraint(R, Ts)


def gs(target, iters, table, L, seed, start=0, levels=256, init_phase=None, init_field=None,
       lut_levels=256):
    """K iterations. Returns (q [H,W] int64, I = |R|^2 [H,W], eps [K], E_state [H,W]).

    ``levels`` is the hologram's phase quantisation; ``lut_levels`` the table codes' levels.
    """
    Ts = energy_scaled_target(target)
    if init_field is not None:
        E = np.asarray(init_field, dtype=np.complex128)
    else:
        E = initial_field(target, table, L, seed, start, lut_levels, init_phase)
    errs = []
    q = R = None
    for _ in range(iters):
        q, R, eps, E = gs_step(E, Ts, levels)
        errs.append(eps)
    return q, np.abs(R) ** 2, np.array(errs), E


def gs_step_fresnel(E, Ts, kappa, levels=256):
    """One GS iteration under Fresnel propagation. Returns (q, R, eps, E_next)."""
    H, W = np.asarray(E).shape
    Q = fresnel_chirp(H, W, kappa)
    Hf = np.conj(Q) * _fft.ifft2(E)
    q = quantise_phase(Hf, levels)
    R = _fft.fft2(hologram_of_codes(q, levels) * Q)
    eps = float(np.sum((np.abs(R) - Ts) ** 2))
    return q, R, eps, amplitude_constraint(R, Ts)


def gs_fresnel(target, iters, table, L, seed, kappa, start=0, levels=256, init_phase=None, lut_levels=256):
    """K iterations under Fresnel propagation; returns as ``gs``."""
    Ts = energy_scaled_target(target)
    E = initial_field(target, table, L, seed, start, lut_levels, init_phase)
    errs = []
    q = R = None
    for _ in range(iters):
        q, R, eps, E = gs_step_fresnel(E, Ts, kappa, levels)
        errs.append(eps)
    return q, np.abs(R) ** 2, np.array(errs), E
