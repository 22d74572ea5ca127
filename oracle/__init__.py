"""FP64 CPU oracle for LUT phase randomisation, OSPR and GS (arXiv 2004.04049).

This package is TEST INFRASTRUCTURE. It is a plain, slow, obviously-correct restatement
of what the paper's method computes, written in float64 numpy with its own radix-2 FFT.
Only the tests, the smoke check in ``__graft_entry__`` and the CPU-baseline leg of
``bench.py`` may import it. The CUDA library never calls it, and it shares no code,
table or constant with the CUDA library: each side implements the published SplitMix64
generator and the DFT of Eq. 1-2 on its own.

Modules
-------
fft    unitary 2D DFT / IDFT (Eq. 1, Eq. 2): brute-force definition and radix-2 FFT.
lut    the phase LUT "pool" (Section 4) drawn cyclically with continuation (Section 5, Fig. 3).
lfsr   m-sequence phase codes, the PRNG alternative Section 7 compares the LUT with.
ospr   One-Step Phase-Retrieval with binary sub-frames (Section 2, Section 3).
gs     Gerchberg-Saxton with a phase-quantised hologram (Section 2).
error  MSE / NMSE of a replay field against its target (Section 5.2, Eq. 3).
conv   the warm-start network's conv layers, forward and backward, in float64.

Readings of points the paper leaves open are listed in the design notes and repeated in
each function's docstring.
"""

from . import conv, fft, lfsr, lut, ospr, gs, error  # noqa: F401
