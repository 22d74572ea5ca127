"""Replay-field error (paper Section 5.2 and Eq. 3), float64.

Test infrastructure only (see the package docstring).

The paper reports a time-averaged MSE of the replay field (Section 5.2) and normalises
it per test image (Eq. 3). It does not say which quantity the MSE is taken over or at
what scale. Reading used here: the intensity domain, comparing the averaged replay
intensity I with the target intensity T^2 after the least-squares optimal scale alpha:

    alpha = sum(I*T^2) / sum(I^2)
    MSE   = (1/P) * sum (alpha*I - T^2)^2
    NMSE  = sum (alpha*I - T^2)^2 / sum T^4        (per-target normalisation)

An optional 0/1 mask restricts every sum (and P) to the masked pixels.

Eq. 3 divides each image's MSE by that image's MSE at a reference LUT length and
multiplies by the Mandrill image's: the images are not available, so ``paper_nmse``
normalises by the same target's MSE without a table (the unrepeated generator).
"""

import numpy as np


def replay_error(I, T, mask=None):
    """Returns (alpha, mse, nmse) as Python floats, two passes in float64."""
    I = np.asarray(I, dtype=np.float64).reshape(-1)
    T2 = np.asarray(T, dtype=np.float64).reshape(-1) ** 2
    if mask is not None:
        m = np.asarray(mask).reshape(-1) != 0
        I = I[m]
        T2 = T2[m]
    P = I.size
    s_it = float(np.sum(I * T2))
    s_ii = float(np.sum(I * I))
    s_tt = float(np.sum(T2 * T2))
    alpha = s_it / s_ii if s_ii > 0.0 else 0.0
    d = alpha * I - T2
    sse = float(np.sum(d * d))
    mse = sse / P if P > 0 else 0.0
    nmse = sse / s_tt if s_tt > 0.0 else 0.0
    return alpha, mse, nmse


def paper_nmse(mse_with_lut, mse_unrepeated):
    """Eq. 3 with the target's own unrepeated-generator MSE as the reference."""
    return float(np.mean(mse_with_lut)) / float(np.mean(mse_unrepeated))
