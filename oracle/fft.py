"""Unitary 2D DFT and inverse DFT in float64 (paper Section 2, Eq. 1 and Eq. 2).

Test infrastructure only (see the package docstring).

Eq. 1:  F[u, v] = 1/sqrt(Nx*Ny) * sum_x sum_y f[x, y] * exp(-2*pi*i*(u*x/Nx + v*y/Ny))
Eq. 2:  f[x, y] = 1/sqrt(Nx*Ny) * sum_u sum_v F[u, v] * exp(+2*pi*i*(u*x/Nx + v*y/Ny))

Two routes are given:
  * ``dft2_brute`` / ``idft2_brute`` write Eq. 1 / Eq. 2 out as a double sum over an
    explicit exponential matrix: O(P^2), used only on tiny arrays to pin the FFT.
  * ``fft2`` / ``ifft2`` evaluate the same sums with an iterative radix-2 Cooley-Tukey
    FFT (the O(N log N) route the paper cites in Section 2), one axis at a time.

Arrays are indexed [row, column]; the transform is separable so the axis order does not
change the result.
"""

import functools

import numpy as np


def _check_pow2(n):
    if n < 1 or (n & (n - 1)) != 0:
        raise ValueError(f"radix-2 FFT needs a power-of-two length, got {n}")


@functools.lru_cache(maxsize=None)
def _bit_reverse_permutation(n):
    """Index array j -> bit-reversed j over log2(n) bits."""
    bits = n.bit_length() - 1
    rev = np.zeros(n, dtype=np.int64)
    for j in range(n):
        r = 0
        v = j
        for _ in range(bits):
            r = (r << 1) | (v & 1)
            v >>= 1
        rev[j] = r
    return rev


def fft_radix2_lastaxis(x, sign):
    """Unnormalised DFT along the last axis: X[k] = sum_n x[n] exp(sign*2*pi*i*n*k/n_len).

    Iterative decimation-in-time: reorder the input into bit-reversed order, then merge
    pairs of half-length transforms with butterflies of growing size 2, 4, ..., n.
    ``sign`` is -1 for Eq. 1 (forward) and +1 for Eq. 2 (inverse).
    """
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[-1]
    _check_pow2(n)
    a = x[..., _bit_reverse_permutation(n)].copy()
    lead = a.shape[:-1]
    size = 2
    while size <= n:
        half = size // 2
        k = np.arange(half, dtype=np.float64)
        w = np.exp(sign * 2j * np.pi * k / size)          # twiddles of this butterfly size
        a = a.reshape(lead + (n // size, size))
        top = a[..., :half].copy()
        bottom = a[..., half:] * w
        a[..., :half] = top + bottom
        a[..., half:] = top - bottom
        a = a.reshape(lead + (n,))
        size *= 2
    return a


def _fft2_unitary(f, sign):
    f = np.asarray(f, dtype=np.complex128)
    if f.ndim != 2:
        raise ValueError("expected a 2D array")
    ny, nx = f.shape
    g = fft_radix2_lastaxis(f, sign)                        # along columns index (axis 1)
    g = fft_radix2_lastaxis(g.T, sign).T                    # along rows index (axis 0)
    return g / np.sqrt(float(nx * ny))


def fft2(f):
    """Eq. 1: unitary forward 2D DFT via radix-2 FFT."""
    return _fft2_unitary(f, -1)


def ifft2(F):
    """Eq. 2: unitary inverse 2D DFT via radix-2 FFT."""
    return _fft2_unitary(F, +1)


def _dft_matrix(n, sign):
    j = np.arange(n, dtype=np.float64)
    return np.exp(sign * 2j * np.pi * np.outer(j, j) / n)


def dft2_brute(f):
    """Eq. 1 written out: F[u,v] = P^-1/2 sum_{x,y} f[x,y] e^{-2 pi i (u x/Nx + v y/Ny)}.

    O(P^2) explicit double sum, for arrays of at most a few thousand pixels.
    """
    f = np.asarray(f, dtype=np.complex128)
    ny, nx = f.shape
    if ny * nx > 4096:
        raise ValueError("brute-force DFT is for tiny arrays only")
    out = np.zeros((ny, nx), dtype=np.complex128)
    Mr = _dft_matrix(ny, -1)
    Mc = _dft_matrix(nx, -1)
    for u in range(ny):
        for v in range(nx):
            out[u, v] = np.sum(f * np.outer(Mr[u], Mc[v]))
    return out / np.sqrt(float(nx * ny))


def idft2_brute(F):
    """Eq. 2 written out, the same double sum with +i."""
    F = np.asarray(F, dtype=np.complex128)
    ny, nx = F.shape
    if ny * nx > 4096:
        raise ValueError("brute-force DFT is for tiny arrays only")
    out = np.zeros((ny, nx), dtype=np.complex128)
    Mr = _dft_matrix(ny, +1)
    Mc = _dft_matrix(nx, +1)
    for x in range(ny):
        for y in range(nx):
            out[x, y] = np.sum(F * np.outer(Mr[x], Mc[y]))
    return out / np.sqrt(float(nx * ny))
