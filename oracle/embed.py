"""Standard multilevel circulant embedding (test infrastructure only).

Sec. I: each Toeplitz level of size n is embedded in a 2n circulant by
"extending the diagonal bands", with one free entry s0 per level; the matvec
is then an FFT convolution on the 2^d-times larger grid followed by a
projection back to the original grid.  Along one level the first column of
the 2n circulant is

    c~[k] = t[k]        for 0 <= k < n,
    c~[n] = s0,
    c~[k] = t[k - 2n]   for n < k < 2n,

(the 2x2 -> 4x4 example: column (t11, t21, s0, t12)).  In d levels a point k
whose index equals n_m in any dimension is a free entry (s0 = 0 by default).

DFT convention: forward exp(-2 pi i f k / N), unnormalised; the symbol is
S = DFT_{2n}(c~) / prod(2 n_m), so that the embedded product is
y = IDFT_unnorm(S * DFT(pad(x))) restricted to the grid.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft

from .toeplitz import grid_shape


def _spatial_axes(arr: np.ndarray, d: int):
    return tuple(range(arr.ndim - d, arr.ndim))


def embedded_generator(t: np.ndarray, s0: complex = 0.0) -> np.ndarray:
    """c~[a][b][k_1..k_d] on the 2n grid, free entries set to s0."""
    c = t.shape[0]
    n = grid_shape(t)
    d = len(n)
    out = t
    for m in range(d):
        nm = n[m]
        k = np.arange(2 * nm)
        idx = np.where(k < nm, k + nm - 1, k - nm - 1)
        idx[nm] = 0                          # placeholder, overwritten below
        out = np.take(out, idx, axis=2 + m)
    out = np.array(out, dtype=np.complex128, copy=True)
    for m in range(d):
        sl = [slice(None)] * (2 + d)
        sl[2 + m] = n[m]
        out[tuple(sl)] = s0
    assert out.shape == (c, c) + tuple(2 * m for m in n)
    return out


def symbol(t: np.ndarray, s0: complex = 0.0, workers: int | None = None) -> np.ndarray:
    """S[a][b][f] = DFT_{2n}(c~_ab)[f] / prod(2 n_m), f in [0, 2n)^d."""
    n = grid_shape(t)
    d = len(n)
    ct = embedded_generator(t, s0)
    scale = 1.0 / float(np.prod([2 * m for m in n]))
    return sfft.fftn(ct, axes=_spatial_axes(ct, d), workers=workers) * scale


def embed_matvec(t: np.ndarray, x: np.ndarray, s0: complex = 0.0,
                 workers: int | None = None) -> np.ndarray:
    """y = T x via the full 2^d circulant embedding (plain method).

    pad x with zeros to the 2n grid, FFT, multiply per frequency by the c x c
    transformed generator, inverse FFT, keep the first n entries per dim.
    """
    c = t.shape[0]
    n = grid_shape(t)
    d = len(n)
    x = np.asarray(x, dtype=np.complex128)
    single = x.ndim == d + 1
    xs = x[None] if single else x
    r = xs.shape[0]
    big = tuple(2 * m for m in n)
    xp = np.zeros((r, c) + big, dtype=np.complex128)
    xp[(slice(None), slice(None)) + tuple(slice(0, m) for m in n)] = xs
    ax = _spatial_axes(xp, d)
    X = sfft.fftn(xp, axes=ax, workers=workers)
    C = sfft.fftn(embedded_generator(t, s0), axes=_spatial_axes(t, d), workers=workers)
    Y = np.einsum("ab...,rb...->ra...", C, X)
    y = sfft.ifftn(Y, axes=ax, workers=workers)
    y = y[(slice(None), slice(None)) + tuple(slice(0, m) for m in n)]
    return y[0] if single else np.ascontiguousarray(y)
