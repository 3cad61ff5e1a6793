"""Algorithm 1 (Sec. II.B) restated in NumPy (test infrastructure only).

Splitting property (Sec. II.A): for v of length n and v~ = [v, 0] of length
2n, the even coefficients of DFT_{2n}(v~) are DFT_n(v) and the odd ones are
DFT_n(P v), with the phase operator read as P[k] = exp(-i pi k / n),
k = 0..n-1 (the sign that matches the forward kernel exp(-2 pi i f k / N)).

Merge (Sec. II.A, applied as in Algorithm 1): after both branches have been
inverse transformed along a level, the projected result on that level is
v_even + conj(P) v_odd (unnormalised inverses; the single 1/prod(2 n_m) scale
lives in the symbol).

Tree (Algorithm 1): at level m > 0 transform along dimension m; if m is not
the last level, create the phase-shifted child along dimension m+1 (sptBrn),
recurse on the parent with the caller's branch id and on the child with the
id that marks dimension m+1 odd (nxtId), merge (mrgBrn); at the last level
multiply by the leaf part T[bId] of the symbol (mulBrn); finally inverse
transform along dimension m.  The leaf part for parity vector b is
S_b[l] = S[2 l + b] (the transformed embedded generator cut into 2^d parts,
Sec. II.C).
"""
from __future__ import annotations

import numpy as np

from .embed import symbol
from .toeplitz import grid_shape


def phase(n: int, odd: int) -> np.ndarray:
    """P_b[k] = exp(-i pi b k / n), k in [0, n)."""
    k = np.arange(n)
    return np.exp(-1j * np.pi * odd * k / n)


def _along(vec: np.ndarray, axis: int, ndim: int) -> np.ndarray:
    shape = [1] * ndim
    shape[axis] = vec.shape[0]
    return vec.reshape(shape)


def leaf_part(S: np.ndarray, b) -> np.ndarray:
    """S_b[a][a'][l] = S[a][a'][2 l + b] (strided slice per dimension)."""
    d = S.ndim - 2
    return S[(slice(None), slice(None)) + tuple(slice(b[m], None, 2) for m in range(d))]


def split_matvec(t: np.ndarray, x: np.ndarray, order=None) -> np.ndarray:
    """y = T x by the recursive split tree of Algorithm 1.

    ``order`` maps level m = 1..d to a physical dimension (a permutation of
    range(d)); the default is the natural order.  The result does not depend
    on it because the per-dimension operators commute.
    """
    c = t.shape[0]
    n = grid_shape(t)
    d = len(n)
    x = np.asarray(x, dtype=np.complex128)
    single = x.ndim == d + 1
    xs = x[None] if single else x
    order = list(range(d)) if order is None else list(order)
    S = symbol(t)
    nd = xs.ndim

    def axis_of(level):            # level in 1..d -> array axis
        return 2 + order[level - 1]

    def toe_mul_brn(level, bid, v):
        if level > 0:
            v = np.fft.fft(v, axis=axis_of(level))
        if level < d:
            ax = axis_of(level + 1)
            nm = n[order[level]]
            p = _along(phase(nm, 1), ax, nd)
            v_child = v * p                                   # sptBrn
            v = toe_mul_brn(level + 1, bid, v)
            child_id = list(bid)
            child_id[order[level]] = 1                        # nxtId
            v_child = toe_mul_brn(level + 1, tuple(child_id), v_child)
            v = v + np.conj(p) * v_child                      # mrgBrn
        else:
            Sb = leaf_part(S, bid)                            # T[bId]
            v = np.einsum("ab...,rb...->ra...", Sb, v)        # mulBrn
        if level > 0:
            ax = axis_of(level)
            v = np.fft.ifft(v, axis=ax) * v.shape[ax]         # unnormalised inverse
        return v

    y = toe_mul_brn(0, (0,) * d, xs)
    return y[0] if single else y


def split_flat(t: np.ndarray, x: np.ndarray) -> np.ndarray:
    """The tree unrolled: y = sum_b conj(P_b) IDFT_unnorm(S_b . DFT(P_b x)).

    P_b is the product of the per-dimension phases P_{b_m} along each dim.
    """
    c = t.shape[0]
    n = grid_shape(t)
    d = len(n)
    x = np.asarray(x, dtype=np.complex128)
    single = x.ndim == d + 1
    xs = x[None] if single else x
    S = symbol(t)
    axes = tuple(range(2, 2 + d))
    y = np.zeros_like(xs)
    for bits in range(1 << d):
        b = tuple((bits >> m) & 1 for m in range(d))
        Pb = np.ones(n, dtype=np.complex128)
        for m in range(d):
            Pb = Pb * _along(phase(n[m], b[m]), m, d)
        X = np.fft.fftn(xs * Pb, axes=axes)
        Y = np.einsum("ab...,rb...->ra...", leaf_part(S, b), X)
        y += np.conj(Pb) * np.fft.ifftn(Y, axes=axes) * float(np.prod(n))
    return y[0] if single else y
