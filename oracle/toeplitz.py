"""The block Toeplitz product by its definition (test infrastructure only).

Definition (Sec. I, "extending the diagonal bands" example): for a d-level
block Toeplitz matrix with c x c blocks generated by t_ab[p],
p_m in [-(n_m - 1), n_m - 1], block (i, j) of T is t[i - j] (the 2x2 example
puts t21, offset +1, below the diagonal), so

    y_a[i] = sum_b sum_{j in grid} t_ab[i - j] x_b[j],   i in grid.

Storage: t[a][b][p_1 + n_1 - 1]...[p_d + n_d - 1];  x[r][b][j_1]...[j_d]
(a single vector may omit the leading r axis).
"""
from __future__ import annotations

import itertools

import numpy as np


def _as_rhs(x: np.ndarray, c: int, d: int):
    x = np.asarray(x, dtype=np.complex128)
    if x.ndim == d + 1:
        return x[None], True
    assert x.ndim == d + 2 and x.shape[1] == c
    return x, False


def grid_shape(t: np.ndarray):
    return tuple((m + 1) // 2 for m in t.shape[2:])


def dense_matrix(t: np.ndarray) -> np.ndarray:
    """Explicit (c*s) x (c*s) matrix, rows (a, i), columns (b, j), i and j in
    row-major grid order; entry = t_ab[i - j].  Tiny grids only."""
    c = t.shape[0]
    n = grid_shape(t)
    pts = list(itertools.product(*[range(m) for m in n]))
    s = len(pts)
    M = np.zeros((c * s, c * s), dtype=np.complex128)
    for ii, i in enumerate(pts):
        for jj, j in enumerate(pts):
            off = tuple(i[m] - j[m] + n[m] - 1 for m in range(len(n)))
            for a in range(c):
                for b in range(c):
                    M[a * s + ii, b * s + jj] = t[(a, b) + off]
    return M


def brute_force_matvec(t: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Pure-Python loops over i, j, a, b (tiny grids only)."""
    c = t.shape[0]
    n = grid_shape(t)
    d = len(n)
    xs, single = _as_rhs(x, c, d)
    y = np.zeros_like(xs)
    pts = list(itertools.product(*[range(m) for m in n]))
    for r in range(xs.shape[0]):
        for i in pts:
            for a in range(c):
                acc = 0j
                for j in pts:
                    off = tuple(i[m] - j[m] + n[m] - 1 for m in range(d))
                    for b in range(c):
                        acc += t[(a, b) + off] * xs[(r, b) + j]
                y[(r, a) + i] = acc
    return y[0] if single else y


def direct_matvec(t: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Direct summation, reordered as a sum over offsets p = i - j:
    y_a[i] += t_ab[p] x_b[i - p] for every i with i - p inside the grid.
    Cost prod(2n-1) * c^2 * s; fine up to about 64 x 64."""
    c = t.shape[0]
    n = grid_shape(t)
    d = len(n)
    xs, single = _as_rhs(x, c, d)
    y = np.zeros_like(xs)
    for p in itertools.product(*[range(-(m - 1), m) for m in n]):
        # output range i with i - p in [0, n): i in [max(0,p), min(n, n+p))
        osl = tuple(slice(max(0, p[m]), min(n[m], n[m] + p[m])) for m in range(d))
        isl = tuple(slice(max(0, p[m]) - p[m], min(n[m], n[m] + p[m]) - p[m]) for m in range(d))
        tp = t[(slice(None), slice(None)) + tuple(p[m] + n[m] - 1 for m in range(d))]
        xin = xs[(slice(None), slice(None)) + isl]          # [r][b][...]
        y[(slice(None), slice(None)) + osl] += np.einsum("ab,rb...->ra...", tp, xin)
    return y[0] if single else y


def direct_points(t: np.ndarray, x: np.ndarray, points) -> np.ndarray:
    """y_a[i] for the listed output points i (all components, all RHS).

    With the summation index reflected, j = n - 1 - j', the offset i - j has
    storage index i + j' (+ n - 1 - (n - 1)), so for a fixed i the
    coefficients form the forward box t[:, :, i : i + n] and the vector is
    read reflected: y_a[i] = sum_b sum_j' t_ab[i + j'] x_b[n - 1 - j'].
    Returns [npts][r][c].
    """
    c = t.shape[0]
    n = grid_shape(t)
    d = len(n)
    xs, single = _as_rhs(x, c, d)
    xr = np.ascontiguousarray(xs[(slice(None), slice(None)) + (slice(None, None, -1),) * d])
    out = np.zeros((len(points), xs.shape[0], c), dtype=np.complex128)
    letters = "ijklmn"[:d]
    expr = f"ab{letters},rb{letters}->ra"
    for k, i in enumerate(points):
        box = t[(slice(None), slice(None)) + tuple(slice(i[m], i[m] + n[m]) for m in range(d))]
        out[k] = np.einsum(expr, box, xr)
    return out[:, 0] if single else out
