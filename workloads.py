"""Seeded synthetic inputs for block Toeplitz matvec tests and benchmarks.

This module only *draws inputs*: generating coefficients t and vectors x.
It contains none of the matvec method's arithmetic (no embedding, no FFT,
no Toeplitz product), so both the CPU oracle's callers and the GPU path's
callers can use it without sharing method code.

Conventions
-----------
* A d-level generator with c x c blocks is stored over all offsets as a
  complex128 array ``t[a][b][p_1 + n_1 - 1]...[p_d + n_d - 1]`` with
  ``p_m in [-(n_m-1), n_m-1]`` (block (i, j) of T holds ``t[i - j]``).
* With per-dimension parity, only the non-negative orthant
  ``t_orth[a][b][p_1]...[p_d]`` (``p_m in [0, n_m)``) is stored, and
  ``parity[a][b][m] in {+1, -1}`` gives ``t(.., -p_m, ..) = parity * t(.., p_m, ..)``.
* Vectors are ``x[r][c][n_1]...[n_d]`` (r right-hand sides), last index fastest.
* Complex normal means real and imaginary parts i.i.d. N(0, 1), drawn from
  ``numpy.random.default_rng(seed)`` (PCG64).  The paper's experiments use
  random complex coefficients and vectors with zero-mean real and imaginary
  parts (Sec. III); the Green-function workloads are physical kernels of the
  kind the paper targets (Sec. I, electromagnetic Green function).
"""
from __future__ import annotations

import math

import numpy as np


def complex_normal(rng: np.random.Generator, shape) -> np.ndarray:
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return re + 1j * im


def offsets_shape(n) -> tuple:
    return tuple(2 * int(m) - 1 for m in n)


# --------------------------------------------------------------------------
# generators over all offsets
# --------------------------------------------------------------------------

def random_generator(n, c: int, seed: int) -> np.ndarray:
    """I.i.d. complex normal t_ab[p] over all offsets (no symmetry)."""
    rng = np.random.default_rng(seed)
    return complex_normal(rng, (c, c) + offsets_shape(n))


def random_vector(n, c: int, seed: int, nrhs: int = 1) -> np.ndarray:
    """I.i.d. complex normal x[r][c][n_1..n_d] (complex128)."""
    rng = np.random.default_rng(seed)
    return complex_normal(rng, (nrhs, c) + tuple(int(m) for m in n))


def orthant_to_full(t_orth: np.ndarray, parity: np.ndarray) -> np.ndarray:
    """Expand an orthant-stored parity generator to the all-offsets layout.

    t(.., -p_m, ..) = parity[a][b][m] * t(.., p_m, ..) for every dim m.
    """
    c = t_orth.shape[0]
    n = t_orth.shape[2:]
    d = len(n)
    full = np.zeros((c, c) + offsets_shape(n), dtype=np.complex128)
    for a in range(c):
        for b in range(c):
            blk = t_orth[a, b]
            out = np.zeros(offsets_shape(n), dtype=np.complex128)
            # fill each sign pattern of the 2^d orthants
            for mask in range(1 << d):
                src = blk
                sign = 1.0
                sl = []
                for m in range(d):
                    nm = n[m]
                    if (mask >> m) & 1:
                        # negative side p = -1..-(n-1) <- orthant p = 1..n-1
                        src = np.flip(np.take(src, np.arange(1, nm), axis=m), axis=m)
                        sign *= float(parity[a, b, m])
                        sl.append(slice(0, nm - 1))
                    else:
                        sl.append(slice(nm - 1, 2 * nm - 1))
                out[tuple(sl)] = sign * src
            full[a, b] = out
    return full


# --------------------------------------------------------------------------
# Green dyadic (electromagnetic) generator
# --------------------------------------------------------------------------

def green_dyadic_orthant(n, kh: float, h: float = 1.0):
    """Dyadic Green function blocks on the non-negative offset orthant.

    G_ab(r) = g(R) [ (1 + i/(kR) - 1/(kR)^2) delta_ab
                     - (1 + 3i/(kR) - 3/(kR)^2) rhat_a rhat_b ],
    g(R) = exp(i k R) / (4 pi R),  R = h |r|,  self term G(0) = identity.

    Requires d == 3 (three spatial axes, c = 3 components).  Returns
    (t_orth[3][3][n1][n2][n3], parity[3][3][3]): diagonal components are even
    in every dimension; the off-diagonal component ab is odd in dims a and b
    and even in the third.  t_ab = t_ba.
    """
    n = tuple(int(m) for m in n)
    assert len(n) == 3, "dyadic Green generator is three-dimensional"
    k = kh / h
    p = np.meshgrid(*[np.arange(m, dtype=np.float64) for m in n], indexing="ij")
    dist = np.sqrt(p[0] ** 2 + p[1] ** 2 + p[2] ** 2)
    R = h * dist
    self_pt = dist == 0
    Rs = np.where(self_pt, 1.0, R)
    kR = k * Rs
    g = np.exp(1j * kR) / (4.0 * math.pi * Rs)
    alpha = g * (1.0 + 1j / kR - 1.0 / kR ** 2)
    beta = g * (1.0 + 3j / kR - 3.0 / kR ** 2)
    distn = np.where(self_pt, 1.0, dist)
    rhat = [pm / distn for pm in p]
    t = np.zeros((3, 3) + n, dtype=np.complex128)
    for a in range(3):
        for b in range(3):
            v = -beta * rhat[a] * rhat[b]
            if a == b:
                v = v + alpha
            v = np.where(self_pt, 1.0 if a == b else 0.0, v)
            t[a, b] = v
    parity = np.ones((3, 3, 3), dtype=np.int8)
    for a in range(3):
        for b in range(3):
            if a != b:
                parity[a, b, a] = -1
                parity[a, b, b] = -1
    return t, parity


def green_scalar_orthant(n, kh: float, h: float = 1.0):
    """Scalar Green function g(R) = exp(ikR)/(4 pi R) on the offset orthant.

    Any dimension d, c = 1, self term 1, even in every dimension.
    Returns (t_orth[1][1][n...], parity[1][1][d] of +1).
    """
    n = tuple(int(m) for m in n)
    k = kh / h
    p = np.meshgrid(*[np.arange(m, dtype=np.float64) for m in n], indexing="ij")
    dist = np.sqrt(sum(pm ** 2 for pm in p))
    self_pt = dist == 0
    Rs = np.where(self_pt, 1.0, h * dist)
    g = np.exp(1j * k * Rs) / (4.0 * math.pi * Rs)
    g = np.where(self_pt, 1.0 + 0j, g)
    t = g.reshape((1, 1) + n).astype(np.complex128)
    parity = np.ones((1, 1, len(n)), dtype=np.int8)
    return t, parity


def skew_orthant(n, seed: int, c: int = 3):
    """Random block-symmetric generator odd in every dimension.

    t_ab = t_ba, t(-p) = -t(p) along each dim separately (so every plane
    p_m = 0 is zero).  Returns (t_orth, parity of all -1).
    """
    n = tuple(int(m) for m in n)
    rng = np.random.default_rng(seed)
    t = np.zeros((c, c) + n, dtype=np.complex128)
    for a in range(c):
        for b in range(a, c):
            v = complex_normal(rng, n)
            for m in range(len(n)):
                idx = [slice(None)] * len(n)
                idx[m] = 0
                v[tuple(idx)] = 0.0
            t[a, b] = v
            t[b, a] = v
    parity = -np.ones((c, c, len(n)), dtype=np.int8)
    return t, parity


def random_parity_orthant(n, c: int, seed: int, parity: np.ndarray, block_sym: bool):
    """Random orthant generator with the given parity signs (zeros forced on
    the p_m = 0 planes of every odd dimension)."""
    n = tuple(int(m) for m in n)
    rng = np.random.default_rng(seed)
    t = np.zeros((c, c) + n, dtype=np.complex128)
    for a in range(c):
        for b in range(c):
            if block_sym and b < a:
                t[a, b] = t[b, a]
                continue
            v = complex_normal(rng, n)
            for m in range(len(n)):
                if parity[a, b, m] < 0:
                    idx = [slice(None)] * len(n)
                    idx[m] = 0
                    v[tuple(idx)] = 0.0
            t[a, b] = v
    return t


# --------------------------------------------------------------------------
# named workloads (sizes and seeds of the benchmark configurations)
# --------------------------------------------------------------------------

KH_GREEN = 2.0 * math.pi / 20.0

WORKLOADS = {
    # d=2 scalar random generator, 64x64, complex128 (FP64 GPU mode)
    "d2_64_c1_random_c128": dict(d=2, n=(64, 64), c=1, kind="random", t_seed=1, x_seed=2,
                                 precision="c128"),
    # d=3 128^3 dyadic Green, fully symmetric, complex64
    "d3_128_c3_green_c64": dict(d=3, n=(128, 128, 128), c=3, kind="green", kh=KH_GREEN,
                                x_seed=3, precision="c64"),
    # d=3 256^3 dyadic Green, complex64
    "d3_256_c3_green_c64": dict(d=3, n=(256, 256, 256), c=3, kind="green", kh=KH_GREEN,
                                x_seed=4, precision="c64"),
    # d=3 192^3 dyadic Green, complex64 (the largest 3-d serving size; composite 192 = 24 x 8)
    "d3_192_c3_green_c64": dict(d=3, n=(192, 192, 192), c=3, kind="green", kh=KH_GREEN,
                                x_seed=8, precision="c64"),
    # d=3 256^3 skew (odd in every dim, t_ab = t_ba), complex64
    "d3_256_c3_skew_c64": dict(d=3, n=(256, 256, 256), c=3, kind="skew", t_seed=5,
                               x_seed=4, precision="c64"),
}

BATCH_DIMS = (24, 32, 48, 60, 64, 84, 96)


def batched_instances(count: int = 64, seed: int = 6, dims=BATCH_DIMS, max_rhs: int = 16):
    """Uneven d=3 Green-dyadic instances: each dim drawn independently from
    ``dims``, kh ~ U[2pi/30, 2pi/10], nrhs ~ U{1..max_rhs}."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = tuple(int(v) for v in rng.choice(dims, size=3))
        kh = float(rng.uniform(2 * math.pi / 30, 2 * math.pi / 10))
        r = int(rng.integers(1, max_rhs + 1))
        xs = int(rng.integers(0, 2 ** 31 - 1))
        out.append(dict(n=n, kh=kh, nrhs=r, x_seed=xs))
    return out
