"""Host-core reproduction of the paper's wall-clock study (Sec. III, Fig. 3).

The paper times, on a multi-core CPU with a library FFT, the split algorithm
against the plain full circulant embedding for d = 1..4 levels at
power-of-two sizes, with random complex generators and vectors whose real
and imaginary parts have zero mean, and plots the ratio of the two wall-clock
times beside the operation-count ratio R_c of Eq. CompRatio.  This module does
the same on the host cores with scipy.fft (``workers`` = the cores this
process may use), scalar blocks (c = 1):

* ``embed_apply``: pad x to the 2n grid, forward transform, multiply by the
  transformed embedded generator, inverse transform, keep the n grid (Sec. I).
* ``split_apply``: Algorithm 1 (Sec. II.B) depth first over the levels: at
  level m a node is transformed along dim m into its even child DFT_n(v) and
  its odd child DFT_n(P_m v) (Sec. II.A splitting property), the leaf with
  parity vector b multiplies by S_b = S[2l + b], and on the way back the
  children are inverse transformed and merged as R_e + conj(P_m) R_o
  (merging property), which is the eager projection onto the n grid.

The symbol (the transform of the embedded generator) is prepared once per
problem, outside the timed region, as the paper's timings cover the matvec.
Transforms are unnormalised in both directions; the single 1/prod(2 n_m)
scale sits in the symbol.  This is a CPU study only: the GPU library does
not use it.
"""
from __future__ import annotations

import os
import time

import numpy as np
import scipy.fft as sfft


def cores() -> int:
    return len(os.sched_getaffinity(0))


def embedded_symbol(t: np.ndarray, workers: int) -> np.ndarray:
    """S on the 2n grid: DFT of the circulant embedding of the generator
    t[p_1 + n_1 - 1, ...] (offsets p_m in [-(n_m - 1), n_m - 1]), with the
    free entry at k_m = n_m set to zero, divided by prod(2 n_m)."""
    n = tuple((m + 1) // 2 for m in t.shape)
    d = len(n)
    emb = t
    for m in range(d):
        k = np.arange(2 * n[m])
        # k < n: offset k (index k + n - 1); k > n: offset k - 2n (index k - n - 1)
        idx = np.where(k < n[m], k + n[m] - 1, k - n[m] - 1)
        emb = np.take(emb, idx, axis=m)
        sl = [slice(None)] * d
        sl[m] = n[m]
        emb[tuple(sl)] = 0.0
    scale = 1.0 / float(np.prod([2 * m for m in n]))
    return sfft.fftn(emb, workers=workers) * scale


def leaf_parts(S: np.ndarray) -> dict:
    """S_b[l] = S[2l + b] for every parity vector b (tuple of 0/1)."""
    d = S.ndim
    parts = {}
    for code in range(1 << d):
        b = tuple((code >> (d - 1 - m)) & 1 for m in range(d))
        parts[b] = np.ascontiguousarray(S[tuple(slice(bm, None, 2) for bm in b)])
    return parts


def phases(n) -> list:
    """P_m[k] = exp(-i pi k / n_m) per level, shaped to broadcast along dim m."""
    d = len(n)
    out = []
    for m in range(d):
        shape = [1] * d
        shape[m] = n[m]
        out.append(np.exp(-1j * np.pi * np.arange(n[m]) / n[m]).reshape(shape))
    return out


def embed_apply(S: np.ndarray, x: np.ndarray, workers: int) -> np.ndarray:
    n = x.shape
    xp = np.zeros(S.shape, dtype=np.complex128)
    xp[tuple(slice(0, m) for m in n)] = x
    Y = sfft.fftn(xp, workers=workers)
    Y *= S
    y = sfft.ifftn(Y, workers=workers, norm="forward")
    return y[tuple(slice(0, m) for m in n)]


def split_apply(parts: dict, P: list, x: np.ndarray, workers: int) -> np.ndarray:
    d = x.ndim

    def node(v, m, prefix):
        if m == d:
            return v * parts[prefix]
        even = sfft.fft(v, axis=m, workers=workers)
        odd = sfft.fft(v * P[m], axis=m, workers=workers)
        re = sfft.ifft(node(even, m + 1, prefix + (0,)), axis=m, workers=workers, norm="forward")
        ro = sfft.ifft(node(odd, m + 1, prefix + (1,)), axis=m, workers=workers, norm="forward")
        return re + np.conj(P[m]) * ro

    return node(x, 0, ())


def time_best(fn, repeats: int) -> float:
    fn()                                       # warm-up (plans, page faults)
    best = float("inf")
    for _ in range(repeats):
        t0 = time.perf_counter()
        fn()
        best = min(best, time.perf_counter() - t0)
    return best


DEFAULT_SIZES = {1: [2 ** k for k in range(10, 21, 2)], 2: [2 ** k for k in range(5, 12)],
                 3: [2 ** k for k in range(4, 9)], 4: [2 ** k for k in range(3, 7)]}


def study(sizes=None, repeats: int = 3, seed: int = 11, workers: int | None = None) -> list:
    """Rows (d, n, split_s, embed_s, ratio embed/split) on the host cores,
    n the same at every level; random complex generator and vector (real and
    imaginary parts i.i.d. standard normal, zero mean)."""
    workers = workers or cores()
    sizes = sizes or DEFAULT_SIZES
    rng = np.random.default_rng(seed)
    rows = []
    for d in sorted(sizes):
        for nm in sizes[d]:
            n = (nm,) * d
            t = rng.standard_normal(tuple(2 * m - 1 for m in n)) + 1j * rng.standard_normal(tuple(2 * m - 1 for m in n))
            x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
            S = embedded_symbol(t, workers)
            parts = leaf_parts(S)
            P = phases(n)
            ts = time_best(lambda: split_apply(parts, P, x, workers), repeats)
            te = time_best(lambda: embed_apply(S, x, workers), repeats)
            rows.append({"d": d, "n": nm, "split_s": ts, "embed_s": te, "ratio_embed_over_split": te / ts})
            del S, parts, t
    return rows


if __name__ == "__main__":
    import json
    for row in study():
        print(json.dumps(row))
