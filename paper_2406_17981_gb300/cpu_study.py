"""Host-core reproduction of the paper's wall-clock study (Sec. III, Fig. 3).

The paper times, on a multi-core CPU with a library FFT, the split algorithm
against the plain full circulant embedding for d = 1..4 levels at
power-of-two sizes, with random complex generators and vectors whose real
and imaginary parts have zero mean, and plots the ratio of the two wall-clock
times beside the operation-count ratio R_c of Eq. CompRatio.  This module does
the same on the host cores with scipy.fft (``workers`` = the cores this
process may use), scalar blocks (c = 1):

* ``EmbedRunner``: pad x to the 2n grid, forward transform, multiply by the
  transformed embedded generator, inverse transform, keep the n grid (Sec. I).
* ``SplitRunner``: Algorithm 1 (Sec. II.B) depth first over the levels: at
  level m a node is transformed along dim m into its even child DFT_n(v) and
  its odd child DFT_n(P_m v) (Sec. II.A splitting property), the leaf with
  parity vector b multiplies by S_b = S[2l + b], and on the way back the
  children are inverse transformed and merged as R_e + conj(P_m) R_o
  (merging property), which is the eager projection onto the n grid.

The symbol (the transform of the embedded generator) and the work arrays are
prepared once per problem, outside the timed region, as the paper's timings
cover the matvec; transforms and products then run in place.
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


class Par:
    """Elementwise products, sums, fills and copies on every core: the arrays
    are cut along their leading axis into one chunk per worker (numpy ufuncs
    release the interpreter lock on large arrays), so that these memory-bound
    passes are as parallel as the library FFTs beside them."""

    def __init__(self, workers: int):
        import concurrent.futures as cf
        self.w = max(1, workers)
        self.pool = cf.ThreadPoolExecutor(max_workers=self.w) if self.w > 1 else None

    def _chunks(self, n0):
        k = min(self.w, n0)
        b = [n0 * i // k for i in range(k + 1)]
        return [slice(b[i], b[i + 1]) for i in range(k)]

    @staticmethod
    def _part(a, sl):
        return a if (a.ndim == 0 or a.shape[0] == 1) else a[sl]

    def run(self, fn, out, *args):
        if self.pool is None or out.shape[0] < 2 or out.size < (1 << 16):
            fn(*args, out=out)
            return out
        futs = [self.pool.submit(fn, *[self._part(a, sl) for a in args], out=out[sl])
                for sl in self._chunks(out.shape[0])]
        for f in futs:
            f.result()
        return out

    def mul(self, a, b, out):
        return self.run(np.multiply, out, a, b)

    def add(self, a, b, out):
        return self.run(np.add, out, a, b)

    def copy(self, src, out):
        return self.run(lambda a, out: np.copyto(out, a), out, src)

    def zero(self, out):
        return self.run(lambda out: out.fill(0.0), out)


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


class EmbedRunner:
    """The full embedding with its 2n-grid work array allocated once and
    every transform and product done in place (as with in-place library FFT
    plans)."""

    def __init__(self, S: np.ndarray, workers: int):
        self.S, self.workers = S, workers
        self.par = Par(workers)
        self.Z = np.empty(S.shape, dtype=np.complex128)
        self.y = None

    def __call__(self, x: np.ndarray) -> np.ndarray:
        n = x.shape
        grid = tuple(slice(0, m) for m in n)
        Z = self.Z
        self.par.zero(Z)
        self.par.copy(x, Z[grid])
        Z = sfft.fftn(Z, workers=self.workers, overwrite_x=True)
        self.par.mul(Z, self.S, Z)
        Z = sfft.ifftn(Z, workers=self.workers, norm="forward", overwrite_x=True)
        if self.y is None:
            self.y = np.empty(n, dtype=np.complex128)
        return self.par.copy(Z[grid], self.y)


class SplitRunner:
    """Algorithm 1 depth first with one work array per level (the node
    vector is transformed in place into its even child, the odd child lives in
    the level's array): the (d + 1)-vector footprint of Sec. II.C, transforms
    and products in place."""

    def __init__(self, parts: dict, P: list, workers: int):
        self.parts, self.P, self.workers = parts, P, workers
        self.par = Par(workers)
        self.Pc = [np.conj(p) for p in P]
        shape = next(iter(parts.values())).shape
        self.d = len(shape)
        self.top = np.empty(shape, dtype=np.complex128)
        self.odd = [np.empty(shape, dtype=np.complex128) for _ in range(self.d)]

    def _node(self, v, m, prefix):
        if m == self.d:
            return self.par.mul(v, self.parts[prefix], v)
        w = self.workers
        odd = self.odd[m]
        self.par.mul(v, self.P[m], odd)
        v = sfft.fft(v, axis=m, workers=w, overwrite_x=True)
        odd = sfft.fft(odd, axis=m, workers=w, overwrite_x=True)
        v = self._node(v, m + 1, prefix + (0,))
        odd = self._node(odd, m + 1, prefix + (1,))
        v = sfft.ifft(v, axis=m, workers=w, norm="forward", overwrite_x=True)
        odd = sfft.ifft(odd, axis=m, workers=w, norm="forward", overwrite_x=True)
        self.par.mul(odd, self.Pc[m], odd)
        return self.par.add(v, odd, v)

    def __call__(self, x: np.ndarray) -> np.ndarray:
        self.par.copy(x, self.top)
        return self._node(self.top, 0, ()).copy()


def embed_apply(S: np.ndarray, x: np.ndarray, workers: int) -> np.ndarray:
    return EmbedRunner(S, workers)(x)


def split_apply(parts: dict, P: list, x: np.ndarray, workers: int) -> np.ndarray:
    return SplitRunner(parts, P, workers)(x)


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
            sr = SplitRunner(parts, P, workers)
            ts = time_best(lambda: sr(x), repeats)
            del sr
            er = EmbedRunner(S, workers)
            te = time_best(lambda: er(x), repeats)
            del er
            rows.append({"d": d, "n": nm, "split_s": ts, "embed_s": te, "ratio_embed_over_split": te / ts})
            del S, parts, t
    return rows


if __name__ == "__main__":
    import json
    for row in study():
        print(json.dumps(row))
