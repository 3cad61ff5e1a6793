"""Operation-count, memory and traffic models (host-side reporting only).

The complexity and peak-memory ratios restate Sec. II.C of the paper
(Eq. CompRatio, Eq. MemRatio, Eq. MemRatioSym, Table 1).  The byte models are
this library's own: algorithmic HBM bytes moved by each kernel of the split
and plain-embedding schedules, used as the numerator of the roofline
fraction.
"""
from __future__ import annotations

import math


# ---------------------------------------------------------------- Sec. II.C

def complexity_split(d: int, n: int) -> float:
    """C_split / s: FFTs 2 sum_{l=1..d} 2^l log2 n, multiply 2^d, phase
    shifts 2 sum_{l=0..d-1} 2^l (level sum read as 1 <= l <= d)."""
    return 2 * (2 ** d - 1) * (2 * math.log2(n) + 1) + 2 ** d


def complexity_embed(d: int, n: int) -> float:
    """C_embed / s = 2^{d+1} log2(2^d s) + 2^d with s = n^d."""
    s_log = d * math.log2(n)
    return 2 ** (d + 1) * (d + s_log) + 2 ** d


def ratio_complexity(d: int, n: int) -> float:
    """R_c = C_embed / C_split (first line of Eq. CompRatio), divided through
    by 2^{d+1} s.  The printed second line carries +1 where this division
    gives +1/2 on both non-log terms; the asymptote is the same."""
    return (d * math.log2(2 * n) + 0.5) / ((1 - 2.0 ** -d) * (2 * math.log2(n) + 1) + 0.5)


def ratio_complexity_printed(d: int, n: int) -> float:
    """Second line of Eq. CompRatio exactly as printed."""
    return (d * math.log2(2 * n) + 1) / ((1 - 2.0 ** -d) * (2 * math.log2(n) + 1) + 1)


def ratio_complexity_asymptotic(d: int) -> float:
    """R_c -> d / (2 - 2^{1-d}) as n -> infinity."""
    return d / (2 - 2.0 ** (1 - d))


def ratio_memory(d: int) -> float:
    """R_m = 2^{d+1} s / ((d+1) s + 2^d s) = 2 / ((d+1) 2^-d + 1)."""
    return 2.0 / ((d + 1) * 2.0 ** -d + 1)


def ratio_memory_sym(d: int) -> float:
    """R_m,sym = (2^d + 1) / (d + 2)."""
    return (2 ** d + 1) / (d + 2)


def ratio_memory_blocks(d: int, c: int, sym_split: float, sym_embed: float) -> float:
    """Peak-memory ratio with c components and c x c symbol blocks, in units
    of s elements: embed holds 2^d c vector + sym_embed symbol, split holds
    (d+1) c vector + sym_split symbol (the paper's accounting with c = 1,
    sym = 2^d / 1 reproduces Eq. MemRatio / Eq. MemRatioSym)."""
    return (2 ** d * c + sym_embed) / ((d + 1) * c + sym_split)


# ---------------------------------------------------------------- traffic

def vector_bytes(n, c: int, nrhs: int, elem_bytes: int) -> int:
    s = 1
    for m in n:
        s *= int(m)
    return c * s * nrhs * elem_bytes


def nsym(c: int, block_sym: bool) -> int:
    return c * (c + 1) // 2 if block_sym else c * c


def symbol_bytes(n, c: int, elem_bytes: int, block_sym: bool, compressed: bool) -> int:
    """Compressed parity store holds prod(n_m + 1) frequencies per component,
    the full store holds prod(2 n_m)."""
    cnt = 1
    for m in n:
        cnt *= (int(m) + 1) if compressed else 2 * int(m)
    return cnt * nsym(c, block_sym) * elem_bytes


def split_pass_bytes(n, c: int, nrhs: int, elem_bytes: int, sym_bytes: int) -> dict:
    """Algorithmic bytes per kernel kind for one split apply (depth-first
    schedule, each tree node written once and read once).

    forward split at level m (1 <= m <= d-1): 2^{m-1} launches' worth of
    nodes, each read V, write 2V.  leaf: 2^{d-1} nodes, read V write V, plus
    the symbol read once.  merge at level m: 2^{m-1} nodes, read 2V write V.
    d = 1: the leaf reads x and writes y.
    """
    d = len(n)
    V = vector_bytes(n, c, nrhs, elem_bytes)
    fwd = sum(2 ** (m - 1) * 3 * V for m in range(1, d))
    mrg = sum(2 ** (m - 1) * 3 * V for m in range(1, d))
    leaf = 2 ** (d - 1) * 2 * V + sym_bytes
    return {"fwd_split": fwd, "leaf": leaf, "bwd_merge": mrg,
            "total": fwd + leaf + mrg, "V": V}


def fused_pass_bytes(n, c: int, nrhs: int, elem_bytes: int, sym_bytes: int) -> dict:
    """Algorithmic bytes of a split apply (d >= 3) with the last two levels
    fused (BTMV_FLAG_FUSED_LEVELS): the forward splits and merges of levels
    1..d-2 as in split_pass_bytes (each 3V per node), each of the 2^(d-2)
    fused launches reading its level-(d-2) node and writing it back (2V; the
    levels below it stay on chip), and the symbol read once.  The fused
    kernel's scratch vector (the even half of the column-dim merge parked off
    chip) is an implementation cost, not counted here.  d = 3: 10 V + symbol
    against 26 V + symbol unfused."""
    d = len(n)
    if d < 3:
        raise ValueError("the fused schedule needs d >= 3")
    V = vector_bytes(n, c, nrhs, elem_bytes)
    passes = sum(2 ** (m - 1) * 3 * V for m in range(1, d - 1))
    fused = 2 ** (d - 2) * 2 * V + sym_bytes
    return {"fwd_split": passes, "fused_levels": fused, "bwd_merge": passes,
            "total": 2 * passes + fused, "V": V}


def apply_kind_bytes(n, c: int, nrhs: int, elem_bytes: int, sym_bytes: int, one_kernel: bool = False) -> dict:
    """Algorithmic bytes per profile kind of one split apply: the split
    schedule's kinds (split_pass_bytes), or, for a d = 2 apply run as one
    cluster kernel (one_kernel), that kernel's x read, y written and symbol
    read once: 2 V + symbol under the kind "fused_levels"."""
    if one_kernel:
        if len(n) != 2:
            raise ValueError("the one-kernel apply is d = 2")
        V = vector_bytes(n, c, nrhs, elem_bytes)
        return {"fused_levels": 2 * V + sym_bytes, "total": 2 * V + sym_bytes, "V": V}
    pb = split_pass_bytes(n, c, nrhs, elem_bytes, sym_bytes)
    return {"fwd_split": pb["fwd_split"], "leaf": pb["leaf"], "merge": pb["bwd_merge"],
            "total": pb["total"], "V": pb["V"]}


def full_pass_bytes(n, c: int, nrhs: int, elem_bytes: int, sym_bytes: int) -> dict:
    """Algorithmic bytes of the plain full embedding with the library's own
    kernels: the first pass reads x (V) and writes the zero-padded,
    dim-1-transformed array (2^d V); each further forward or inverse pass on
    the padded grid reads and writes 2^d V; the leaf pass (forward, multiply
    by the full symbol, inverse along the last dim) reads and writes 2^d V and
    the symbol; the last inverse pass reads only the lines that survive the
    projection (2V) and writes y (V)."""
    d = len(n)
    V = vector_bytes(n, c, nrhs, elem_bytes)
    big = 2 ** d * V
    if d == 1:
        leaf = V + V + sym_bytes           # pad+fwd+mul+inv+project in one pass
        return {"first": 0, "middle": 0, "leaf": leaf, "last": 0, "total": leaf, "V": V}
    first = V + big
    middle = 2 * (d - 2) * 2 * big
    leaf = 2 * big + sym_bytes
    last = 2 * V + V
    return {"first": first, "middle": middle, "leaf": leaf, "last": last,
            "total": first + middle + leaf + last, "V": V}
