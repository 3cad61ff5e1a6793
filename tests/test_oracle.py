"""Pins for the CPU oracle: it is checked against what the paper and the
mathematics fix, never against itself or the CUDA library."""
import itertools
import math

import numpy as np
import pytest

import workloads as W
from oracle import embed as OE
from oracle import split as OS
from oracle import toeplitz as OT
from tests.conftest import read_golden

RNG = np.random.default_rng(1234)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


TINY = [((5,), 1), ((4,), 3), ((3, 4), 1), ((2, 3), 3), ((2, 3, 2), 1), ((2, 2, 3), 3),
        ((1, 3), 1), ((1,), 2)]


@pytest.mark.parametrize("n,c", TINY)
def test_dense_bruteforce_direct_embed_split_agree(n, c):
    t = W.random_generator(n, c, seed=11)
    x = W.random_vector(n, c, seed=12, nrhs=2)
    M = OT.dense_matrix(t)
    s = int(np.prod(n))
    y_dense = np.stack([(M @ x[r].reshape(c * s)).reshape((c,) + n) for r in range(2)])
    y_bf = OT.brute_force_matvec(t, x)
    assert rel(y_bf, y_dense) < 1e-13
    assert rel(OT.direct_matvec(t, x), y_dense) < 1e-13
    assert rel(OE.embed_matvec(t, x), y_dense) < 1e-12
    assert rel(OS.split_matvec(t, x), y_dense) < 1e-12
    assert rel(OS.split_flat(t, x), y_dense) < 1e-12


def test_d1_is_numpy_convolution():
    n = 9
    tarr = W.complex_normal(RNG, (2 * n - 1,))
    x = W.complex_normal(RNG, (n,))
    t = tarr.reshape(1, 1, -1)
    y_ref = np.convolve(tarr, x)[n - 1: 2 * n - 1]
    for f in (OT.direct_matvec, OE.embed_matvec, OS.split_matvec):
        y = f(t, x.reshape(1, n))[0]
        assert rel(y, y_ref) < 1e-13


@pytest.mark.parametrize("n,c", [((6,), 1), ((4, 5), 3), ((3, 4, 5), 1)])
def test_identity_generator_gives_x(n, c):
    t = np.zeros((c, c) + W.offsets_shape(n), dtype=np.complex128)
    center = tuple(m - 1 for m in n)
    for a in range(c):
        t[(a, a) + center] = 1.0
    x = W.random_vector(n, c, seed=3)[0]
    for f in (OT.direct_matvec, OE.embed_matvec, OS.split_matvec):
        assert rel(f(t, x), x) < 1e-14


@pytest.mark.parametrize("n,p0", [((7,), (2,)), ((7,), (-3,)), ((4, 5), (1, -2)),
                                  ((3, 4, 5), (-1, 2, 3))])
def test_single_offset_generator_is_shift(n, p0):
    """t = delta_{p0}  =>  y[i] = x[i - p0] with zero fill: pins the i - j
    convention and the sign of the forward kernel and phase operator."""
    d = len(n)
    t = np.zeros((1, 1) + W.offsets_shape(n), dtype=np.complex128)
    t[(0, 0) + tuple(p0[m] + n[m] - 1 for m in range(d))] = 1.0
    x = W.random_vector(n, 1, seed=4)[0]
    y_ref = np.zeros_like(x)
    for i in itertools.product(*[range(m) for m in n]):
        j = tuple(i[m] - p0[m] for m in range(d))
        if all(0 <= j[m] < n[m] for m in range(d)):
            y_ref[(0,) + i] = x[(0,) + j]
    for f in (OT.direct_matvec, OE.embed_matvec, OS.split_matvec, OS.split_flat):
        assert rel(f(t, x), y_ref) < 1e-13


def test_linearity_and_shift_equivariance():
    n, c = (6, 5), 3
    t = W.random_generator(n, c, seed=21)
    x = W.random_vector(n, c, seed=22)[0]
    z = W.random_vector(n, c, seed=23)[0]
    al, be = 0.7 - 1.3j, -2.1 + 0.4j
    for f in (OE.embed_matvec, OS.split_matvec):
        assert rel(f(t, al * x + be * z), al * f(t, x) + be * f(t, z)) < 1e-12
    # shift equivariance: support inside grid cap (grid - delta)
    delta = (1, 2)
    xs = np.zeros_like(x)
    xs[:, :n[0] - delta[0], :n[1] - delta[1]] = x[:, :n[0] - delta[0], :n[1] - delta[1]]
    shifted = np.zeros_like(x)
    shifted[:, delta[0]:, delta[1]:] = xs[:, :n[0] - delta[0], :n[1] - delta[1]]
    for f in (OT.direct_matvec, OE.embed_matvec, OS.split_matvec):
        y0 = f(t, xs)
        y1 = f(t, shifted)
        assert rel(y1[:, delta[0]:, delta[1]:], y0[:, :n[0] - delta[0], :n[1] - delta[1]]) < 1e-12


def adjoint_generator(t):
    """Generator of T^H: t^H_ab[p] = conj(t_ba[-p])."""
    d = t.ndim - 2
    flipped = t[(slice(None), slice(None)) + (slice(None, None, -1),) * d]
    return np.conj(np.swapaxes(flipped, 0, 1))


def test_adjoint_identity():
    n, c = (4, 3, 5), 3
    t = W.random_generator(n, c, seed=31)
    x = W.random_vector(n, c, seed=32)[0]
    z = W.random_vector(n, c, seed=33)[0]
    th = adjoint_generator(t)
    M = OT.dense_matrix(t)
    assert rel(OT.dense_matrix(th), M.conj().T) < 1e-15
    for f in (OT.direct_matvec, OE.embed_matvec, OS.split_matvec):
        lhs = np.vdot(z, f(t, x))            # <T x, z> as z^H (T x)
        rhs = np.vdot(f(th, z), x)           # <x, T^H z>
        assert abs(lhs - rhs) < 1e-11 * abs(lhs)


def test_symmetric_bilinear_identity():
    """t_ab(-p) = t_ba(p)  =>  T^T = T  =>  z^T T x = x^T T z."""
    n, c = (4, 5), 3
    t = W.random_generator(n, c, seed=41)
    d = len(n)
    tf = t[(slice(None), slice(None)) + (slice(None, None, -1),) * d]
    t = 0.5 * (t + np.swapaxes(tf, 0, 1))
    x = W.random_vector(n, c, seed=42)[0]
    z = W.random_vector(n, c, seed=43)[0]
    M = OT.dense_matrix(t)
    assert rel(M, M.T) < 1e-15
    for f in (OT.direct_matvec, OE.embed_matvec, OS.split_matvec):
        a = np.sum(z * f(t, x))
        b = np.sum(x * f(t, z))
        assert abs(a - b) < 1e-11 * abs(a)


def test_skew_bilinear_identity():
    """t_ab = t_ba and t odd in every dim => T^T = -T => x^T T x = 0."""
    n = (4, 3, 5)
    t_orth, par = W.skew_orthant(n, seed=5)
    t = W.orthant_to_full(t_orth, par)
    M = OT.dense_matrix(t)
    assert rel(M, -M.T) < 1e-15
    x = W.random_vector(n, 3, seed=51)[0]
    scale = np.linalg.norm(x) ** 2 * np.abs(t).max()
    for f in (OT.direct_matvec, OE.embed_matvec, OS.split_matvec):
        assert abs(np.sum(x * f(t, x))) < 1e-11 * scale


def test_s0_invariance():
    n, c = (4, 6), 3
    t = W.random_generator(n, c, seed=61)
    x = W.random_vector(n, c, seed=62)[0]
    y0 = OE.embed_matvec(t, x, s0=0.0)
    y1 = OE.embed_matvec(t, x, s0=3.7 - 1.1j)
    assert rel(y1, y0) < 1e-13


@pytest.mark.parametrize("order", list(itertools.permutations(range(3))))
def test_level_order_invariance(order):
    n, c = (3, 4, 5), 3
    t = W.random_generator(n, c, seed=71)
    x = W.random_vector(n, c, seed=72)[0]
    assert rel(OS.split_matvec(t, x, order=order), OT.direct_matvec(t, x)) < 1e-12


def explicit_dft(v, sign=-1):
    """Plain O(n^2) DFT sum, unnormalised, kernel exp(sign 2 pi i f k / N)."""
    N = len(v)
    out = np.zeros(N, dtype=np.complex128)
    for f in range(N):
        acc = 0j
        for k in range(N):
            acc += v[k] * complex(math.cos(2 * math.pi * f * k / N),
                                  sign * math.sin(2 * math.pi * f * k / N))
        out[f] = acc
    return out


@pytest.mark.parametrize("n", [1, 2, 5, 8, 12])
def test_splitting_property(n):
    """Sec. II.A: even coefficients of DFT_{2n}([v,0]) are DFT_n(v), odd
    ones are DFT_n(P v) with P[k] = exp(-i pi k/n)."""
    v = W.complex_normal(RNG, (n,))
    full = explicit_dft(np.concatenate([v, np.zeros(n)]))
    assert rel(full[0::2], explicit_dft(v)) < 1e-13
    assert rel(full[1::2], explicit_dft(OS.phase(n, 1) * v)) < 1e-13
    if n > 1:
        # the phase as printed (+ sign) does not give the odd coefficients
        wrong = np.exp(+1j * np.pi * np.arange(n) / n)
        assert rel(full[1::2], explicit_dft(wrong * v)) > 1e-2


@pytest.mark.parametrize("n", [3, 8])
def test_merge_property(n):
    """Merge: the first n entries of IDFT_{2n}(Z) equal
    IDFT_n(Z_even) + conj(P) IDFT_n(Z_odd), all unnormalised."""
    Z = W.complex_normal(RNG, (2 * n,))
    full = explicit_dft(Z, sign=+1)[:n]
    merged = explicit_dft(Z[0::2], +1) + np.conj(OS.phase(n, 1)) * explicit_dft(Z[1::2], +1)
    assert rel(merged, full) < 1e-13


def test_golden_embedding_2x2():
    rows = read_golden("embedding_2x2.txt")
    vals = {"t11": 1.5 + 0.25j, "t12": -0.75 + 2.0j, "t21": 0.5 - 1.25j, "s0": 3.0 + 7.0j}
    expect = np.array([[vals[e] for e in r] for r in rows])
    t = np.array([vals["t12"], vals["t11"], vals["t21"]]).reshape(1, 1, 3)   # p = -1, 0, +1
    col = OE.embedded_generator(t, s0=vals["s0"])[0, 0]
    circ = np.array([[col[(i - j) % 4] for j in range(4)] for i in range(4)])
    assert np.array_equal(circ, expect)
    # and the upper-left 2x2 block is the Toeplitz matrix itself
    assert np.array_equal(OT.dense_matrix(t), expect[:2, :2])


def test_golden_two_level_symmetric_layout():
    rows = read_golden("symmetric_two_level.txt")
    n = (4, 4)
    orth = W.complex_normal(RNG, n)
    par = np.ones((1, 1, 2), dtype=np.int8)
    t = W.orthant_to_full(orth.reshape(1, 1, 4, 4), par)
    ct = OE.embedded_generator(t)[0, 0]
    for i in range(8):
        for j in range(8):
            e = rows[i][j]
            want = 0.0 if e == "0" else orth[int(e[1]), int(e[2])]
            assert ct[i, j] == want


@pytest.mark.parametrize("c", [1, 3])
def test_symbol_mirror_symmetry(c):
    """Even generator in dim m => S[f] = S[2n - f] along m; odd => S[2n-f] =
    -S[f] with S = 0 at f = 0 and f = n (reading of Sec. II.C)."""
    n = (4, 5, 6)
    if c == 3:
        t_orth, par = W.green_dyadic_orthant(n, kh=W.KH_GREEN)
    else:
        par = np.array([[[1, -1, 1]]], dtype=np.int8)
        t_orth = W.random_parity_orthant(n, 1, 81, par, block_sym=False)
    S = OE.symbol(W.orthant_to_full(t_orth, par))
    for a in range(c):
        for b in range(c):
            for m in range(3):
                Sm = np.moveaxis(S[a, b], m, 0)
                nm = n[m]
                mir = np.concatenate([Sm[:1], Sm[1:][::-1]], axis=0)   # f -> 2n - f
                sg = par[a, b, m]
                assert rel(mir, sg * Sm) < 1e-13 or np.abs(Sm).max() < 1e-14
                if sg < 0:
                    assert np.abs(Sm[0]).max() < 1e-13 and np.abs(Sm[nm]).max() < 1e-13


def test_direct_points_match_direct():
    n, c = (5, 4, 6), 3
    t = W.random_generator(n, c, seed=91)
    x = W.random_vector(n, c, seed=92, nrhs=2)
    y = OT.direct_matvec(t, x)
    pts = [(0, 0, 0), (4, 3, 5), (2, 1, 3), (1, 3, 0)]
    got = OT.direct_points(t, x, pts)
    for k, p in enumerate(pts):
        assert rel(got[k], y[(slice(None), slice(None)) + p]) < 1e-13


def test_embed_matches_direct_points_moderate():
    n = (16, 12, 20)
    t_orth, par = W.green_dyadic_orthant(n, kh=W.KH_GREEN)
    t = W.orthant_to_full(t_orth, par)
    x = W.random_vector(n, 3, seed=93)[0]
    y = OE.embed_matvec(t, x)
    pts = [(0, 0, 0), (15, 11, 19), (7, 3, 11), (2, 10, 5)]
    got = OT.direct_points(t, x, pts)
    for k, p in enumerate(pts):
        assert rel(got[k], y[(slice(None),) + p]) < 1e-13


# ------------------------------------------------------------------ inputs

def test_green_generator_closed_form_values():
    n = (3, 3, 3)
    kh = W.KH_GREEN
    t_orth, par = W.green_dyadic_orthant(n, kh=kh)
    assert np.array_equal(t_orth[:, :, 0, 0, 0], np.eye(3))
    # r = (1, 0, 0): rhat = e_0, kR = kh
    k = kh
    g = np.exp(1j * k) / (4 * math.pi)
    G00 = g * ((1 + 1j / k - 1 / k ** 2) - (1 + 3j / k - 3 / k ** 2))
    G11 = g * (1 + 1j / k - 1 / k ** 2)
    assert abs(t_orth[0, 0, 1, 0, 0] - G00) < 1e-15
    assert abs(t_orth[1, 1, 1, 0, 0] - G11) < 1e-15
    assert t_orth[0, 1, 1, 0, 0] == 0
    # r = (1, 1, 0): off-diagonal 01 = -beta * 1/2
    R = math.sqrt(2)
    g = np.exp(1j * k * R) / (4 * math.pi * R)
    beta = g * (1 + 3j / (k * R) - 3 / (k * R) ** 2)
    assert abs(t_orth[0, 1, 1, 1, 0] - (-beta * 0.5)) < 1e-15
    # parity of the expansion matches direct evaluation at negative offsets
    t = W.orthant_to_full(t_orth, par)
    assert abs(t[0, 1, 2 - 1, 2 + 1, 2] - (+beta * 0.5)) < 1e-15    # r = (-1, 1, 0)
    assert np.allclose(t, np.swapaxes(t, 0, 1))


def test_orthant_expansion_parity():
    n = (3, 4)
    par = np.array([[[1, -1]]], dtype=np.int8)
    orth = W.random_parity_orthant(n, 1, 5, par, block_sym=False)
    t = W.orthant_to_full(orth, par)
    for p1 in range(-2, 3):
        for p2 in range(-3, 4):
            v = orth[0, 0, abs(p1), abs(p2)] * (-1 if p2 < 0 else 1)
            assert t[0, 0, p1 + 2, p2 + 3] == v


# ------------------------------------------------- planted-mistake checks

def test_planted_phase_sign_mistake_is_caught(monkeypatch):
    """A wrong phase sign in the split restatement must fail the pins."""
    n, c = (4, 5), 1
    t = W.random_generator(n, c, seed=101)
    x = W.random_vector(n, c, seed=102)[0]
    good = OT.direct_matvec(t, x)
    monkeypatch.setattr(OS, "phase", lambda m, odd: np.exp(+1j * np.pi * odd * np.arange(m) / m))
    assert rel(OS.split_matvec(t, x), good) > 1e-3


def test_planted_transpose_mistake_is_caught():
    """Swapping the block indices (t_ba for t_ab) must fail brute force."""
    n, c = (3, 4), 3
    t = W.random_generator(n, c, seed=103)
    x = W.random_vector(n, c, seed=104)[0]
    good = OT.brute_force_matvec(t, x)
    bad = OT.direct_matvec(np.swapaxes(t, 0, 1).copy(), x)
    assert rel(bad, good) > 1e-2
