"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Gates: relative L2 error <= 1e-5 for complex64 and <= 1e-12 for complex128
(the FP64 GPU mode), element by element over the whole output.
"""
import numpy as np
import pytest

import workloads as W
from oracle import embed as OE
from oracle import toeplitz as OT
from tests.gpu_util import TOL, rel, round_input, run_btmv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

bt = pytest.importorskip("paper_2406_17981_gb300.btmv")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    bt.lib()


SIZES = [(1,), (2,), (5,), (16,), (60,), (128,), (3, 4), (7, 6), (12, 10), (1, 8), (4, 1),
         (16, 16), (5, 6, 7), (8, 8, 8), (3, 1, 4), (24, 12, 10), (2, 3, 4, 5), (20, 21, 14)]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("c", [1, 3])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("algo", [0, 1])
def test_random_generator_vs_oracle(n, c, precision, algo):
    t = W.random_generator(n, c, seed=100 + len(n))
    x = W.random_vector(n, c, seed=200 + sum(n), nrhs=2)
    y = run_btmv(t, x, n, c, precision, algo)
    ref = OE.embed_matvec(t, round_input(x, precision))
    assert rel(y, ref) <= TOL[precision]


def test_config_d2_64_c1_c128_vs_direct_sum():
    """64 x 64, scalar, random complex generator, complex128 vs the direct sum."""
    cfg = W.WORKLOADS["d2_64_c1_random_c128"]
    n = cfg["n"]
    t = W.random_generator(n, 1, seed=cfg["t_seed"])
    x = W.random_vector(n, 1, seed=cfg["x_seed"])
    for algo in (0, 1):
        y = run_btmv(t, x, n, 1, 1, algo)
        ref = OT.direct_matvec(t, x)
        assert rel(y, ref) <= 1e-12


@pytest.mark.parametrize("n", [(6, 5, 7), (16, 12, 20), (32, 32, 32)])
@pytest.mark.parametrize("precision", [0, 1])
def test_green_parity_compressed_symbol(n, precision):
    t_orth, par = W.green_dyadic_orthant(n, kh=W.KH_GREEN)
    x = W.random_vector(n, 3, seed=7)
    flags = bt.BTMV_SYM_BLOCK | bt.BTMV_SYM_PARITY
    y = run_btmv(t_orth, x, n, 3, precision, 0, flags, par)
    ref = OE.embed_matvec(W.orthant_to_full(t_orth, par), round_input(x, precision))
    assert rel(y, ref) <= TOL[precision]
    # the same generator without any symmetry flag gives the same product
    y2 = run_btmv(W.orthant_to_full(t_orth, par), x, n, 3, precision, 0)
    assert rel(y2, ref) <= TOL[precision]


@pytest.mark.parametrize("n", [(5, 6, 7), (16, 16, 16)])
def test_skew_parity(n):
    t_orth, par = W.skew_orthant(n, seed=5)
    x = W.random_vector(n, 3, seed=8)
    y = run_btmv(t_orth, x, n, 3, 0, 0, bt.BTMV_SYM_BLOCK | bt.BTMV_SYM_PARITY, par)
    tf = W.orthant_to_full(t_orth, par)
    ref = OE.embed_matvec(tf, round_input(x, 0))
    assert rel(y, ref) <= 1e-5
    # skew: x^T T x = 0
    xr = round_input(x, 0)
    assert abs(np.sum(xr * y)) <= 1e-5 * np.linalg.norm(xr) * np.linalg.norm(y)


@pytest.mark.parametrize("n,par", [((6, 7), [[[1, -1]]]), ((5, 4, 6), [[[-1, 1, -1]]])])
def test_scalar_mixed_parity(n, par):
    par = np.array(par, dtype=np.int8)
    t = W.random_parity_orthant(n, 1, 9, par, block_sym=False)
    x = W.random_vector(n, 1, seed=10)
    for precision in (0, 1):
        y = run_btmv(t, x, n, 1, precision, 0, bt.BTMV_SYM_PARITY, par)
        ref = OE.embed_matvec(W.orthant_to_full(t, par), round_input(x, precision))
        assert rel(y, ref) <= TOL[precision]


def test_block_symmetric_unstructured_c3():
    n = (9, 10)
    t = W.random_generator(n, 3, seed=11)
    t = 0.5 * (t + np.swapaxes(t, 0, 1))
    x = W.random_vector(n, 3, seed=12, nrhs=3)
    for precision in (0, 1):
        y = run_btmv(t, x, n, 3, precision, 0, bt.BTMV_SYM_BLOCK)
        ref = OE.embed_matvec(t, round_input(x, precision))
        assert rel(y, ref) <= TOL[precision]


@pytest.mark.parametrize("n,c,flags", [((6, 5), 1, 0), ((4, 3, 5), 3, 0), ((6, 5, 4), 3, 3)])
def test_symbol_store_matches_oracle_symbol(n, c, flags):
    """Leaf parts S_b[j] = S[2j + b] (Sec. II.C) as stored on the device."""
    d = len(n)
    if flags & bt.BTMV_SYM_PARITY:
        t_in, par = W.green_dyadic_orthant(n, kh=W.KH_GREEN)
        tf = W.orthant_to_full(t_in, par)
    else:
        t_in, par = W.random_generator(n, c, seed=13), None
        tf = t_in
    S = OE.symbol(tf)
    for precision in (0, 1):
        plan = bt.Plan(n, c, precision)
        plan.set_kernel(t_in, flags, par)
        info = plan.info
        got = bt.btmv_get_symbol(plan.handle)
        plan.close()
        nsym = info["nsym"]
        blocks = [(a, a) for a in range(c)] + [(a, b) for a in range(c) for b in range(a + 1, c)] \
            if flags & bt.BTMV_SYM_BLOCK else [(a, b) for a in range(c) for b in range(c)]
        exp = []
        for cls in range(1 << d):
            bits = [(cls >> (d - 1 - m)) & 1 for m in range(d)]
            J = [((n[m] - bits[m]) // 2 + 1) if info["compressed"] else n[m] for m in range(d)]
            for (a, b) in blocks[:nsym]:
                sl = tuple(slice(bits[m], bits[m] + 2 * J[m], 2) for m in range(d))
                exp.append(S[(a, b) + sl].ravel())
        exp = np.concatenate(exp)
        assert got.shape == exp.shape
        assert rel(got.astype(np.complex128), exp) <= (1e-7 if precision == 0 else 1e-14)


def test_multi_rhs_and_host_pointers():
    n, c, r = (10, 12, 6), 3, 5
    t_orth, par = W.green_dyadic_orthant(n, kh=W.KH_GREEN)
    x = W.random_vector(n, c, seed=14, nrhs=r)
    tf = W.orthant_to_full(t_orth, par)
    flags = bt.BTMV_SYM_BLOCK | bt.BTMV_SYM_PARITY
    for precision in (0, 1):
        ref = OE.embed_matvec(tf, round_input(x, precision))
        yd = run_btmv(t_orth, x, n, c, precision, 0, flags, par)
        yh = run_btmv(t_orth, x, n, c, precision, 0, flags, par, host=True)
        assert rel(yd, ref) <= TOL[precision]
        assert rel(yh, ref) <= TOL[precision]
        # each rhs independently equals its single-rhs product
        y1 = run_btmv(t_orth, x[2:3], n, c, precision, 0, flags, par)
        assert rel(yd[2:3], y1) <= TOL[precision]


def test_errors_and_noop():
    n = (8, 8)
    plan = bt.Plan(n, 1, 0)
    xd = torch.zeros((1, 1) + n, dtype=torch.complex64, device="cuda")
    yd = torch.zeros_like(xd)
    with pytest.raises(bt.BtmvError) as ei:
        plan.apply(xd, yd, 1)
    assert ei.value.status == bt.BTMV_E_STATE
    plan.set_kernel(W.random_generator(n, 1, seed=1))
    plan.apply(xd, yd, 0)                       # nrhs = 0: no-op
    with pytest.raises(bt.BtmvError) as ei:
        bt.btmv_apply(plan.handle, xd, xd, 1)   # x and y alias
    assert ei.value.status == bt.BTMV_E_ARG
    with pytest.raises(bt.BtmvError) as ei:
        plan.apply(xd, yd, 2)                   # more rhs than planned
    assert ei.value.status == bt.BTMV_E_ARG
    plan.close()


REG_SIZES = [(32,), (64,), (128,), (256,), (512,), (32, 64), (8, 256), (512, 8), (64, 32, 128),
             (16, 32, 64), (3, 128, 5), (128, 128, 16),
             (24,), (48,), (60,), (96,), (192,), (24, 48), (60, 12), (96, 24, 6), (12, 30, 48), (20, 192),
             (160,), (320,), (384,), (768,), (160, 12), (320, 20), (384, 6), (3, 768), (160, 8, 10),
             (84,), (84, 24), (12, 10, 84), (84, 6, 14),
             (640,), (1024,), (640, 6), (4, 1024), (3, 2, 640), (2, 3, 1024)]


@pytest.mark.parametrize("n", REG_SIZES)
@pytest.mark.parametrize("c", [1, 3])
@pytest.mark.parametrize("algo", [0, 1])
def test_register_kernels_vs_oracle_and_generic(n, c, algo):
    """Power-of-two lines take the register-resident kernels; they must agree
    with the oracle and with the generic shared-memory kernels."""
    t = W.random_generator(n, c, seed=300 + sum(n))
    x = W.random_vector(n, c, seed=301, nrhs=2)
    y = run_btmv(t, x, n, c, 0, algo)
    ref = OE.embed_matvec(t, round_input(x, 0))
    assert rel(y, ref) <= 1e-5
    plan = bt.Plan(n, c, 0, algo, max_rhs=2, flags=bt.BTMV_FLAG_GENERIC)
    plan.set_kernel(t)
    xd = torch.from_numpy(x.astype(np.complex64)).cuda()
    yd = torch.zeros_like(xd)
    plan.apply(xd, yd, 2)
    torch.cuda.synchronize()
    plan.close()
    yg = yd.cpu().numpy().astype(np.complex128)
    assert rel(yg, ref) <= 1e-5
    assert rel(y, yg) <= 2e-6


FULL_COMPRESSED = [((12, 10, 8), 3, "green"), ((16, 32, 64), 3, "green"), ((5, 7, 9), 3, "green"),
                   ((96, 24, 6), 3, "green"), ((64, 64), 1, "green"), ((24, 96), 1, "green"),
                   ((6, 10), 3, "skew"), ((8, 6, 4), 3, "skew")]


@pytest.mark.parametrize("n,c,kind", FULL_COMPRESSED)
@pytest.mark.parametrize("generic", [False, True])
def test_full_embedding_reads_the_compressed_store(n, c, kind, generic):
    """The plain embedding on the mirror-compressed store (Sec. II.C
    symmetric / skew storage): its full-grid frequencies f > n are read at
    2n - f with the block's parity sign."""
    if kind == "skew":
        t_orth, par = W.skew_orthant(n, seed=71, c=c)
    elif c == 3:
        t_orth, par = W.green_dyadic_orthant(n, kh=W.KH_GREEN)
    else:
        t_orth, par = W.green_scalar_orthant(n, kh=W.KH_GREEN)
    flags = bt.BTMV_SYM_PARITY | (bt.BTMV_SYM_BLOCK if c == 3 else 0)
    x = W.random_vector(n, c, seed=72, nrhs=2)
    tf = W.orthant_to_full(t_orth, par)
    for precision in (0, 1):
        plan = bt.Plan(n, c, precision, bt.BTMV_ALGO_FULL, max_rhs=2,
                       flags=bt.BTMV_FLAG_GENERIC if generic else 0)
        try:
            plan.set_kernel(t_orth, flags, par)
            assert plan.info["compressed"] == 1
            dt = torch.complex64 if precision == 0 else torch.complex128
            xd = torch.from_numpy(x).to(dt).cuda()
            yd = torch.zeros_like(xd)
            plan.apply(xd, yd, 2)
            torch.cuda.synchronize()
        finally:
            plan.close()
        ref = OE.embed_matvec(tf, round_input(x, precision))
        assert rel(yd.cpu().numpy().astype(np.complex128), ref) <= TOL[precision]


CUFFT_CASES = [((32,), 1, "random"), ((64, 64), 1, "random"), ((6, 5, 4), 3, "random"), ((12, 10, 8), 3, "green"),
               ((16, 32, 64), 3, "green"), ((8, 6, 4), 3, "skew"), ((24, 96), 1, "green")]


@pytest.mark.parametrize("n,c,kind", CUFFT_CASES)
def test_cufft_embedding_vs_oracle(n, c, kind):
    """BTMV_ALGO_FULL_CUFFT (the comparator: cuFFT transforms, own pad,
    multiply and projection kernels) on the full and the compressed store."""
    if kind == "random":
        t_in, par, flags = W.random_generator(n, c, seed=81), None, 0
        tf = t_in
    else:
        if kind == "skew":
            t_in, par = W.skew_orthant(n, seed=82, c=c)
        elif c == 3:
            t_in, par = W.green_dyadic_orthant(n, kh=W.KH_GREEN)
        else:
            t_in, par = W.green_scalar_orthant(n, kh=W.KH_GREEN)
        flags = bt.BTMV_SYM_PARITY | (bt.BTMV_SYM_BLOCK if c == 3 else 0)
        tf = W.orthant_to_full(t_in, par)
    x = W.random_vector(n, c, seed=83, nrhs=2)
    for precision in (0, 1):
        y = run_btmv(t_in, x, n, c, precision, bt.BTMV_ALGO_FULL_CUFFT, flags, par)
        ref = OE.embed_matvec(tf, round_input(x, precision))
        assert rel(y, ref) <= TOL[precision]


LEAF3_CASES = [((6, 5, 64), "green", 1), ((5, 3, 64), "green", 3), ((3, 4, 128), "green", 2),
               ((2, 3, 256), "green", 1), ((2, 2, 512), "green", 2), ((1, 2, 1024), "green", 1),
               ((4, 6, 128), "skew", 2), ((6, 64), "skew", 3), ((3, 2, 2, 256), "skew", 1)]


@pytest.mark.parametrize("n,kind,nrhs", LEAF3_CASES)
def test_component_in_thread_leaf(n, kind, nrhs, monkeypatch):
    """The c = 3 leaf that holds all three components of a line in one
    thread group (64..1024-point lines, compressed block-symmetric store,
    right-hand sides ordered fastest) against the FP64 oracle and against the
    component-group leaf (BTMV_LEAF3=0)."""
    if kind == "skew":
        t_orth, par = W.skew_orthant(n, seed=91, c=3)
    else:
        t_orth, par = W.green_dyadic_orthant(n, kh=W.KH_GREEN)
    flags = bt.BTMV_SYM_BLOCK | bt.BTMV_SYM_PARITY
    x = W.random_vector(n, 3, seed=92, nrhs=nrhs)
    ref = OE.embed_matvec(W.orthant_to_full(t_orth, par), round_input(x, 0))
    monkeypatch.setenv("BTMV_LEAF3", "0")
    yg = run_btmv(t_orth, x, n, 3, 0, 0, flags, par)
    assert rel(yg, ref) <= 1e-5
    monkeypatch.setenv("BTMV_LEAF3", "1")
    y3 = run_btmv(t_orth, x, n, 3, 0, 0, flags, par)
    assert rel(y3, ref) <= 1e-5
    assert rel(y3, yg) <= 2e-6


TMA_SIZES = [(32, 64), (64, 32, 128), (16, 32, 64), (128, 128, 16), (256, 32), (32, 256, 16), (64, 64, 64)]


@pytest.mark.parametrize("n", TMA_SIZES)
@pytest.mark.parametrize("c", [1, 3])
def test_tma_staged_passes(n, c, monkeypatch):
    """The strided passes with TMA-staged input tiles (persistent blocks,
    2-D box copies completing on mbarriers) do the same arithmetic as the
    register passes: the apply must match the FP64 oracle and the default
    kernels bit for bit."""
    t = W.random_generator(n, c, seed=400 + sum(n))
    x = W.random_vector(n, c, seed=401, nrhs=2)
    monkeypatch.setenv("BTMV_PASS_TMA", "0")
    y0 = run_btmv(t, x, n, c, 0, 0)
    monkeypatch.setenv("BTMV_PASS_TMA", "1")
    y1 = run_btmv(t, x, n, c, 0, 0)
    ref = OE.embed_matvec(t, round_input(x, 0))
    assert rel(y1, ref) <= 1e-5
    assert np.array_equal(y0, y1)


def test_tma_pass_wait_limit_reports_timeout_and_context_survives():
    """A TMA-staged pass whose mbarrier is told to expect more bytes than the
    copy delivers gives up its wait after the limit and reports it (no
    fault); afterwards a split apply whose merges take the TMA-staged kernel
    (256-point lines) still matches the FP64 oracle."""
    st = bt.btmv_selftest_tma_timeout(50)
    assert st == bt.BTMV_E_TIMEOUT, bt.btmv_last_error()
    n, c = (256, 16), 3
    t = W.random_generator(n, c, seed=411)
    x = W.random_vector(n, c, seed=412)
    y = run_btmv(t, x, n, c, 0, 0)
    assert rel(y, OE.embed_matvec(t, round_input(x, 0))) <= 1e-5


def test_plan_clone_shares_the_symbol():
    n, c = (10, 12, 8), 3
    t_orth, par = W.green_dyadic_orthant(n, kh=W.KH_GREEN)
    master = bt.Plan(n, c, 0)
    master.set_kernel(t_orth, bt.BTMV_SYM_BLOCK | bt.BTMV_SYM_PARITY, par)
    clone = master.clone(max_rhs=2)
    info_m, info_c = master.info, clone.info
    assert info_c["has_symbol"] == 1 and info_c["symbol_bytes"] == info_m["symbol_bytes"]
    assert info_c["max_rhs"] == 2
    x = W.random_vector(n, c, seed=15, nrhs=2)
    xd = torch.from_numpy(x.astype(np.complex64)).cuda()
    ym, yc = torch.zeros_like(xd), torch.zeros_like(xd)
    master.apply(xd[:1], ym[:1], 1)
    master.close()                          # the clone keeps the shared symbol alive
    clone.apply(xd, yc, 2)
    torch.cuda.synchronize()
    assert torch.equal(ym[:1], yc[:1])
    ref = OE.embed_matvec(W.orthant_to_full(t_orth, par), round_input(x, 0))
    assert rel(yc.cpu().numpy().astype(np.complex128), ref) <= 1e-5
    # a new generator on the clone builds its own symbol
    t2 = W.random_generator(n, c, seed=16)
    clone.set_kernel(t2)
    clone.apply(xd, yc, 2)
    torch.cuda.synchronize()
    assert rel(yc.cpu().numpy().astype(np.complex128), OE.embed_matvec(t2, round_input(x, 0))) <= 1e-5
    clone.close()


@pytest.mark.parametrize("n,r", [((16, 20, 24), 9), ((32, 32, 32), 16), ((12, 60), 8)])
@pytest.mark.parametrize("flag", ["shared", "tensor"])
def test_multi_rhs_contraction_paths(n, r, flag):
    """All right-hand sides of a line share each symbol read (CUDA cores), or
    the c x c x nrhs contraction runs on tensor cores (TF32 high/low split):
    both match the oracle within the complex64 gate and the default path."""
    c = 3
    if len(n) == 3:
        t_orth, par = W.green_dyadic_orthant(n, kh=W.KH_GREEN)
        flags_s = bt.BTMV_SYM_BLOCK | bt.BTMV_SYM_PARITY
        tf = W.orthant_to_full(t_orth, par)
    else:
        t_orth, par, flags_s = W.random_generator(n, c, seed=17), None, 0
        tf = t_orth
    x = W.random_vector(n, c, seed=18, nrhs=r)
    pf = bt.BTMV_FLAG_SHARED_RHS if flag == "shared" else bt.BTMV_FLAG_TENSOR_CORE
    plan = bt.Plan(n, c, 0, max_rhs=r, flags=pf)
    plan.set_kernel(t_orth, flags_s, par)
    xd = torch.from_numpy(x.astype(np.complex64)).cuda()
    yd = torch.zeros_like(xd)
    plan.apply(xd, yd, r)
    torch.cuda.synchronize()
    plan.close()
    y = yd.cpu().numpy().astype(np.complex128)
    ref = OE.embed_matvec(tf, round_input(x, 0))
    assert rel(y, ref) <= 1e-5
    y0 = run_btmv(t_orth, x, n, c, 0, 0, flags_s, par)
    assert rel(y, y0) <= 2e-6


@pytest.mark.parametrize("n", [(16, 12, 20), (128, 64, 32), (6, 8, 10, 12)])
def test_two_stream_schedule(n):
    """The two top-level subtrees on two streams give the one-stream result."""
    c = 3 if len(n) == 3 else 1
    t = W.random_generator(n, c, seed=19)
    x = W.random_vector(n, c, seed=20, nrhs=2)
    plan = bt.Plan(n, c, 0, max_rhs=2, flags=bt.BTMV_FLAG_TWO_STREAMS)
    plan.set_kernel(t)
    assert plan.info["workspace_bytes"] == (2 * len(n) - 3) * plan.info["vector_bytes"] * 2
    xd = torch.from_numpy(x.astype(np.complex64)).cuda()
    yd = torch.zeros_like(xd)
    for _ in range(2):
        plan.apply(xd, yd, 2)
    torch.cuda.synchronize()
    plan.close()
    y = yd.cpu().numpy().astype(np.complex128)
    assert rel(y, OE.embed_matvec(t, round_input(x, 0))) <= 1e-5
    assert rel(y, run_btmv(t, x, n, c, 0, 0)) <= 1e-6


@pytest.mark.parametrize("n, c, form, algo", [((6, 5), 1, "full", 0), ((4, 3, 5), 3, "full", 0),
                                              ((7, 6), 3, "block", 1), ((5, 4, 6), 3, "green", 0),
                                              ((6, 8), 1, "skew1", 0), ((4, 6, 8), 3, "skew", 1)])
def test_adjoint_symbol(n, c, form, algo):
    """BTMV_SYM_ADJOINT: the apply equals conj(T)^T x, T the oracle's dense
    matrix of the generator as given (every storage form)."""
    par = None
    if form == "full":
        t = W.random_generator(n, c, seed=71)
        tf, flags = t, 0
    elif form == "block":
        t = W.random_generator(n, c, seed=72)
        t = 0.5 * (t + t.transpose(1, 0, *range(2, t.ndim)))          # t_ab = t_ba
        tf, flags = t, bt.BTMV_SYM_BLOCK
    elif form == "green":
        t, par = W.green_dyadic_orthant(n, kh=0.45)
        tf, flags = W.orthant_to_full(t, par), bt.BTMV_SYM_BLOCK | bt.BTMV_SYM_PARITY
    else:
        t, par = W.skew_orthant(n, seed=73, c=c)
        tf, flags = W.orthant_to_full(t, par), bt.BTMV_SYM_BLOCK | bt.BTMV_SYM_PARITY
    x = W.random_vector(n, c, seed=74, nrhs=2)
    T = OT.dense_matrix(tf)
    ref = (T.conj().T @ x.reshape(2, -1).T).T.reshape(x.shape)
    y = run_btmv(t, x, n, c, 0, algo, flags | bt.BTMV_SYM_ADJOINT, par)
    assert rel(y, ref) <= 1e-5
    y2 = run_btmv(t, x, n, c, 1, algo, flags | bt.BTMV_SYM_ADJOINT, par)
    assert rel(y2, ref) <= 1e-12


@pytest.mark.parametrize("n", [(2, 3, 2, 3, 4), (3, 2, 4, 2, 2, 3), (2, 2, 2, 3, 32), (2, 3, 2, 2, 24, 2)])
@pytest.mark.parametrize("c", [1, 3])
@pytest.mark.parametrize("precision", [0, 1])
def test_five_and_six_levels(n, c, precision):
    """d = 5 and 6 (Table 1's deeper levels), split algorithm, against the
    oracle; the plain embedding stops at d = 4."""
    t = W.random_generator(n, c, seed=90 + len(n))
    x = W.random_vector(n, c, seed=91, nrhs=2)
    y = run_btmv(t, x, n, c, precision, 0)
    ref = OE.embed_matvec(t, round_input(x, precision))
    assert rel(y, ref) <= TOL[precision]


def test_pipelined_host_applies():
    """btmv_apply_host_async: a run of pipelined applies on pinned host
    buffers gives each input's own result (bit for bit the synchronous
    host-pointer apply), whatever the overlap of copies and applies."""
    n, c = (24, 20, 32), 3
    t, par = W.green_dyadic_orthant(n, kh=0.4)
    plan = bt.Plan(n, c, 0, max_rhs=2)
    plan.set_kernel(t, 3, par)
    try:
        xs = [torch.from_numpy(W.random_vector(n, c, seed=200 + k, nrhs=2).astype(np.complex64)).pin_memory()
              for k in range(5)]
        ys = [torch.zeros_like(x).pin_memory() for x in xs]
        for k in range(12):                                  # slots reused several times
            bt.btmv_apply_host_async(plan.handle, xs[k % 5], ys[k % 5], 2 if k % 3 else 1)
        bt.btmv_host_wait(plan.handle)
        for k in range(7, 12):                               # the last write of each y
            r = 2 if k % 3 else 1
            ya = np.zeros((r,) + xs[k % 5].shape[1:], dtype=np.complex64)
            bt.btmv_apply(plan.handle, xs[k % 5].numpy()[:r].copy(), ya, r)
            assert np.array_equal(ys[k % 5].numpy()[:r], ya), k
        ref = OE.embed_matvec(W.orthant_to_full(t, par), xs[0].numpy().astype(np.complex128))
        bt.btmv_apply_host_async(plan.handle, xs[0], ys[0], 2)
        bt.btmv_host_wait(plan.handle)
        assert rel(ys[0].numpy().astype(np.complex128), ref) <= 1e-5
    finally:
        plan.close()


def test_stream_order_with_foreign_kernels():
    """The register kernels start early (programmatic dependent launch) but
    read their input only after the previous kernel of the stream: an input
    written by a torch kernel right before each apply, and an output read
    by one right after, match the oracle every time."""
    n, c = (32, 24, 64), 3
    t, par = W.green_dyadic_orthant(n, kh=0.3)
    plan = bt.Plan(n, c, 0, max_rhs=1)
    plan.set_kernel(t, 3, par)
    try:
        srcs = [W.random_vector(n, c, seed=300 + k).astype(np.complex64) for k in range(3)]
        dsrc = [torch.from_numpy(v).cuda() for v in srcs]
        x = torch.zeros_like(dsrc[0])
        y = torch.zeros_like(x)
        sums = []
        for k in range(6):
            x.copy_(dsrc[k % 3] * (k + 1))          # a torch kernel writes x just before the apply
            plan.apply(x, y, 1)
            sums.append((y * 2).sum())              # a torch kernel reads y just after
        torch.cuda.synchronize()
        tf = W.orthant_to_full(t, par)
        for k in range(6):
            ref = OE.embed_matvec(tf, srcs[k % 3].astype(np.complex128) * (k + 1))
            got = complex(sums[k].item()) / 2
            assert abs(got - ref.sum()) <= 1e-5 * np.abs(ref).sum(), k
    finally:
        plan.close()


@pytest.mark.parametrize("n", [(11,), (13, 7), (17, 5, 4), (127, 3), (3, 2, 101), (61, 9), (2, 3, 4, 13)])
@pytest.mark.parametrize("c", [1, 3])
@pytest.mark.parametrize("precision", [0, 1])
def test_sizes_that_are_not_seven_smooth(n, c, precision):
    """Prime and other non-7-smooth sizes: the split plan runs the operator
    zero-padded to the next 7-smooth sizes and returns the caller's part."""
    t = W.random_generator(n, c, seed=400 + sum(n))
    x = W.random_vector(n, c, seed=401, nrhs=2)
    y = run_btmv(t, x, n, c, precision, 0)
    ref = OE.embed_matvec(t, round_input(x, precision))
    assert rel(y, ref) <= TOL[precision]
    yh = run_btmv(t, x, n, c, precision, 0, host=True)             # host pointers (staging)
    assert rel(yh, ref) <= TOL[precision]


@pytest.mark.parametrize("n", [(13, 11, 7), (31, 17, 29)])
def test_padded_green_parity_and_adjoint(n):
    """Compressed parity store and the adjoint on a padded (prime-size) plan."""
    t, par = W.green_dyadic_orthant(n, kh=0.3)
    tf = W.orthant_to_full(t, par)
    x = W.random_vector(n, 3, seed=402, nrhs=1)
    y = run_btmv(t, x, n, 3, 0, 0, bt.BTMV_SYM_BLOCK | bt.BTMV_SYM_PARITY, par)
    assert rel(y, OE.embed_matvec(tf, round_input(x, 0))) <= 1e-5
    plan = bt.Plan(n, 3, 0)
    assert tuple(plan.info["n"]) == n
    plan.close()
    tz, parz = W.skew_orthant(n, seed=403)
    yf = run_btmv(tz, x, n, 3, 1, 0, bt.BTMV_SYM_BLOCK | bt.BTMV_SYM_PARITY, parz)
    assert rel(yf, OE.embed_matvec(W.orthant_to_full(tz, parz), x)) <= 1e-12
    z = W.random_vector(n, 3, seed=404, nrhs=1)
    yz = run_btmv(tz, z, n, 3, 1, 0, bt.BTMV_SYM_BLOCK | bt.BTMV_SYM_PARITY | bt.BTMV_SYM_ADJOINT, parz)
    lhs = np.vdot(z, yf)
    rhs = np.vdot(yz, x)
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(yf) * np.linalg.norm(z)


FUSED_CASES = [((1, 64, 64), "green", 1), ((3, 64, 64), "green", 2), ((7, 64, 64), "skew", 3),
               ((16, 64, 64), "green", 1), ((5, 64, 64), "skew", 1), ((2, 3, 64, 64), "skew", 2),
               ((3, 1, 64, 64), "skew", 1), ((2, 2, 2, 64, 64), "skew", 1), ((11, 64, 64), "green", 2)]


def _fused_launches(d):
    """Forward split + merge per node of levels 0..d-3, one fused launch per level-(d-2) node."""
    return sum(2 << m for m in range(d - 2)) + (1 << (d - 2))


def _fused_instance(n, kind, nrhs):
    if kind == "skew":
        t_orth, par = W.skew_orthant(n, seed=95, c=3)
    else:
        t_orth, par = W.green_dyadic_orthant(n, kh=W.KH_GREEN)
    x = W.random_vector(n, 3, seed=96, nrhs=nrhs)
    return t_orth, par, x


@pytest.mark.parametrize("n,kind,nrhs", FUSED_CASES)
@pytest.mark.parametrize("streams", [0, 1])
def test_fused_two_levels(n, kind, nrhs, streams, monkeypatch):
    """The last two levels of Algorithm 1 as one kernel per level-1 node
    (dim-1 split, leaf along dim 2, dim-1 merge on a shared-memory slab)
    against the FP64 oracle and the unfused schedule, with and without the
    two-stream traversal, d = 3..5; a d = 3 fused plan launches 4 kernels
    per apply (fusion forced on these small grids)."""
    monkeypatch.setenv("BTMV_FUSE_MIN_BLOCKS", "0")
    t_orth, par, x = _fused_instance(n, kind, nrhs)
    flags = bt.BTMV_SYM_BLOCK | bt.BTMV_SYM_PARITY
    extra = bt.BTMV_FLAG_TWO_STREAMS if streams else 0
    ref = OE.embed_matvec(W.orthant_to_full(t_orth, par), round_input(x, 0))
    y0 = run_btmv(t_orth, x, n, 3, 0, 0, flags, par, flags=extra)
    y1 = run_btmv(t_orth, x, n, 3, 0, 0, flags, par, flags=extra | bt.BTMV_FLAG_FUSED_LEVELS)
    assert rel(y1, ref) <= 1e-5
    assert rel(y1, y0) <= 1e-6
    plan = bt.Plan(n, 3, 0, max_rhs=nrhs, flags=bt.BTMV_FLAG_FUSED_LEVELS)
    try:
        plan.set_kernel(t_orth, flags, par)
        assert plan.info["launches_per_apply"] == _fused_launches(len(n))
    finally:
        plan.close()


@pytest.mark.parametrize("n,c,sym", [((4, 32, 32), 3, 3), ((4, 64, 64), 1, 0), ((4, 64, 64), 3, 0),
                                     ((2, 64, 64, 8), 3, 3), ((4, 64, 128), 3, 3)])
def test_fused_flag_ignored_elsewhere(n, c, sym):
    """Plans without a fused kernel (other sizes, c = 1, the full store,
    d = 4) run the unfused schedule under BTMV_FLAG_FUSED_LEVELS."""
    if sym and len(n) == 3:
        t, par = W.green_dyadic_orthant(n, kh=W.KH_GREEN)
    elif sym:
        t, par = W.skew_orthant(n, seed=97, c=3)
    else:
        t, par = W.random_generator(n, c, seed=97), None
    x = W.random_vector(n, c, seed=98, nrhs=1)
    full = W.orthant_to_full(t, par) if par is not None else t
    ref = OE.embed_matvec(full, round_input(x, 0))
    y = run_btmv(t, x, n, c, 0, 0, sym, par, flags=bt.BTMV_FLAG_FUSED_LEVELS)
    assert rel(y, ref) <= 1e-5
    plan = bt.Plan(n, c, 0, max_rhs=1, flags=bt.BTMV_FLAG_FUSED_LEVELS)
    try:
        plan.set_kernel(t, sym, par)
        d = len(n)
        assert plan.info["launches_per_apply"] == sum(2 << m for m in range(d - 1)) + (1 << (d - 2))
    finally:
        plan.close()


def test_fused_two_levels_profile(monkeypatch):
    """BTMV_FLAG_PROFILE reports the fused launches under their own kind."""
    monkeypatch.setenv("BTMV_FUSE_MIN_BLOCKS", "0")
    n = (4, 64, 64)
    t_orth, par, x = _fused_instance(n, "green", 1)
    plan = bt.Plan(n, 3, 0, max_rhs=1, flags=bt.BTMV_FLAG_FUSED_LEVELS | bt.BTMV_FLAG_PROFILE)
    try:
        plan.set_kernel(t_orth, bt.BTMV_SYM_BLOCK | bt.BTMV_SYM_PARITY, par)
        xd = torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64))).cuda()
        yd = torch.zeros_like(xd)
        bt.btmv_profile_read(plan.handle)
        plan.apply(xd, yd, 1)
        prof = bt.btmv_profile_read(plan.handle)
        assert prof["fused_levels"][1] == 2
        assert prof["leaf"][1] == 0
        assert prof["fwd_split"][1] == 1 and prof["merge"][1] == 1
    finally:
        plan.close()


def test_fused_two_levels_grid_threshold(monkeypatch):
    """By default an apply fuses from 4 blocks per SM (nrhs n_0 >= 4 x SMs),
    2 with the two-stream traversal: on (76, 64, 64) eight right-hand sides
    fuse and one does not, on (38, 64, 64) eight fuse only with two streams,
    and every result matches the oracle."""
    monkeypatch.delenv("BTMV_FUSE_MIN_BLOCKS", raising=False)
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    n0 = -(-4 * nsm // 8)
    n, r = (n0, 64, 64), 8
    t_orth, par = W.green_dyadic_orthant(n, kh=W.KH_GREEN)
    x = W.random_vector(n, 3, seed=99, nrhs=r)
    ref = OE.embed_matvec(W.orthant_to_full(t_orth, par), round_input(x, 0))
    plan = bt.Plan(n, 3, 0, max_rhs=r, flags=bt.BTMV_FLAG_FUSED_LEVELS | bt.BTMV_FLAG_PROFILE)
    try:
        plan.set_kernel(t_orth, bt.BTMV_SYM_BLOCK | bt.BTMV_SYM_PARITY, par)
        assert plan.info["launches_per_apply"] == 4
        xd = torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64))).cuda()
        yd = torch.zeros_like(xd)
        bt.btmv_profile_read(plan.handle)
        plan.apply(xd, yd, r)
        prof = bt.btmv_profile_read(plan.handle)
        assert prof["fused_levels"][1] == 2 and prof["leaf"][1] == 0
        assert rel(yd.cpu().numpy().astype(np.complex128), ref) <= 1e-5
        y1 = torch.zeros_like(xd[:1])
        plan.apply(xd[:1], y1, 1)
        prof = bt.btmv_profile_read(plan.handle)
        assert prof["fused_levels"][1] == 0 and prof["leaf"][1] == 2
        assert rel(y1.cpu().numpy().astype(np.complex128), ref[:1]) <= 1e-5
    finally:
        plan.close()
    # half the grid: unfused on one stream, fused with the two-stream traversal
    n2 = (-(-2 * nsm // 8), 64, 64)
    t2, par2 = W.green_dyadic_orthant(n2, kh=W.KH_GREEN)
    x2 = W.random_vector(n2, 3, seed=100, nrhs=r)
    ref2 = OE.embed_matvec(W.orthant_to_full(t2, par2), round_input(x2, 0))
    x2d = torch.from_numpy(np.ascontiguousarray(x2.astype(np.complex64))).cuda()
    for extra, fused in ((0, False), (bt.BTMV_FLAG_TWO_STREAMS, True)):
        plan = bt.Plan(n2, 3, 0, max_rhs=r, flags=bt.BTMV_FLAG_FUSED_LEVELS | bt.BTMV_FLAG_PROFILE | extra)
        try:
            plan.set_kernel(t2, bt.BTMV_SYM_BLOCK | bt.BTMV_SYM_PARITY, par2)
            y2 = torch.zeros_like(x2d)
            bt.btmv_profile_read(plan.handle)
            plan.apply(x2d, y2, r)
            prof = bt.btmv_profile_read(plan.handle)
            assert (prof["fused_levels"][1] == 2) == fused
            assert rel(y2.cpu().numpy().astype(np.complex128), ref2) <= 1e-5
        finally:
            plan.close()


SMALL2D_CASES = [("random", 0, 1), ("random", 1, 3), ("green", 0, 2), ("green", 1, 1), ("skew", 1, 2),
                 ("mixed", 0, 1), ("mixed", 1, 2)]


def _small2d_instance(kind, n):
    if kind == "random":
        return W.random_generator(n, 1, seed=301), None, 0
    if kind == "green":
        t, par = W.green_scalar_orthant(n, kh=W.KH_GREEN)
        return t, par, bt.BTMV_SYM_PARITY
    if kind == "skew":
        t, par = W.skew_orthant(n, seed=302, c=1)
        return t, par, bt.BTMV_SYM_PARITY
    par = np.array([[[1, -1]]], dtype=np.int8)
    return W.random_parity_orthant(n, 1, seed=303, parity=par, block_sym=False), par, bt.BTMV_SYM_PARITY


@pytest.mark.parametrize("kind,precision,nrhs", SMALL2D_CASES)
@pytest.mark.parametrize("cluster", ["16", "8"])
def test_small_two_level_cluster_apply(kind, precision, nrhs, cluster, monkeypatch):
    """d = 2, c = 1, 64 x 64: the whole split apply as one launch of a
    thread-block cluster per right-hand side (columns, leaf rows and columns
    again exchanged through distributed shared memory) against the FP64
    oracle and the three-kernel schedule, on the full store and on the
    compressed store with even, odd and mixed parities; clusters of 16 CTAs
    (taken on GB300) and of 8 (the form for devices that refuse 16)."""
    if cluster == "8":
        monkeypatch.setenv("BTMV_SMALL2D_CLUSTER", "8")
    n = (64, 64)
    t, par, sym = _small2d_instance(kind, n)
    x = W.random_vector(n, 1, seed=304, nrhs=nrhs)
    full = W.orthant_to_full(t, par) if par is not None else t
    ref = OE.embed_matvec(full, round_input(x, precision))
    monkeypatch.setenv("BTMV_SMALL2D", "0")
    y0 = run_btmv(t, x, n, 1, precision, 0, sym, par)
    monkeypatch.delenv("BTMV_SMALL2D")
    y1 = run_btmv(t, x, n, 1, precision, 0, sym, par)
    assert rel(y1, ref) <= TOL[precision]
    assert rel(y1, y0) <= (1e-6 if precision == 0 else 1e-13)
    plan = bt.Plan(n, 1, precision, max_rhs=nrhs, flags=bt.BTMV_FLAG_PROFILE)
    try:
        plan.set_kernel(t, sym, par)
        assert plan.info["launches_per_apply"] == 1
        dt = np.complex64 if precision == 0 else np.complex128
        xd = torch.from_numpy(np.ascontiguousarray(x.astype(dt))).cuda()
        yd = torch.zeros_like(xd)
        bt.btmv_profile_read(plan.handle)
        plan.apply(xd, yd, nrhs)
        prof = bt.btmv_profile_read(plan.handle)
        assert prof["fused_levels"][1] == 1 and prof["leaf"][1] == 0
        assert rel(yd.cpu().numpy().astype(np.complex128), ref) <= TOL[precision]
    finally:
        plan.close()


def test_small_two_level_more_rhs_than_one_grid_dimension(monkeypatch):
    """More than 65535 right-hand sides (the grid's y limit) run the
    one-launch d = 2 apply in chunks: the right-hand sides on both sides of
    each chunk boundary and the last one against the FP64 oracle, sampled
    right-hand sides against the three-kernel schedule."""
    n, r = (64, 64), 65535 + 4
    t = W.random_generator(n, 1, seed=305)
    g = torch.Generator(device="cuda").manual_seed(306)
    xd = torch.randn((r, 1) + n, dtype=torch.complex64, device="cuda", generator=g)
    ys = {}
    for env in ("1", "0"):
        monkeypatch.setenv("BTMV_SMALL2D", env)
        plan = bt.Plan(n, 1, 0, max_rhs=r)
        try:
            plan.set_kernel(t)
            yd = torch.zeros_like(xd)
            plan.apply(xd, yd, r)
            torch.cuda.synchronize()
            ys[env] = yd
        finally:
            plan.close()
    for q in (0, 65534, 65535, r - 1):
        xq = xd[q:q + 1].cpu().numpy().astype(np.complex128)
        ref = OE.embed_matvec(t, xq)
        assert rel(ys["1"][q:q + 1].cpu().numpy().astype(np.complex128), ref) <= 1e-5
    idx = torch.arange(0, r, 997, device="cuda")
    a = ys["1"][idx].cpu().numpy().astype(np.complex128)
    b = ys["0"][idx].cpu().numpy().astype(np.complex128)
    assert rel(a, b) <= 1e-6


FUSED128_CASES = [((4, 128, 128), "green", 1), ((3, 128, 128), "skew", 2), ((2, 2, 128, 128), "skew", 1)]


@pytest.mark.parametrize("n,kind,nrhs", FUSED128_CASES)
@pytest.mark.parametrize("streams", [0, 1])
def test_fused_two_levels_cluster_128(n, kind, nrhs, streams, monkeypatch):
    """The last two levels fused for 128 x 128 slabs, one 16-CTA cluster per
    slab exchanging columns and rows through distributed shared memory,
    against the FP64 oracle and the unfused schedule.  The form is opt-in
    (BTMV_FUSE_CLUSTER=1; it measured slower than the unfused schedule), and
    fusion is forced on these small grids."""
    monkeypatch.setenv("BTMV_FUSE_MIN_BLOCKS", "0")
    monkeypatch.setenv("BTMV_FUSE_CLUSTER", "1")
    t_orth, par, x = _fused_instance(n, kind, nrhs)
    flags = bt.BTMV_SYM_BLOCK | bt.BTMV_SYM_PARITY
    extra = bt.BTMV_FLAG_TWO_STREAMS if streams else 0
    ref = OE.embed_matvec(W.orthant_to_full(t_orth, par), round_input(x, 0))
    y0 = run_btmv(t_orth, x, n, 3, 0, 0, flags, par, flags=extra)
    y1 = run_btmv(t_orth, x, n, 3, 0, 0, flags, par, flags=extra | bt.BTMV_FLAG_FUSED_LEVELS)
    assert rel(y1, ref) <= 1e-5
    assert rel(y1, y0) <= 1e-6
    plan = bt.Plan(n, 3, 0, max_rhs=nrhs, flags=bt.BTMV_FLAG_FUSED_LEVELS | bt.BTMV_FLAG_PROFILE)
    try:
        plan.set_kernel(t_orth, flags, par)
        assert plan.info["launches_per_apply"] == _fused_launches(len(n))
        xd = torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64))).cuda()
        yd = torch.zeros_like(xd)
        bt.btmv_profile_read(plan.handle)
        plan.apply(xd, yd, nrhs)
        prof = bt.btmv_profile_read(plan.handle)
        assert prof["fused_levels"][1] == 1 << (len(n) - 2) and prof["leaf"][1] == 0
    finally:
        plan.close()


def test_fused_flag_leaves_128_slabs_unfused_by_default(monkeypatch):
    """Without BTMV_FUSE_CLUSTER=1 a 128 x 128-slab plan under
    BTMV_FLAG_FUSED_LEVELS runs the unfused schedule."""
    monkeypatch.setenv("BTMV_FUSE_MIN_BLOCKS", "0")
    monkeypatch.delenv("BTMV_FUSE_CLUSTER", raising=False)
    n = (2, 128, 128)
    t_orth, par, x = _fused_instance(n, "green", 1)
    plan = bt.Plan(n, 3, 0, max_rhs=1, flags=bt.BTMV_FLAG_FUSED_LEVELS)
    try:
        plan.set_kernel(t_orth, bt.BTMV_SYM_BLOCK | bt.BTMV_SYM_PARITY, par)
        assert plan.info["launches_per_apply"] == 8
    finally:
        plan.close()
