"""btmv_apply_batched: many uneven problems in one persistent launch.

Every problem's result in the batch must match the FP64 oracle and its own
btmv_apply result (the alone-vs-in-the-mix check), replays of the captured
graph must reproduce the first result bit for bit, and the bounded waits of
the persistent kernel must report an expired wait without harming the
context.
"""
import numpy as np
import pytest

import workloads as W
from oracle import embed as OE
from tests.gpu_util import batched_instance_oracle, oracle_pool_map, rel, round_input, sample_points

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

bt = pytest.importorskip("paper_2406_17981_gb300.btmv")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    bt.lib()


def make_batch(insts, precision=bt.BTMV_C64):
    plans, xs, ys, refs_in = [], [], [], []
    dt = torch.complex64 if precision == bt.BTMV_C64 else torch.complex128
    for k, it in enumerate(insts):
        n, r = it["n"], it["nrhs"]
        t_orth, par = W.green_dyadic_orthant(n, kh=it["kh"])
        p = bt.Plan(n, 3, precision, bt.BTMV_ALGO_SPLIT, max_rhs=r)
        p.set_kernel(t_orth, bt.BTMV_SYM_BLOCK | bt.BTMV_SYM_PARITY, par)
        x = W.random_vector(n, 3, seed=it["x_seed"], nrhs=r)
        xd = torch.from_numpy(x).to(dt).cuda()
        plans.append(p)
        xs.append(xd)
        ys.append(torch.zeros_like(xd))
        refs_in.append((t_orth, par, x))
    return plans, xs, ys, refs_in


def run_batch(plans, xs, ys):
    bt.btmv_apply_batched([p.handle for p in plans], xs, ys, [x.shape[0] for x in xs])
    torch.cuda.synchronize()
    return [y.cpu().numpy().astype(np.complex128) for y in ys]


SMALL = [dict(n=(8, 12, 6), kh=0.4, nrhs=1, x_seed=1), dict(n=(24, 24, 24), kh=0.3, nrhs=3, x_seed=2),
         dict(n=(5, 7, 9), kh=0.5, nrhs=2, x_seed=3), dict(n=(32, 16, 60), kh=0.25, nrhs=1, x_seed=4),
         dict(n=(12, 20, 14), kh=0.6, nrhs=4, x_seed=5), dict(n=(3, 4, 5), kh=0.2, nrhs=1, x_seed=6)]


@pytest.mark.parametrize("precision", [bt.BTMV_C64, bt.BTMV_C128])
def test_batched_matches_oracle_and_single_apply(precision):
    plans, xs, ys, refs_in = make_batch(SMALL, precision)
    tol = 1e-5 if precision == bt.BTMV_C64 else 1e-12
    try:
        out = run_batch(plans, xs, ys)
        for p, x, y, (t_orth, par, xh) in zip(plans, xs, out, refs_in):
            ref = OE.embed_matvec(W.orthant_to_full(t_orth, par), round_input(xh, precision))
            assert rel(y, ref) <= tol
            ya = torch.zeros_like(x)
            p.apply(x, ya, x.shape[0])
            torch.cuda.synchronize()
            assert rel(y, ya.cpu().numpy().astype(np.complex128)) <= tol      # alone vs in the mix
        # graph replay: same arguments, bit-identical result
        for y in ys:
            y.zero_()
        again = run_batch(plans, xs, ys)
        for a, b in zip(out, again):
            assert np.array_equal(a, b)
        cfg = bt.btmv_batch_tuning([p.handle for p in plans], xs, ys, [x.shape[0] for x in xs])
        assert cfg["mode"] in (0, 1)
        if cfg["mode"] == 0:
            assert cfg["stages"] == sum(8 for _ in SMALL) and cfg["blocks"] >= 1
    finally:
        for p in plans:
            p.close()


_BATCH64_REF = {}


def _batch64_oracle(insts):
    """Per instance: 8 corners + 8 seeded random points and the FP64 oracle's
    direct sum there (computed once for the module, in spawned workers)."""
    if not _BATCH64_REF:
        jobs = [(it["n"], it["kh"], it["nrhs"], it["x_seed"], sample_points(it["n"], 8, seed=100 + i))
                for i, it in enumerate(insts)]
        refs = oracle_pool_map(batched_instance_oracle, jobs)
        for i, (job, ref) in enumerate(zip(jobs, refs)):
            _BATCH64_REF[i] = (job[4], ref)
    return _BATCH64_REF


@pytest.mark.parametrize("mode", ["tuned", "persistent"])
def test_batched_config_64_uneven_instances(mode, monkeypatch):
    """64 instances, each dim from {24,32,48,60,64,84,96}, kh ~ U[2pi/30, 2pi/10],
    1..16 right-hand sides, complex64.  Every instance is checked against the
    FP64 oracle's direct sum (Sec. I definition) at its 8 corners and 8
    random points, over all its right-hand sides and components, and against
    its own btmv_apply (alone vs in the mix).  "tuned" runs the autotuner's
    choice, "persistent" forces the one-persistent-kernel mode."""
    if mode == "persistent":
        monkeypatch.setenv("BTMV_NO_AUTOTUNE", "1")
        monkeypatch.setenv("BTMV_BATCH_MODE", "0")
    insts = W.batched_instances()
    plans, xs, ys, refs_in = make_batch(insts)
    try:
        out = run_batch(plans, xs, ys)
        if mode == "persistent":
            cfg = bt.btmv_batch_tuning([p.handle for p in plans], xs, ys, [x.shape[0] for x in xs])
            assert cfg["mode"] == 0
        oracle = _batch64_oracle(insts)
        for i, (p, x, y) in enumerate(zip(plans, xs, out)):
            ya = torch.zeros_like(x)
            p.apply(x, ya, x.shape[0])
            torch.cuda.synchronize()
            assert rel(y, ya.cpu().numpy().astype(np.complex128)) <= 1e-5, i
            pts, ref = oracle[i]
            got = np.stack([y[(slice(None), slice(None)) + q] for q in pts])
            err = rel(got, ref)
            assert err <= 1e-5, (i, insts[i]["n"], insts[i]["nrhs"], err)
    finally:
        for p in plans:
            p.close()


def test_batched_mixed_algorithms_run_in_sequence():
    n = (6, 8, 10)
    t_orth, par = W.green_dyadic_orthant(n, kh=0.3)
    pf = bt.Plan(n, 3, bt.BTMV_C64, bt.BTMV_ALGO_FULL)
    pf.set_kernel(t_orth, bt.BTMV_SYM_BLOCK | bt.BTMV_SYM_PARITY, par)
    ps = bt.Plan(n, 3, bt.BTMV_C128, bt.BTMV_ALGO_SPLIT)
    ps.set_kernel(t_orth, bt.BTMV_SYM_BLOCK | bt.BTMV_SYM_PARITY, par)
    x = W.random_vector(n, 3, seed=9)
    xf = torch.from_numpy(x.astype(np.complex64)).cuda()
    xs = torch.from_numpy(x).cuda()
    yf, ys = torch.zeros_like(xf), torch.zeros_like(xs)
    try:
        bt.btmv_apply_batched([pf.handle, ps.handle], [xf, xs], [yf, ys], [1, 1])
        torch.cuda.synchronize()
        ref = OE.embed_matvec(W.orthant_to_full(t_orth, par), x)
        assert rel(ys.cpu().numpy(), ref) <= 1e-12
        assert rel(yf.cpu().numpy().astype(np.complex128), ref) <= 1e-5
    finally:
        pf.close()
        ps.close()


def test_batched_argument_errors():
    n = (4, 4, 4)
    p = bt.Plan(n, 3, bt.BTMV_C64)
    p.set_kernel(W.green_dyadic_orthant(n, kh=0.3)[0], 3, W.green_dyadic_orthant(n, kh=0.3)[1])
    x = torch.zeros((1, 3) + n, dtype=torch.complex64, device="cuda")
    y = torch.zeros_like(x)
    try:
        with pytest.raises(bt.BtmvError) as ei:
            bt.btmv_apply_batched([p.handle, p.handle], [x, x], [y, y], [1, 1])
        assert ei.value.status == bt.BTMV_E_ARG
        with pytest.raises(bt.BtmvError) as ei:
            bt.btmv_apply_batched([p.handle], [x.cpu()], [y], [1])
        assert ei.value.status == bt.BTMV_E_ARG
        bt.btmv_apply_batched([], [], [], [])
    finally:
        p.close()


def test_persistent_wait_limit_reports_timeout_and_context_survives():
    st = bt.btmv_selftest_wait_timeout(200)
    assert st == bt.BTMV_E_TIMEOUT, bt.btmv_last_error()
    # the context is still usable: a normal batch runs and is correct
    plans, xs, ys, refs_in = make_batch(SMALL[:2])
    try:
        out = run_batch(plans, xs, ys)
        t_orth, par, xh = refs_in[0]
        ref = OE.embed_matvec(W.orthant_to_full(t_orth, par), round_input(xh, 0))
        assert rel(out[0], ref) <= 1e-5
    finally:
        for p in plans:
            p.close()


@pytest.mark.parametrize("mode", ["persistent", "branches", "direct"])
def test_each_batched_execution_mode(mode, monkeypatch):
    """Every execution mode of btmv_apply_batched matches the FP64 oracle
    (circulant embedding) and each problem's own apply: the persistent kernel
    (tuning off), the graph of branches, and the direct stream fork used by
    the server."""
    if mode in ("persistent", "branches"):
        monkeypatch.setenv("BTMV_NO_AUTOTUNE", "1")
        monkeypatch.setenv("BTMV_BATCH_MODE", "0" if mode == "persistent" else "1")
    else:
        monkeypatch.setenv("BTMV_BATCH_DIRECT", "1")
    insts = [dict(SMALL[k], x_seed=SMALL[k]["x_seed"] + 50 + 7 * len(mode)) for k in range(len(SMALL))]
    plans, xs, ys, refs_in = make_batch(insts)
    try:
        out = run_batch(plans, xs, ys)
        for p, x, y, (t_orth, par, xh) in zip(plans, xs, out, refs_in):
            ref = OE.embed_matvec(W.orthant_to_full(t_orth, par), round_input(xh, 0))
            assert rel(y, ref) <= 1e-5                                          # FP64 oracle
            ya = torch.zeros_like(x)
            p.apply(x, ya, x.shape[0])
            torch.cuda.synchronize()
            assert rel(y, ya.cpu().numpy().astype(np.complex128)) <= 1e-5     # alone vs in the mix
        if mode != "direct":
            cfg = bt.btmv_batch_tuning([p.handle for p in plans], xs, ys, [x.shape[0] for x in xs])
            assert cfg["mode"] == (0 if mode == "persistent" else 1)
            # persistent: 8 stages per d = 3 problem; branches: its 8 kernel launches
            assert cfg["stages"] == 8 * len(insts)
    finally:
        for p in plans:
            p.close()


def test_batched_plans_with_fused_or_one_launch_applies(monkeypatch):
    """Plans whose own btmv_apply takes a fused form -- the last two levels
    in one kernel (BTMV_FLAG_FUSED_LEVELS, forced on a small grid) and the
    one-launch d = 2 apply -- run the plain schedule inside a batch; every
    problem of the batch still matches the FP64 oracle."""
    monkeypatch.setenv("BTMV_FUSE_MIN_BLOCKS", "0")
    specs = []
    n3 = (3, 64, 64)
    t3, par3 = W.green_dyadic_orthant(n3, kh=W.KH_GREEN)
    p3 = bt.Plan(n3, 3, bt.BTMV_C64, bt.BTMV_ALGO_SPLIT, max_rhs=2, flags=bt.BTMV_FLAG_FUSED_LEVELS)
    p3.set_kernel(t3, bt.BTMV_SYM_BLOCK | bt.BTMV_SYM_PARITY, par3)
    specs.append((p3, W.random_vector(n3, 3, seed=71, nrhs=2), W.orthant_to_full(t3, par3)))
    n2 = (64, 64)
    t2 = W.random_generator(n2, 1, seed=72)
    p2 = bt.Plan(n2, 1, bt.BTMV_C64, bt.BTMV_ALGO_SPLIT, max_rhs=3)
    p2.set_kernel(t2)
    assert p2.info["launches_per_apply"] == 1
    specs.append((p2, W.random_vector(n2, 1, seed=73, nrhs=3), t2))
    try:
        xs = [torch.from_numpy(x.astype(np.complex64)).cuda() for _, x, _ in specs]
        ys = [torch.zeros_like(x) for x in xs]
        bt.btmv_apply_batched([p.handle for p, _, _ in specs], xs, ys, [x.shape[0] for x in xs])
        torch.cuda.synchronize()
        for (p, x, tf), yd in zip(specs, ys):
            ref = OE.embed_matvec(tf, round_input(x, 0))
            assert rel(yd.cpu().numpy().astype(np.complex128), ref) <= 1e-5
    finally:
        for p, _, _ in specs:
            p.close()
