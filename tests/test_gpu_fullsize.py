"""Parity at the benchmark sizes, in the launch configuration bench.py
times: 128^3 c=3 Green (complex64) against the full FP64 oracle, 256^3 Green
and skew against the direct sum at sampled output points (the definition,
evaluated point by point), plus the skew identity x^T T x = 0 at full size."""
import os

import numpy as np
import pytest

import workloads as W
from oracle import embed as OE
from oracle import toeplitz as OT
from tests.gpu_util import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

bt = pytest.importorskip("paper_2406_17981_gb300.btmv")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    bt.lib()


def _apply(n, t, par, flags_sym, x, plan_flags=0):
    plan = bt.Plan(n, 3, bt.BTMV_C64, bt.BTMV_ALGO_SPLIT, max_rhs=1, flags=plan_flags)
    plan.set_kernel(t, flags_sym, par)
    xd = torch.from_numpy(x).cuda()
    yd = torch.zeros_like(xd)
    plan.apply(xd, yd, 1)
    torch.cuda.synchronize()
    plan.close()
    return yd.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("plan_flags", [0, bt.BTMV_FLAG_TWO_STREAMS])
def test_128_cubed_green_against_full_oracle(plan_flags):
    cfg = W.WORKLOADS["d3_128_c3_green_c64"]
    n = cfg["n"]
    t, par = W.green_dyadic_orthant(n, kh=cfg["kh"])
    x = W.random_vector(n, 3, seed=cfg["x_seed"]).astype(np.complex64)
    y = _apply(n, t, par, 3, x, plan_flags)
    ref = OE.embed_matvec(W.orthant_to_full(t, par), x.astype(np.complex128),
                          workers=len(os.sched_getaffinity(0)))
    assert rel(y, ref) <= 1e-5


@pytest.mark.parametrize("name", ["d3_256_c3_green_c64", "d3_256_c3_skew_c64"])
def test_256_cubed_sampled_direct_sum(name):
    cfg = W.WORKLOADS[name]
    n = cfg["n"]
    if cfg["kind"] == "green":
        t, par = W.green_dyadic_orthant(n, kh=cfg["kh"])
    else:
        t, par = W.skew_orthant(n, seed=cfg["t_seed"])
    x = W.random_vector(n, 3, seed=cfg["x_seed"]).astype(np.complex64)
    y = _apply(n, t, par, 3, x)
    rng = np.random.default_rng(41)
    pts = [tuple(int(v) for v in rng.integers(0, n)) for _ in range(12)]
    pts += [(0, 0, 0), (255, 255, 255), (0, 255, 128)]            # corners and a face
    ref = OT.direct_points(W.orthant_to_full(t, par), x.astype(np.complex128), pts)[:, 0]
    got = np.stack([y[(0, slice(None)) + p] for p in pts])
    assert rel(got, ref) <= 1e-5
    if cfg["kind"] == "skew":
        xr = x.astype(np.complex128)
        assert abs(np.sum(xr * y)) <= 1e-5 * np.linalg.norm(xr) * np.linalg.norm(y)


@pytest.mark.parametrize("name", ["d3_128_c3_green_c64", "d3_256_c3_skew_c64"])
def test_adjoint_identity_at_benchmark_size(name):
    """<T x, z> = <x, T^H z> with T^H from BTMV_SYM_ADJOINT, at full size."""
    cfg = W.WORKLOADS[name]
    n = cfg["n"]
    if cfg["kind"] == "green":
        t, par = W.green_dyadic_orthant(n, kh=cfg["kh"])
    else:
        t, par = W.skew_orthant(n, seed=cfg["t_seed"])
    x = W.random_vector(n, 3, seed=cfg["x_seed"]).astype(np.complex64)
    z = W.random_vector(n, 3, seed=cfg["x_seed"] + 100).astype(np.complex64)
    tx = _apply(n, t, par, 3, x)
    thz = _apply(n, t, par, 3 | bt.BTMV_SYM_ADJOINT, z)
    lhs = np.vdot(z.astype(np.complex128), tx)           # <T x, z> as z^H (T x)
    rhs = np.vdot(thz, x.astype(np.complex128))          # (T^H z)^H x
    scale = np.linalg.norm(tx) * np.linalg.norm(z)
    assert abs(lhs - rhs) <= 1e-5 * scale


def test_fused_levels_bench_size_sampled_direct_sum():
    """The fused last two levels (BTMV_FLAG_FUSED_LEVELS) at the size
    bench.py times them, 512 x 64 x 64 c=3 Green with 8 right-hand sides:
    every right-hand side against the direct sum at the grid's corners and
    six sampled points, and the whole output against the unfused schedule."""
    import bench
    from tests.gpu_util import sample_points
    n, r = (512, 64, 64), 8
    assert (bench.FUSED_N, bench.FUSED_RHS) == (n, r)
    t, par = W.green_dyadic_orthant(n, kh=W.KH_GREEN)
    x = W.random_vector(n, 3, seed=37, nrhs=r).astype(np.complex64)
    xd = torch.from_numpy(x).cuda()
    ys = []
    for fl in (bt.BTMV_FLAG_FUSED_LEVELS | bt.BTMV_FLAG_PROFILE, 0):
        plan = bt.Plan(n, 3, bt.BTMV_C64, bt.BTMV_ALGO_SPLIT, max_rhs=r, flags=fl)
        plan.set_kernel(t, 3, par)
        yd = torch.zeros_like(xd)
        if fl:
            bt.btmv_profile_read(plan.handle)
        plan.apply(xd, yd, r)
        if fl:
            assert bt.btmv_profile_read(plan.handle)["fused_levels"][1] == 2
        ys.append(yd.cpu().numpy().astype(np.complex128))
        plan.close()
    yf, yu = ys
    assert rel(yf, yu) <= 1e-6
    pts = sample_points(n, 6, seed=43)
    vals = OT.direct_points(W.orthant_to_full(t, par), x.astype(np.complex128), pts)   # [npts][r][c]
    got = np.stack([yf[(slice(None), slice(None)) + p] for p in pts])
    assert rel(got, vals) <= 1e-5
