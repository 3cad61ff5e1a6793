"""btmv_apply_host_noalloc: the host-pointer apply that allocates nothing.

It serves callers that cannot let the library call cudaMalloc when they call
it (device memory reserved by another allocator, or a loop that must stay off
the driver's allocation path): x and y are staged through a fixed device
array compiled into the library.  Its result must equal btmv_apply's on the
same plan and inputs, call after call, since the shared array keeps whatever
the previous call left in it.

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import workloads as W
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


def _device_apply(plan, x):
    xd = torch.from_numpy(x).cuda()
    yd = torch.zeros_like(xd)
    bt.btmv_apply(plan.handle, xd, yd, x.shape[0])
    torch.cuda.synchronize()
    return yd.cpu().numpy()


@pytest.mark.parametrize("precision", [bt.BTMV_C64, bt.BTMV_C128])
def test_noalloc_matches_btmv_apply_on_consecutive_calls(precision):
    n, c, r = (24, 20, 16), 3, 2
    t_orth, par = W.green_dyadic_orthant(n, kh=W.KH_GREEN)
    dt = np.complex64 if precision == bt.BTMV_C64 else np.complex128
    tol = 1e-5 if precision == bt.BTMV_C64 else 1e-12
    plan = bt.Plan(n, c, precision, bt.BTMV_ALGO_SPLIT, max_rhs=r)
    plan.set_kernel(t_orth, bt.BTMV_SYM_BLOCK | bt.BTMV_SYM_PARITY, par)
    try:
        for call, seed in enumerate((41, 42)):          # two calls in a row, new x each time
            x = W.random_vector(n, c, seed=seed, nrhs=r).astype(dt)
            y = np.full_like(x, np.nan)
            bt.btmv_apply_host_noalloc(plan.handle, x, y, r)
            y_ref = _device_apply(plan, x)
            assert np.all(np.isfinite(y)), f"call {call}"
            assert rel(y.astype(np.complex128), y_ref.astype(np.complex128)) <= tol, f"call {call}"
    finally:
        plan.close()


def test_noalloc_rejects_vectors_beyond_the_limit():
    n, c = (64, 64, 64), 3                                # 6 MiB per rhs (complex64)
    t_orth, par = W.green_dyadic_orthant(n, kh=W.KH_GREEN)
    plan = bt.Plan(n, c, bt.BTMV_C64, bt.BTMV_ALGO_SPLIT, max_rhs=3)
    plan.set_kernel(t_orth, bt.BTMV_SYM_BLOCK | bt.BTMV_SYM_PARITY, par)
    try:
        x = W.random_vector(n, c, seed=43, nrhs=3).astype(np.complex64)   # 18 MiB > 16 MiB
        y = np.zeros_like(x)
        with pytest.raises(bt.BtmvError) as ei:
            bt.btmv_apply_host_noalloc(plan.handle, x, y, 3)
        assert ei.value.status == bt.BTMV_E_UNSUPPORTED
        assert "BTMV_NOALLOC_MAX_BYTES" in str(ei.value)
        # within the limit it runs and agrees with btmv_apply
        x2 = np.ascontiguousarray(x[:2])
        y2 = np.zeros_like(x2)
        bt.btmv_apply_host_noalloc(plan.handle, x2, y2, 2)
        assert rel(y2.astype(np.complex128), _device_apply(plan, x2).astype(np.complex128)) <= 1e-5
    finally:
        plan.close()


def test_noalloc_allocates_no_device_memory():
    """The property the entry point exists for: once the library's staging
    array is resident (the first call on the device), calls on a freshly
    created plan leave the device's free memory unchanged."""
    n, c, r = (24, 20, 16), 3, 2
    t_orth, par = W.green_dyadic_orthant(n, kh=W.KH_GREEN)
    x = W.random_vector(n, c, seed=44, nrhs=r).astype(np.complex64)
    y = np.zeros_like(x)
    warm = bt.Plan(n, c, bt.BTMV_C64, bt.BTMV_ALGO_SPLIT, max_rhs=r)
    warm.set_kernel(t_orth, bt.BTMV_SYM_BLOCK | bt.BTMV_SYM_PARITY, par)
    plan = bt.Plan(n, c, bt.BTMV_C64, bt.BTMV_ALGO_SPLIT, max_rhs=r)
    plan.set_kernel(t_orth, bt.BTMV_SYM_BLOCK | bt.BTMV_SYM_PARITY, par)
    try:
        bt.btmv_apply_host_noalloc(warm.handle, x, y, r)   # loads the array and the kernels
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(4):
            bt.btmv_apply_host_noalloc(plan.handle, x, y, r)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert rel(y.astype(np.complex128), _device_apply(plan, x).astype(np.complex128)) <= 1e-5
    finally:
        warm.close()
        plan.close()


def test_noalloc_padded_size_on_a_torch_stream():
    """Sizes that are not 7-smooth (23 is prime) run zero-padded inside the
    plan; the call is issued on a non-default torch stream."""
    n, c, r = (23, 20, 16), 3, 1
    t_orth, par = W.green_dyadic_orthant(n, kh=W.KH_GREEN)
    plan = bt.Plan(n, c, bt.BTMV_C64, bt.BTMV_ALGO_SPLIT, max_rhs=r)
    plan.set_kernel(t_orth, bt.BTMV_SYM_BLOCK | bt.BTMV_SYM_PARITY, par)
    stream = torch.cuda.Stream()
    try:
        for seed in (45, 46):
            x = W.random_vector(n, c, seed=seed, nrhs=r).astype(np.complex64)
            y = np.full_like(x, np.nan)
            bt.btmv_apply_host_noalloc(plan.handle, x, y, r, stream=stream)
            assert np.all(np.isfinite(y))
            assert rel(y.astype(np.complex128), _device_apply(plan, x).astype(np.complex128)) <= 1e-5
    finally:
        plan.close()


def test_noalloc_success_clears_an_earlier_error():
    n, c = (8, 8, 8), 3
    t_orth, par = W.green_dyadic_orthant(n, kh=W.KH_GREEN)
    plan = bt.Plan(n, c, bt.BTMV_C64, bt.BTMV_ALGO_SPLIT, max_rhs=1)
    plan.set_kernel(t_orth, bt.BTMV_SYM_BLOCK | bt.BTMV_SYM_PARITY, par)
    try:
        x = W.random_vector(n, c, seed=47).astype(np.complex64)
        y = np.zeros_like(x)
        with pytest.raises(bt.BtmvError):
            bt.btmv_apply_host_noalloc(plan.handle, x, y, 2)     # nrhs beyond the plan's max_rhs
        assert bt.btmv_last_error() != ""
        bt.btmv_apply_host_noalloc(plan.handle, x, y, 1)
        assert bt.btmv_last_error() == ""
    finally:
        plan.close()


def test_noalloc_on_the_fused_and_one_launch_paths(monkeypatch):
    """The staged apply also takes the fused forms btmv_apply takes -- the
    last two levels in one kernel (BTMV_FLAG_FUSED_LEVELS, forced here) and
    the one-launch d = 2 apply -- and matches btmv_apply on two calls in a
    row."""
    monkeypatch.setenv("BTMV_FUSE_MIN_BLOCKS", "0")
    cases = []
    n3 = (2, 64, 64)
    t3, par3 = W.green_dyadic_orthant(n3, kh=W.KH_GREEN)
    p3 = bt.Plan(n3, 3, bt.BTMV_C64, bt.BTMV_ALGO_SPLIT, max_rhs=1, flags=bt.BTMV_FLAG_FUSED_LEVELS)
    p3.set_kernel(t3, bt.BTMV_SYM_BLOCK | bt.BTMV_SYM_PARITY, par3)
    cases.append((p3, n3, 3, np.complex64, 1e-6))
    n2 = (64, 64)
    p2 = bt.Plan(n2, 1, bt.BTMV_C128, bt.BTMV_ALGO_SPLIT, max_rhs=1)
    p2.set_kernel(W.random_generator(n2, 1, seed=74))
    cases.append((p2, n2, 1, np.complex128, 1e-13))
    try:
        for plan, n, c, dt, tol in cases:
            for call in range(2):
                x = np.ascontiguousarray(W.random_vector(n, c, seed=75 + call, nrhs=1).astype(dt))
                y = np.zeros_like(x)
                bt.btmv_apply_host_noalloc(plan.handle, x, y, 1)
                assert rel(y.astype(np.complex128), _device_apply(plan, x).astype(np.complex128)) <= tol
    finally:
        for plan, *_ in cases:
            plan.close()
