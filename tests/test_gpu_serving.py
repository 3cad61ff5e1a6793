"""Continuous-batching server: concurrent BiCGSTAB solves share batched
matvec launches; each result must be the same alone and in the mix."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import embed as OE
from tests.gpu_util import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

bt = pytest.importorskip("paper_2406_17981_gb300.btmv")
serve = pytest.importorskip("paper_2406_17981_gb300.serve")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    bt.lib()


def make_specs(shapes, arrival_gap=0.002):
    specs = []
    for k, (n, c) in enumerate(shapes):
        if c == 3:
            t, par = W.green_dyadic_orthant(n, kh=W.KH_GREEN)
        else:
            t, par = W.green_scalar_orthant(n, kh=W.KH_GREEN)
        flags = (bt.BTMV_SYM_BLOCK if c == 3 else 0) | bt.BTMV_SYM_PARITY
        alpha = serve.scaled_alpha(t, par, flags, n, c)
        specs.append(serve.SolveSpec(n, c, t, par, flags, alpha, b_seed=100 + k, max_matvecs=40, tol=1e-5,
                                     arrival=k * arrival_gap, name=f"s{k}"))
    return specs


SHAPES = [((32, 32), 1), ((12, 16, 10), 3), ((48, 32), 1), ((16, 16, 16), 3), ((24, 20), 1),
          ((8, 12, 24), 3), ((64, 48), 1), ((20, 20, 12), 3)]


def test_solves_alone_and_in_the_mix_agree():
    specs = make_specs(SHAPES)
    record = {"s1": [], "s2": []}
    mix = serve.Server(budget_bytes=8 * 10 ** 9, record=record).run(specs)
    assert mix["solves"] == len(specs)
    assert mix["mean_batch"] > 1.0                 # requests really were batched together
    assert mix["max_residual"] <= 1e-4
    for spec in specs:
        alone = serve.Server(budget_bytes=8 * 10 ** 9).run([serve.SolveSpec(
            spec.n, spec.c, spec.t, spec.parity, spec.sym_flags, spec.alpha, spec.b_seed,
            spec.max_matvecs, spec.tol, 0.0, spec.name)])
        a = alone["solutions"][spec.name].cpu().numpy().astype(np.complex128)
        m = mix["solutions"][spec.name].cpu().numpy().astype(np.complex128)
        assert rel(m, a) <= 1e-5, spec.name
        # each request of a tick runs the problem's own kernels on a forked
        # stream, so a solve in the mix repeats its alone run bit for bit
        assert np.array_equal(m, a), spec.name
    # every recorded matvec of the mix equals the same matvec done alone
    for name, pairs in record.items():
        spec = specs[int(name[1:])]
        p = bt.Plan(spec.n, spec.c, bt.BTMV_C64)
        p.set_kernel(spec.t, spec.sym_flags, spec.parity)
        for x, y in pairs:
            ya = torch.zeros_like(y)
            p.apply(x, ya, 1)
            torch.cuda.synchronize()
            assert rel(y.cpu().numpy().astype(np.complex128), ya.cpu().numpy().astype(np.complex128)) <= 1e-5
            assert torch.equal(y, ya)
        p.close()


def test_solution_solves_the_system_by_the_oracle():
    specs = make_specs([((12, 16, 10), 3)])
    out = serve.Server().run(specs)
    spec = specs[0]
    x = out["solutions"][spec.name].cpu().numpy().astype(np.complex128)[0]
    b = out["rhs"][spec.name].cpu().numpy().astype(np.complex128)[0]
    Tx = OE.embed_matvec(W.orthant_to_full(spec.t, spec.parity), x)
    assert rel(x - spec.alpha * Tx, b) <= 1e-4


def test_admission_respects_the_hbm_budget():
    specs = make_specs([((16, 16, 16), 3)] * 4, arrival_gap=0.0)
    # room for the shared symbol and two solves at a time
    budget = specs[0].symbol_footprint() + specs[0].footprint() * 2 + 1
    out = serve.Server(budget_bytes=budget).run(specs)
    assert out["solves"] == 4
    assert out["peak_active_solves"] <= 2


def _alone(spec):
    return serve.Server(budget_bytes=8 * 10 ** 9).run([serve.SolveSpec(
        spec.n, spec.c, spec.t, spec.parity, spec.sym_flags, spec.alpha, spec.b_seed,
        spec.max_matvecs, spec.tol, 0.0, spec.name)])


def test_client_that_aborts_mid_solve():
    """A client that goes away after a few matvecs leaves the server: its
    workspace is released, and every other solve still equals its result
    alone."""
    specs = make_specs(SHAPES[:4])
    specs[1].abort_after = 3
    out = serve.Server(budget_bytes=8 * 10 ** 9).run(specs)
    assert out["aborted"] == 1 and out["solves"] == 3
    assert specs[1].name not in out["solutions"]
    for spec in (specs[0], specs[2], specs[3]):
        a = _alone(spec)["solutions"][spec.name].cpu().numpy().astype(np.complex128)
        m = out["solutions"][spec.name].cpu().numpy().astype(np.complex128)
        assert rel(m, a) <= 1e-5, spec.name
    # only the resident operators' symbols are still counted against the budget
    assert out["budget_in_use_at_end"] == sum(s.symbol_footprint() for s in specs)


def test_aborted_solve_frees_room_for_a_waiting_one():
    n = (16, 16, 16)
    t, par = W.green_dyadic_orthant(n, kh=W.KH_GREEN)              # one operator, shared symbol
    flags = bt.BTMV_SYM_BLOCK | bt.BTMV_SYM_PARITY
    alpha = serve.scaled_alpha(t, par, flags, n, 3)
    specs = [serve.SolveSpec(n, 3, t, par, flags, alpha, b_seed=500 + k, max_matvecs=40, tol=1e-5,
                             arrival=0.0, name=f"w{k}", abort_after=2 if k == 0 else None) for k in range(2)]
    budget = specs[0].symbol_footprint() + specs[0].footprint() + 1     # one solve at a time
    out = serve.Server(budget_bytes=budget).run(specs)
    assert out["aborted"] == 1 and out["solves"] == 1
    assert out["peak_active_solves"] == 1
    assert out["max_residual"] <= 1e-4


def test_failed_batch_is_retried_one_solve_at_a_time(monkeypatch):
    """Host-side fault: the batched call fails once; the server retries the
    batch's solves one at a time and every result equals its alone result."""
    specs = make_specs(SHAPES[:4])
    real = serve.bt.btmv_apply_batched
    calls = {"n": 0}

    def flaky(*args, **kw):
        calls["n"] += 1
        if calls["n"] == 2:
            raise bt.BtmvError(bt.BTMV_E_CUDA, "injected failure")
        return real(*args, **kw)

    monkeypatch.setattr(serve.bt, "btmv_apply_batched", flaky)
    out = serve.Server(budget_bytes=8 * 10 ** 9).run(specs)
    assert calls["n"] >= 2 and out["failed"] == 0 and out["solves"] == len(specs)
    for spec in specs:
        a = _alone(spec)["solutions"][spec.name].cpu().numpy().astype(np.complex128)
        m = out["solutions"][spec.name].cpu().numpy().astype(np.complex128)
        assert rel(m, a) <= 1e-5, spec.name


def test_solve_whose_apply_fails_is_reported(monkeypatch):
    """Host-side fault: batches always fail and one solve's own apply fails
    too; that solve is reported and removed, the others finish as alone."""
    specs = make_specs(SHAPES[:4])
    server = serve.Server(budget_bytes=8 * 10 ** 9)

    def fail_batch(*args, **kw):
        raise bt.BtmvError(bt.BTMV_E_CUDA, "injected batch failure")

    real_apply = serve.bt.btmv_apply
    bad = {}

    def apply(handle, x, y, nrhs, stream=None):
        if bad and handle == bad.get("h"):
            raise bt.BtmvError(bt.BTMV_E_CUDA, "injected apply failure")
        return real_apply(handle, x, y, nrhs, stream=stream)

    real_admit = server._admit

    def admit(spec):
        s = real_admit(spec)
        if spec.name == "s2":
            bad["h"] = s.plan.handle
        return s

    monkeypatch.setattr(serve.bt, "btmv_apply_batched", fail_batch)
    monkeypatch.setattr(serve.bt, "btmv_apply", apply)
    monkeypatch.setattr(server, "_admit", admit)
    out = server.run(specs)
    assert out["failed"] == 1 and out["failed_names"] == ["s2"] and out["solves"] == 3
    monkeypatch.undo()                                  # the alone runs use the real calls
    for spec in (specs[0], specs[1], specs[3]):
        a = _alone(spec)["solutions"][spec.name].cpu().numpy().astype(np.complex128)
        m = out["solutions"][spec.name].cpu().numpy().astype(np.complex128)
        assert rel(m, a) <= 1e-5, spec.name
