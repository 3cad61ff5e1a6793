"""Continuous-batching matvec server for concurrent iterative solves.

Many solves (BiCGSTAB on A = I - alpha T, T a block Toeplitz operator) run at
once.  Each admitted solve keeps its plan (symbol, twiddles, workspace) and
its Krylov vectors resident on the GPU; solves are admitted in arrival order
while their device footprint fits an HBM budget, and leave (freeing their
memory) when they finish or their client goes away.  Every scheduler tick
gathers the matvec requests of all solves that are ready and enqueues them as
ONE btmv_apply_batched call (each problem's launches forked onto a pool of
streams, since the mix changes every tick); while a batch is on the GPU the
host admits newcomers, runs the Krylov updates of finished requests and forms
the next batch, with up to ``max_inflight`` batches queued on the device.  A
batch whose launch fails is retried one solve at a time; a solve whose own
apply fails as well leaves the server and is reported.

The matvec is the library's (C ABI); the Krylov updates are plain torch
vector operations on the device.  Latency of a request = time from the moment
its input is ready to the moment its result is visible to the host.
"""
from __future__ import annotations

import collections
import math
import os
import time

import numpy as np

from . import analysis as A
from . import btmv as bt


class SolveSpec:
    """One solve: grid n (d = len(n)), c components, generator (t, parity,
    flags), right-hand side seed, alpha scaling of A = I - alpha T, and the
    matvec budget."""

    def __init__(self, n, c, t, parity, sym_flags, alpha, b_seed, max_matvecs=60, tol=1e-6, arrival=0.0,
                 name="", abort_after=None):
        self.n = tuple(int(v) for v in n)
        self.c = int(c)
        self.t, self.parity, self.sym_flags = t, parity, sym_flags
        self.alpha = float(alpha)
        self.b_seed = int(b_seed)
        self.max_matvecs = int(max_matvecs)
        self.tol = float(tol)
        self.arrival = float(arrival)
        self.name = name
        # the client gives up after this many matvecs (its solve leaves the
        # server unfinished); None: runs to convergence or max_matvecs
        self.abort_after = abort_after

    @property
    def op_key(self):
        """Solves with equal keys apply the same operator T and share its
        resident symbol."""
        return (self.n, self.c, id(self.t), self.sym_flags)

    def symbol_footprint(self) -> int:
        compressed = bool(self.sym_flags & bt.BTMV_SYM_PARITY)
        return A.symbol_bytes(self.n, self.c, 8, bool(self.sym_flags & bt.BTMV_SYM_BLOCK), compressed) + 64 * 1024

    def footprint(self, nvec=9) -> int:
        """Device bytes of one admitted solve on an operator already resident:
        workspace and nvec vectors (matvec input/output plus the BiCGSTAB
        vectors)."""
        d = len(self.n)
        V = A.vector_bytes(self.n, self.c, 1, 8)
        return (d - 1) * V + nvec * V


class Solve:
    """BiCGSTAB state machine; each call of ``step`` consumes the last matvec
    result and returns True when it has put a new request in ``self.xin``.

    The recurrence scalars stay on the device (no host synchronisation in a
    step); the residual norm of each iteration is copied to pinned host
    memory asynchronously and tested one iteration later."""

    def __init__(self, spec: SolveSpec, plan, torch, algo):
        self.spec = spec
        self.plan = plan
        self.torch = torch
        shape = (1, spec.c) + spec.n
        dev = "cuda"
        g = torch.Generator(device=dev)
        g.manual_seed(spec.b_seed)                 # seeded right-hand side, drawn on the device
        self.b = torch.randn(shape, generator=g, dtype=torch.complex64, device=dev)
        z = lambda: torch.zeros(shape, dtype=torch.complex64, device=dev)  # noqa: E731
        self.xin, self.yout = z(), z()
        self.x = z()
        self.r = self.b.clone()
        self.r0 = self.b.clone()
        self.p, self.v, self.s, self.tv = z(), z(), z(), z()
        one = torch.ones((), dtype=torch.complex64, device=dev)
        self.rho, self.alpha_k, self.omega = one.clone(), one.clone(), one.clone()
        self.bnorm = torch.linalg.vector_norm(self.b)
        self.res_host = torch.zeros((), dtype=torch.float32).pin_memory()
        self.res_host.fill_(1.0)
        self.res_ev = None
        self.phase = "start"
        self.matvecs = 0
        self.done = False
        self.aborted = False
        self.resid = 1.0
        self.algo = algo

    @staticmethod
    def _safe_div(th, a, b):
        return th.where(b != 0, a / th.where(b != 0, b, th.ones_like(b)), th.zeros_like(a))

    def step(self) -> bool:
        th = self.torch
        if self.spec.abort_after is not None and self.matvecs >= self.spec.abort_after:
            self.aborted = True                    # the client went away mid-solve
            self.done = True
            return False
        vd = lambda a, b: th.vdot(a.flatten(), b.flatten())  # noqa: E731
        al = self.spec.alpha
        if self.phase == "start":
            self.rho = vd(self.r0, self.r)
            self.p.copy_(self.r)
            self.xin.copy_(self.p)
            self.phase = "v"
            return True
        if self.phase == "v":                      # yout = T p  ->  v = A p
            self.v = self.p - al * self.yout
            self.alpha_k = self._safe_div(th, self.rho, vd(self.r0, self.v))
            self.s = self.r - self.alpha_k * self.v
            self.xin.copy_(self.s)
            self.phase = "t"
            return True
        if self.phase == "t":                      # yout = T s  ->  t = A s
            self.tv = self.s - al * self.yout
            tt = vd(self.tv, self.tv)
            self.omega = self._safe_div(th, vd(self.tv, self.s), tt)
            self.x += self.alpha_k * self.p + self.omega * self.s
            self.r = self.s - self.omega * self.tv
            # the previous iteration's residual, if its copy has landed
            prev = float(self.res_host) if (self.res_ev is not None and self.res_ev.query()) else 1.0
            res = th.linalg.vector_norm(self.r) / self.bnorm
            self.res_host.copy_(res, non_blocking=True)
            self.res_ev = th.cuda.Event()
            self.res_ev.record()
            if prev <= self.spec.tol or self.matvecs + 2 > self.spec.max_matvecs:
                self.res_ev.synchronize()
                return self._finish(float(self.res_host))
            rho_new = vd(self.r0, self.r)
            beta = self._safe_div(th, rho_new, self.rho) * self._safe_div(th, self.alpha_k, self.omega)
            self.rho = rho_new
            self.p = self.r + beta * (self.p - self.omega * self.v)
            self.xin.copy_(self.p)
            self.phase = "v"
            return True
        return False

    def _finish(self, res):
        self.resid = res
        self.done = True
        return False


class Server:
    """Continuous-batching server.  ``run(specs)`` plays the arrivals in
    ``spec.arrival`` (seconds after start) and returns statistics."""

    def __init__(self, budget_bytes=80 * 10 ** 9, max_inflight=2, algo=bt.BTMV_ALGO_SPLIT, batched=True,
                 record=None):
        import torch
        self.torch = torch
        self.budget = int(budget_bytes)
        self.max_inflight = max(1, int(max_inflight))
        self.algo = algo
        self.batched = batched
        self.record = record          # optional: {solve name: [(x, y), ...]} filled with matvec pairs
        self.streams = [torch.cuda.Stream() for _ in range(self.max_inflight)]
        self.upd = torch.cuda.Stream()  # Krylov updates: waits only on the batch whose results it reads
        self.ops = {}                 # operator key -> master plan holding the shared symbol

    def _cost(self, spec):
        return spec.footprint() + (0 if spec.op_key in self.ops else spec.symbol_footprint())

    def _admit(self, spec):
        # one resident symbol per operator; each solve gets a clone (own workspace)
        if spec.op_key not in self.ops:
            master = bt.Plan(spec.n, spec.c, bt.BTMV_C64, self.algo, max_rhs=1)
            master.set_kernel(spec.t, spec.sym_flags, spec.parity)
            self.ops[spec.op_key] = master
        return Solve(spec, self.ops[spec.op_key].clone(1), self.torch, self.algo)

    def _launch(self, batch, st):
        """Enqueue the batch's matvecs on st; returns (solves launched, solves
        lost).  A batch whose launch fails is retried one solve at a time;
        a solve whose own apply fails too is lost (reported by run)."""
        if self.batched:
            try:
                bt.btmv_apply_batched([s.plan.handle for s in batch], [s.xin for s in batch],
                                      [s.yout for s in batch], [1] * len(batch), stream=st)
                return batch, []
            except bt.BtmvError:
                pass                                           # retried one at a time below
        ok, lost = [], []
        for s in batch:
            try:
                bt.btmv_apply(s.plan.handle, s.xin, s.yout, 1, stream=st)
                ok.append(s)
            except bt.BtmvError:
                lost.append(s)
        return ok, lost

    def run(self, specs):
        th = self.torch
        if self.batched:
            os.environ.setdefault("BTMV_BATCH_DIRECT", "1")    # request mixes change every tick
        pending = collections.deque(sorted(specs, key=lambda s: s.arrival))
        active, ready = [], []
        inflight = collections.deque()                       # (event, [solves], t_launch)
        used = 0
        lat, t_ready = [], {}
        peak_active = 0
        nbatches = 0
        batch_sizes = []
        matvecs = 0
        t0 = time.perf_counter()
        finished, aborted, failed = [], [], []
        while pending or active or inflight:
            now = time.perf_counter() - t0
            # admission by arrival time and HBM budget
            while pending and pending[0].arrival <= now and used + self._cost(pending[0]) <= self.budget:
                spec = pending.popleft()
                used += self._cost(spec)
                with th.cuda.stream(self.upd):
                    s = self._admit(spec)
                    s.step()                                 # first request
                active.append(s)
                ready.append(s)
                t_ready[id(s)] = time.perf_counter()
            if pending and not active and not inflight and used + self._cost(pending[0]) > self.budget:
                raise RuntimeError(f"solve {pending[0].name} does not fit the HBM budget")
            peak_active = max(peak_active, len(active))
            # completions
            while inflight and (inflight[0][0].query() or len(inflight) >= self.max_inflight and not ready):
                ev, batch, _ = inflight.popleft()
                ev.synchronize()
                tdone = time.perf_counter()
                self.upd.wait_event(ev)
                for s in batch:
                    lat.append(tdone - t_ready.pop(id(s)))
                    s.matvecs += 1
                    if self.record is not None and s.spec.name in self.record:
                        self.record[s.spec.name].append((s.xin.clone(), s.yout.clone()))
                    with th.cuda.stream(self.upd):
                        more = s.step()
                    if more:
                        ready.append(s)
                        t_ready[id(s)] = time.perf_counter()
                    elif s.done:
                        active.remove(s)
                        used -= s.spec.footprint()
                        if s.aborted:
                            aborted.append(s)
                            s.plan.close()                   # its workspace goes back at once
                        else:
                            finished.append(s)
            # launch the ready requests as one batch
            if ready and len(inflight) < self.max_inflight:
                batch, ready = ready, []
                st = self.streams[nbatches % self.max_inflight]
                st.wait_stream(self.upd)                     # the batch reads the updated inputs
                batch, lost = self._launch(batch, st)
                for s in lost:                               # reported, removed, budget share returned
                    active.remove(s)
                    used -= s.spec.footprint()
                    t_ready.pop(id(s), None)
                    s.plan.close()
                    failed.append(s)
                if not batch:
                    continue
                ev = th.cuda.Event()
                ev.record(st)
                inflight.append((ev, batch, time.perf_counter()))
                nbatches += 1
                batch_sizes.append(len(batch))
                matvecs += len(batch)
            elif not ready and not inflight and pending:
                time.sleep(max(0.0, min(0.001, pending[0].arrival - (time.perf_counter() - t0))))
        th.cuda.synchronize()
        wall = time.perf_counter() - t0
        for s in finished:
            s.plan.close()
        for m in self.ops.values():
            m.close()
        self.ops = {}
        lat_ms = np.array(lat) * 1e3
        return {
            "matvecs": matvecs, "wall_s": wall, "matvecs_per_s": matvecs / wall,
            "p50_ms": float(np.percentile(lat_ms, 50)) if len(lat_ms) else None,
            "p99_ms": float(np.percentile(lat_ms, 99)) if len(lat_ms) else None,
            "batches": nbatches, "mean_batch": float(np.mean(batch_sizes)) if batch_sizes else 0.0,
            "peak_active_solves": peak_active, "solves": len(finished), "aborted": len(aborted),
            "failed": len(failed), "failed_names": [s.spec.name for s in failed],
            "budget_in_use_at_end": used,
            "max_residual": max((s.resid for s in finished), default=0.0),
            "solutions": {s.spec.name: s.x for s in finished},
            "rhs": {s.spec.name: s.b for s in finished},
        }


def scaled_alpha(spec_t, parity, sym_flags, n, c, target=0.5):
    """alpha = target / (c max over frequencies of |symbol entry|), a bound on
    the spectral norm of T, so that ||alpha T|| <= target < 1 and BiCGSTAB on
    I - alpha T converges.  Computed from the library's
    own symbol (full 2n-grid transform scaled back to the unnormalised
    coefficients)."""
    p = bt.Plan(n, c, bt.BTMV_C64, bt.BTMV_ALGO_SPLIT)
    p.set_kernel(spec_t, sym_flags, parity)
    S = bt.btmv_get_symbol(p.handle)
    p.close()
    scale = float(np.prod([2 * m for m in n]))
    return target / (c * float(np.abs(S).max()) * scale)
