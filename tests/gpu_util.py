"""Helpers for GPU tests: run the CUDA path through the C ABI."""
import numpy as np

TOL = {0: 1e-5, 1: 1e-12}        # rel-L2 gates: complex64, complex128


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def round_input(x, precision):
    """The vector the GPU actually sees, back in complex128 for the oracle."""
    dt = np.complex64 if precision == 0 else np.complex128
    return x.astype(dt).astype(np.complex128)


def run_btmv(t, x, n, c, precision, algo=0, sym_flags=0, parity=None, nrhs=None, host=False, flags=0):
    import torch

    from paper_2406_17981_gb300 import btmv as bt
    nrhs = x.shape[0] if nrhs is None else nrhs
    plan = bt.Plan(n, c, precision, algo, max_rhs=max(1, nrhs), flags=flags)
    try:
        plan.set_kernel(t, sym_flags, parity)
        dt = np.complex64 if precision == 0 else np.complex128
        xa = np.ascontiguousarray(x.astype(dt))
        if host:
            ya = np.zeros_like(xa)
            plan.apply(xa, ya, nrhs)
            return ya.astype(np.complex128)
        xd = torch.from_numpy(xa).cuda()
        yd = torch.zeros_like(xd)
        plan.apply(xd, yd, nrhs)
        torch.cuda.synchronize()
        return yd.cpu().numpy().astype(np.complex128)
    finally:
        plan.close()


def sample_points(n, count, seed):
    """The 2^d corners of the grid plus `count` seeded random points."""
    import itertools
    rng = np.random.default_rng(seed)
    pts = [tuple(int(c) for c in corner) for corner in itertools.product(*[(0, m - 1) for m in n])]
    pts += [tuple(int(v) for v in rng.integers(0, n)) for _ in range(count)]
    return pts


def batched_instance_oracle(job):
    """FP64 oracle values of one batched instance at sampled points (runs in
    a worker process).  job = (n, kh, nrhs, x_seed, points); the Green
    generator and x are redrawn from their seeds, x rounded to complex64 as
    the GPU saw it.  Returns [npts][r][c]."""
    import workloads as W
    from oracle import toeplitz as OT
    n, kh, nrhs, x_seed, pts = job
    t_orth, par = W.green_dyadic_orthant(n, kh=kh)
    x = round_input(W.random_vector(n, 3, seed=x_seed, nrhs=nrhs), 0)
    return OT.direct_points(W.orthant_to_full(t_orth, par), x, pts)


def oracle_pool_map(fn, jobs):
    """Map fn over jobs in a pool of spawned processes (never forked: the
    parent holds a CUDA context)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import os
    workers = max(1, min(len(jobs), len(os.sched_getaffinity(0))))
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(fn, jobs))
