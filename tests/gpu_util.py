"""Helpers for GPU tests: run the CUDA path through the C ABI."""
import numpy as np

TOL = {0: 1e-5, 1: 1e-12}        # rel-L2 gates: complex64, complex128


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def round_input(x, precision):
    """The vector the GPU actually sees, back in complex128 for the oracle."""
    dt = np.complex64 if precision == 0 else np.complex128
    return x.astype(dt).astype(np.complex128)


def run_btmv(t, x, n, c, precision, algo=0, sym_flags=0, parity=None, nrhs=None, host=False):
    import torch

    from paper_2406_17981_gb300 import btmv as bt
    nrhs = x.shape[0] if nrhs is None else nrhs
    plan = bt.Plan(n, c, precision, algo, max_rhs=max(1, nrhs))
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
