"""ctypes binding of libbtmv (include/btmv.h): argument marshalling only.

Every function here has the name of the C entry point it calls and forwards
plain pointers and sizes; all compute runs in the CUDA library.  Vectors may
be torch tensors (CUDA or CPU) or NumPy arrays; generators and parity arrays
are host NumPy arrays.  Raises ``BtmvError`` (carrying the status code and
``btmv_last_error()``) on any non-zero status.  There is no fallback: if the
shared library is missing, loading fails loudly.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbtmv.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "btmv.h")

BTMV_OK, BTMV_E_ARG, BTMV_E_NOMEM, BTMV_E_CUDA, BTMV_E_STATE, BTMV_E_UNSUPPORTED, BTMV_E_TIMEOUT = range(7)
BTMV_C64, BTMV_C128 = 0, 1
BTMV_ALGO_SPLIT, BTMV_ALGO_FULL, BTMV_ALGO_FULL_CUFFT = 0, 1, 2
BTMV_SYM_NONE, BTMV_SYM_BLOCK, BTMV_SYM_PARITY, BTMV_SYM_ADJOINT = 0, 1, 2, 4
BTMV_FLAG_NONE, BTMV_FLAG_PROFILE, BTMV_FLAG_GENERIC, BTMV_FLAG_SHARED_RHS, BTMV_FLAG_TENSOR_CORE = 0, 1, 2, 4, 8
BTMV_FLAG_TWO_STREAMS, BTMV_FLAG_FUSED_LEVELS = 16, 32
KINDS = ["fwd_split", "leaf", "merge", "full_fwd", "full_leaf", "full_inv", "copy", "fused_levels"]
BTMV_K_NKINDS = len(KINDS)


class BtmvError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"btmv status {status}: {msg}")
        self.status = status


class btmv_plan_info_t(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("c", ctypes.c_int), ("precision", ctypes.c_int),
                ("algo", ctypes.c_int), ("max_rhs", ctypes.c_int), ("n", ctypes.c_int * 6),
                ("nsym", ctypes.c_int), ("compressed", ctypes.c_int), ("has_symbol", ctypes.c_int),
                ("launches_per_apply", ctypes.c_int), ("symbol_bytes", ctypes.c_size_t),
                ("workspace_bytes", ctypes.c_size_t), ("table_bytes", ctypes.c_size_t),
                ("vector_bytes", ctypes.c_size_t)]


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, u32, st = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_int
        L.btmv_plan_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(ctypes.c_int32), i32, i32, i32, i32, u32]
        L.btmv_plan_clone.argtypes = [vp, i32, u32, ctypes.POINTER(vp)]
        L.btmv_set_kernel.argtypes = [vp, ctypes.POINTER(ctypes.c_double), u32, ctypes.POINTER(ctypes.c_int8), vp]
        L.btmv_apply.argtypes = [vp, vp, vp, i32, vp]
        L.btmv_apply_host_noalloc.argtypes = [vp, vp, vp, i32, vp]
        L.btmv_apply_host_async.argtypes = [vp, vp, vp, i32, vp]
        L.btmv_host_wait.argtypes = [vp]
        L.btmv_apply_batched.argtypes = [i32, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                         ctypes.POINTER(ctypes.c_int), vp]
        L.btmv_destroy.argtypes = [vp]
        L.btmv_last_error.argtypes = []
        L.btmv_last_error.restype = ctypes.c_char_p
        L.btmv_plan_get_info.argtypes = [vp, ctypes.POINTER(btmv_plan_info_t)]
        L.btmv_get_symbol.argtypes = [vp, vp, ctypes.c_size_t]
        L.btmv_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
        L.btmv_batch_tuning.argtypes = [i32, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        L.btmv_selftest_wait_timeout.argtypes = [i32, vp]
        L.btmv_selftest_tma_timeout.argtypes = [i32, vp]
        for name in ("btmv_plan_create", "btmv_plan_clone", "btmv_set_kernel", "btmv_apply", "btmv_apply_host_noalloc",
                     "btmv_apply_batched", "btmv_batch_tuning", "btmv_selftest_wait_timeout",
                     "btmv_selftest_tma_timeout",
                     "btmv_destroy", "btmv_plan_get_info", "btmv_get_symbol", "btmv_profile_read"):
            getattr(L, name).restype = st
        _lib = L
    return _lib


def declared_symbols() -> list:
    """Entry points declared in include/btmv.h."""
    with open(HEADER) as fh:
        txt = fh.read()
    return re.findall(r"BTMV_API\s+[\w\s\*]+?\b(btmv_\w+)\s*\(", txt)


def _check(status: int):
    if status != BTMV_OK:
        raise BtmvError(status, lib().btmv_last_error().decode())


def _ptr(a) -> int:
    if a is None:
        return 0
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()          # torch tensor


def _stream(stream) -> int:
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream    # torch.cuda.Stream


def btmv_last_error() -> str:
    return lib().btmv_last_error().decode()


def btmv_plan_create(d, n, c, precision=BTMV_C64, algo=BTMV_ALGO_SPLIT, max_rhs=1, flags=0) -> int:
    arr = (ctypes.c_int32 * max(1, len(n)))(*[int(v) for v in n])
    h = ctypes.c_void_p()
    _check(lib().btmv_plan_create(ctypes.byref(h), int(d), arr, int(c), int(precision), int(algo),
                                  int(max_rhs), int(flags)))
    return h.value


def btmv_plan_clone(plan, max_rhs=1, flags=0) -> int:
    h = ctypes.c_void_p()
    _check(lib().btmv_plan_clone(plan, int(max_rhs), int(flags), ctypes.byref(h)))
    return h.value


def btmv_set_kernel(plan, t: np.ndarray, sym_flags=BTMV_SYM_NONE, parity=None, stream=None):
    t = np.ascontiguousarray(t, dtype=np.complex128)
    tp = t.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    pp = None
    if parity is not None:
        parity = np.ascontiguousarray(parity, dtype=np.int8)
        pp = parity.ctypes.data_as(ctypes.POINTER(ctypes.c_int8))
    _check(lib().btmv_set_kernel(plan, tp, int(sym_flags), pp, _stream(stream)))


def btmv_apply(plan, x, y, nrhs, stream=None):
    _check(lib().btmv_apply(plan, _ptr(x), _ptr(y), int(nrhs), _stream(stream)))


def btmv_apply_host_noalloc(plan, x, y, nrhs, stream=None):
    """y = T x for host x, y staged through the library's fixed device array
    (no device allocation; see include/btmv.h for the size limit)."""
    _check(lib().btmv_apply_host_noalloc(plan, _ptr(x), _ptr(y), int(nrhs), _stream(stream)))


def btmv_apply_host_async(plan, x, y, nrhs, stream=None):
    """Pipelined y = T x for pinned host x, y; y is valid after
    btmv_host_wait(plan)."""
    _check(lib().btmv_apply_host_async(plan, _ptr(x), _ptr(y), int(nrhs), _stream(stream)))


def btmv_host_wait(plan):
    _check(lib().btmv_host_wait(plan))


def btmv_apply_batched(plans, xs, ys, nrhs, stream=None):
    k = len(plans)
    P = (ctypes.c_void_p * max(1, k))(*plans)
    X = (ctypes.c_void_p * max(1, k))(*[_ptr(x) for x in xs])
    Y = (ctypes.c_void_p * max(1, k))(*[_ptr(y) for y in ys])
    R = (ctypes.c_int * max(1, k))(*[int(r) for r in nrhs])
    _check(lib().btmv_apply_batched(k, P, X, Y, R, _stream(stream)))


def btmv_batch_tuning(plans, xs, ys, nrhs) -> dict:
    k = len(plans)
    P = (ctypes.c_void_p * max(1, k))(*plans)
    X = (ctypes.c_void_p * max(1, k))(*[_ptr(x) for x in xs])
    Y = (ctypes.c_void_p * max(1, k))(*[_ptr(y) for y in ys])
    R = (ctypes.c_int * max(1, k))(*[int(r) for r in nrhs])
    out = (ctypes.c_int * 8)()
    _check(lib().btmv_batch_tuning(k, P, X, Y, R, out))
    keys = ("tile_lines", "leaf_lines", "leaf_rhs", "radix_order", "stages", "items", "blocks", "mode")
    return dict(zip(keys, list(out)))


def btmv_selftest_wait_timeout(timeout_ms=200, stream=None) -> int:
    """Runs the bounded-wait self test; returns the status code (expected:
    BTMV_E_TIMEOUT)."""
    return lib().btmv_selftest_wait_timeout(int(timeout_ms), _stream(stream))


def btmv_selftest_tma_timeout(timeout_ms=50, stream=None) -> int:
    """Runs the self test of the TMA-staged passes' bounded waits; returns the
    status code (expected: BTMV_E_TIMEOUT)."""
    return lib().btmv_selftest_tma_timeout(int(timeout_ms), _stream(stream))


def btmv_destroy(plan):
    _check(lib().btmv_destroy(plan))


def btmv_plan_get_info(plan) -> dict:
    info = btmv_plan_info_t()
    _check(lib().btmv_plan_get_info(plan, ctypes.byref(info)))
    out = {f: getattr(info, f) for f, _ in btmv_plan_info_t._fields_}
    out["n"] = list(info.n)[: info.d]
    return out


def btmv_get_symbol(plan) -> np.ndarray:
    info = btmv_plan_get_info(plan)
    dt = np.complex64 if info["precision"] == BTMV_C64 else np.complex128
    out = np.empty(info["symbol_bytes"] // np.dtype(dt).itemsize, dtype=dt)
    _check(lib().btmv_get_symbol(plan, out.ctypes.data, out.nbytes))
    return out


def btmv_profile_read(plan):
    ms = (ctypes.c_double * BTMV_K_NKINDS)()
    n = (ctypes.c_int64 * BTMV_K_NKINDS)()
    _check(lib().btmv_profile_read(plan, ms, n))
    return {KINDS[k]: (ms[k], n[k]) for k in range(BTMV_K_NKINDS)}


class Plan:
    """Owning wrapper: ``Plan(n, c, ...)``; ``set_kernel``, ``apply``, ``close``."""

    def __init__(self, n, c, precision=BTMV_C64, algo=BTMV_ALGO_SPLIT, max_rhs=1, flags=0, _handle=None):
        self.n = tuple(int(v) for v in n)
        self.d = len(self.n)
        self.c = int(c)
        self.precision = precision
        self.max_rhs = int(max_rhs)
        self.handle = _handle if _handle is not None else btmv_plan_create(self.d, self.n, self.c, precision,
                                                                           algo, max_rhs, flags)

    def clone(self, max_rhs=1, flags=0) -> "Plan":
        """A plan sharing this plan's symbol and tables, with its own workspace."""
        return Plan(self.n, self.c, self.precision, max_rhs=max_rhs, _handle=btmv_plan_clone(self.handle, max_rhs, flags))

    @property
    def info(self) -> dict:
        return btmv_plan_get_info(self.handle)

    def set_kernel(self, t, sym_flags=BTMV_SYM_NONE, parity=None, stream=None):
        btmv_set_kernel(self.handle, t, sym_flags, parity, stream)

    def apply(self, x, y, nrhs=None, stream=None):
        if nrhs is None:
            nrhs = x.shape[0] if len(x.shape) == self.d + 2 else 1
        btmv_apply(self.handle, x, y, nrhs, stream)
        return y

    def apply_host_async(self, x, y, nrhs=None, stream=None):
        """Pipelined apply on pinned host buffers; y is valid after host_wait()."""
        if nrhs is None:
            nrhs = x.shape[0] if len(x.shape) == self.d + 2 else 1
        btmv_apply_host_async(self.handle, x, y, nrhs, stream)
        return y

    def host_wait(self):
        btmv_host_wait(self.handle)

    def close(self):
        if self.handle:
            btmv_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
