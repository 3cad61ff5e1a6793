"""C-ABI checks that need no GPU: the library builds, loads, exports every
symbol include/btmv.h declares, and rejects bad arguments before touching
the device."""
import ctypes

import pytest

from paper_2406_17981_gb300 import btmv as bt
from paper_2406_17981_gb300 import build as B


@pytest.fixture(scope="module")
def L():
    B.build()
    return bt.lib()


def test_header_declares_core_entry_points():
    syms = bt.declared_symbols()
    for name in ("btmv_plan_create", "btmv_set_kernel", "btmv_apply", "btmv_apply_batched",
                 "btmv_destroy", "btmv_last_error"):
        assert name in syms


def test_library_exports_every_declared_symbol(L):
    for name in bt.declared_symbols():
        assert hasattr(L, name), name
        ctypes.cast(getattr(L, name), ctypes.c_void_p)


@pytest.mark.parametrize("kw,status", [
    (dict(d=0, n=[4], c=1), bt.BTMV_E_ARG),
    (dict(d=7, n=[4] * 7, c=1), bt.BTMV_E_ARG),
    (dict(d=1, n=[4], c=0), bt.BTMV_E_ARG),
    (dict(d=1, n=[4], c=4), bt.BTMV_E_ARG),
    (dict(d=1, n=[0], c=1), bt.BTMV_E_ARG),
    (dict(d=1, n=[4], c=1, precision=7), bt.BTMV_E_ARG),
    (dict(d=1, n=[4], c=1, algo=9), bt.BTMV_E_ARG),
    (dict(d=1, n=[4], c=1, max_rhs=0), bt.BTMV_E_ARG),
    (dict(d=1, n=[4], c=1, flags=1 << 7), bt.BTMV_E_ARG),
    (dict(d=1, n=[11], c=1, algo=1), bt.BTMV_E_UNSUPPORTED),
    (dict(d=5, n=[4, 4, 4, 4, 11], c=1), bt.BTMV_E_UNSUPPORTED),
    (dict(d=2, n=[8, 2048], c=1), bt.BTMV_E_UNSUPPORTED),
    (dict(d=5, n=[4] * 5, c=1, algo=1), bt.BTMV_E_UNSUPPORTED),
])
def test_plan_create_rejects_bad_arguments(L, kw, status):
    args = dict(precision=bt.BTMV_C64, algo=bt.BTMV_ALGO_SPLIT, max_rhs=1, flags=0)
    args.update(kw)
    with pytest.raises(bt.BtmvError) as ei:
        bt.btmv_plan_create(args["d"], args["n"], args["c"], args["precision"], args["algo"],
                            args["max_rhs"], args["flags"])
    assert ei.value.status == status
    assert bt.btmv_last_error() != ""


def test_null_plan_calls_fail_cleanly(L):
    assert L.btmv_apply(None, None, None, 1, None) == bt.BTMV_E_ARG
    assert L.btmv_set_kernel(None, None, 0, None, None) == bt.BTMV_E_ARG
    assert L.btmv_destroy(None) == bt.BTMV_OK
    assert L.btmv_apply_batched(0, None, None, None, None, None) == bt.BTMV_OK
    assert L.btmv_apply_batched(-1, None, None, None, None, None) == bt.BTMV_E_ARG
    assert L.btmv_plan_get_info(None, None) == bt.BTMV_E_ARG


def _header_enums():
    """NAME = value pairs of the header's enums (integers and 1u << k)."""
    import re
    text = open(bt.HEADER).read()
    out = {}
    for name, val in re.findall(r"^\s*(BTMV_[A-Z0-9_]+)\s*=\s*([0-9u<\s]+?)\s*[,/\n]", text, re.M):
        val = val.replace("u", "").strip()
        out[name] = (1 << int(val.split("<<")[1])) if "<<" in val else int(val)
    return out


def test_binding_constants_match_header():
    """Every enum constant the Python binding defines has the header's value,
    and the profile kinds are in the header's order."""
    enums = _header_enums()
    assert enums["BTMV_FLAG_FUSED_LEVELS"] == 32 and enums["BTMV_K_NKINDS"] == len(bt.KINDS)
    checked = 0
    for name, val in enums.items():
        if hasattr(bt, name):
            assert getattr(bt, name) == val, name
            checked += 1
    assert checked >= 20
    kinds = sorted((v, k) for k, v in enums.items() if k.startswith("BTMV_K_") and k != "BTMV_K_NKINDS")
    assert [k[len("BTMV_K_"):].lower() for _, k in kinds] == bt.KINDS


def test_plan_create_accepts_every_declared_flag(L):
    """Plan flags declared in the header are accepted (the plan is created
    on the host side only when no device is present: creation fails there
    with a CUDA status, not BTMV_E_ARG)."""
    enums = _header_enums()
    flags = 0
    for name, val in enums.items():
        if name.startswith("BTMV_FLAG_"):
            flags |= val
    try:
        h = bt.btmv_plan_create(1, [4], 1, bt.BTMV_C64, bt.BTMV_ALGO_SPLIT, 1, flags)
    except bt.BtmvError as e:
        assert e.status != bt.BTMV_E_ARG, bt.btmv_last_error()
    else:
        bt.btmv_destroy(h)
