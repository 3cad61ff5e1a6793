"""Host-side complexity / memory models against Table 1 and Sec. IV."""
import math

import pytest

from paper_2406_17981_gb300 import analysis as A
from tests.conftest import read_golden


def test_table1_values():
    for d, rc, rm, rms in read_golden("table1.txt"):
        d = int(d)
        # printed to two decimals, halves rounded up (65/8 = 8.125 -> 8.13)
        assert abs(A.ratio_complexity_asymptotic(d) - float(rc)) <= 0.005 + 1e-12
        assert abs(A.ratio_memory(d) - float(rm)) <= 0.005 + 1e-12
        assert abs(A.ratio_memory_sym(d) - float(rms)) <= 0.005 + 1e-12


def test_outlook_d3_fractions():
    want = {r[0]: int(r[1]) / int(r[2]) for r in read_golden("outlook_d3.txt")}
    assert A.ratio_complexity_asymptotic(3) == pytest.approx(want["R_c"], rel=1e-15)
    assert A.ratio_memory(3) == pytest.approx(want["R_m"], rel=1e-15)
    assert A.ratio_memory_sym(3) == pytest.approx(want["R_m_sym"], rel=1e-15)


@pytest.mark.parametrize("d", [1, 2, 3, 4, 6])
def test_compratio_lines_agree_and_converge(d):
    # the first line of Eq. CompRatio (C_embed / C_split) equals the second
    for n in (2, 16, 1024):
        assert A.complexity_embed(d, n) / A.complexity_split(d, n) == pytest.approx(
            A.ratio_complexity(d, n), rel=1e-12)
    big = 2 ** 200
    assert A.ratio_complexity(d, big) == pytest.approx(A.ratio_complexity_asymptotic(d), rel=0.01)
    assert A.ratio_complexity_printed(d, big) == pytest.approx(A.ratio_complexity_asymptotic(d), rel=0.01)


def test_block_memory_ratio_reduces_to_paper():
    for d in range(2, 7):
        # c = 1, full symbol 2^d s on both sides: Eq. MemRatio
        assert A.ratio_memory_blocks(d, 1, 2 ** d, 2 ** d) == pytest.approx(A.ratio_memory(d))
        # c = 1, symbol stored in s elements on both sides: Eq. MemRatioSym
        assert A.ratio_memory_blocks(d, 1, 1, 1) == pytest.approx(A.ratio_memory_sym(d))


def test_split_traffic_model_d3():
    V = A.vector_bytes((8, 8, 8), 3, 1, 8)
    b = A.split_pass_bytes((8, 8, 8), 3, 1, 8, 0)
    assert b["total"] == 26 * V
    V2 = A.vector_bytes((8, 8), 1, 1, 8)
    assert A.split_pass_bytes((8, 8), 1, 1, 8, 0)["total"] == 10 * V2
    V1 = A.vector_bytes((8,), 1, 1, 8)
    assert A.split_pass_bytes((8,), 1, 1, 8, 0)["total"] == 2 * V1


def test_fused_pass_bytes_drop_the_inner_levels():
    """Fusing the last two levels of a d = 3 apply removes the dim-1 split,
    the leaf's separate reads and writes and the dim-1 merge: 26 V -> 10 V
    (plus the symbol once in both)."""
    n, c, S = (16, 64, 64), 3, 12345
    V = 16 * 64 * 64 * 3 * 8
    split = A.split_pass_bytes(n, c, 1, 8, S)
    fused = A.fused_pass_bytes(n, c, 1, 8, S)
    assert split["total"] == 26 * V + S
    assert fused["total"] == 10 * V + S
    assert fused["fwd_split"] + fused["bwd_merge"] == 6 * V
    with pytest.raises(ValueError):
        A.fused_pass_bytes((8, 8), 1, 1, 8, 0)
    # d = 4: levels 1 and 2 keep their passes (3V + 2 x 3V each way), four
    # fused nodes move 2V each: 26 V + symbol against 58 V + symbol unfused
    n4 = (4, 4, 64, 64)
    V4 = 4 * 4 * 64 * 64 * 3 * 8
    assert A.fused_pass_bytes(n4, 3, 1, 8, S)["total"] == 26 * V4 + S
    assert A.split_pass_bytes(n4, 3, 1, 8, S)["total"] == 58 * V4 + S


def test_apply_kind_bytes_one_kernel_and_split():
    """Per-kind bytes: the split kinds sum to the split total; the d = 2 apply
    as one cluster kernel moves x and y once plus the symbol."""
    n, S = (64, 64), 777
    V = 64 * 64 * 16
    one = A.apply_kind_bytes(n, 1, 1, 16, S, one_kernel=True)
    assert one["fused_levels"] == one["total"] == 2 * V + S
    sp = A.apply_kind_bytes(n, 1, 1, 16, S)
    assert sp["fwd_split"] + sp["leaf"] + sp["merge"] == sp["total"] == 10 * V + S
    with pytest.raises(ValueError):
        A.apply_kind_bytes((8, 8, 8), 1, 1, 8, 0, one_kernel=True)
