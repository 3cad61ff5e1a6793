"""The host-core study of Sec. III (split vs full embedding wall-clock on the
CPU): both of its matvec implementations must reproduce the oracle's
definition of y = T x before their times mean anything."""
import numpy as np
import pytest

import workloads as W
from oracle import toeplitz as OT
from paper_2406_17981_gb300 import cpu_study as CS


@pytest.mark.parametrize("n", [(16,), (5,), (8, 4), (6, 7), (4, 4, 4), (3, 5, 2), (4, 2, 4, 2)])
def test_split_and_embed_match_the_direct_sum(n):
    t = W.random_generator(n, 1, seed=61)[0, 0]
    x = W.random_vector(n, 1, seed=62)[0, 0]
    ref = OT.direct_matvec(t[None, None], x[None])[0]
    S = CS.embedded_symbol(t, workers=1)
    ys = CS.split_apply(CS.leaf_parts(S), CS.phases(n), x, workers=1)
    ye = CS.embed_apply(S, x, workers=1)
    assert np.linalg.norm(ys - ref) / np.linalg.norm(ref) < 1e-12
    assert np.linalg.norm(ye - ref) / np.linalg.norm(ref) < 1e-12


def test_study_rows():
    rows = CS.study(sizes={1: [64], 2: [8]}, repeats=1, workers=1)
    assert [(r["d"], r["n"]) for r in rows] == [(1, 64), (2, 8)]
    assert all(r["split_s"] > 0 and r["embed_s"] > 0 for r in rows)
