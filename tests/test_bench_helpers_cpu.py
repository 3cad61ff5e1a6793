"""bench.py helpers that run without a GPU: metric names per workload, and
the rule that a recorded ncu DRAM figure is used only while the kernel's
sources are unchanged."""
import bench
import workloads as W


def test_metric_names():
    assert bench.WORKLOAD == "d3_256_c3_green_c64"
    assert bench.metric_name(W.WORKLOADS[bench.WORKLOAD]) == \
        "block Toeplitz matvecs/s (split FFT, d=3 256^3 c=3 Green, complex64)"
    assert "128^3" in bench.metric_name(W.WORKLOADS["d3_128_c3_green_c64"])
    assert "256^3" in bench.metric_name(W.WORKLOADS["d3_256_c3_skew_c64"])
    assert "complex128" in bench.metric_name(W.WORKLOADS["d2_64_c1_random_c128"])


def test_ncu_traffic_follows_the_kernel_sources(monkeypatch):
    v = bench.ncu_traffic("leaf", "d3_128_c3_green_c64")
    assert v is None or v > 1e8                         # a figure, or none once the sources changed
    assert bench.ncu_traffic("leaf", "no_such_workload") is None
    import re
    text = open(bench.os.path.join(bench.ROOT, "profiles", "ncu_leaf_d3_128_c3_green_c64.md")).read()
    recorded = re.search(r"sources_sha256:\s*([0-9a-f]+)", text).group(1)
    monkeypatch.setattr(bench, "source_sha", lambda kind=None: recorded)
    assert bench.ncu_traffic("leaf", "d3_128_c3_green_c64") > 1e8      # matching sources: used
    monkeypatch.setattr(bench, "source_sha", lambda kind=None: "0" * 16)
    assert bench.ncu_traffic("leaf", "d3_128_c3_green_c64") is None   # changed sources: not used


def test_source_sha_depends_on_the_kind():
    assert bench.source_sha("leaf") != bench.source_sha("fwd_split")
    assert len(bench.source_sha()) == 16


def test_chunks_give_percentiles_at_the_driver_step_counts():
    for steps in (10, 20, 50, 1000):
        assert steps // bench.chunk_steps(steps) >= 10
    assert bench.chunk_steps(3) == 1
