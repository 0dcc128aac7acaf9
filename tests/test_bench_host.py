"""Host logic of bench.py's roofline fields (no GPU): the `traffic` lookup in the
committed ncu summary (per tile variant, keyed by the kernel-source digest) and the
digest itself."""
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    import bench as b
    return b


def _traffic_file():
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
        return json.load(f)


def test_source_digest_is_stable_and_covers_the_kernel_sources(bench):
    d1, d2 = bench.source_digest(), bench.source_digest()
    assert d1 == d2 and len(d1) == 16 and int(d1, 16) >= 0
    for name in bench.DIGEST_SOURCES:
        assert os.path.exists(os.path.join(ROOT, "paper_1508_02363_gb300", "csrc", name)), name


def test_traffic_scales_the_captured_ratio_per_variant(bench, monkeypatch):
    d = _traffic_file()
    monkeypatch.setattr(bench, "source_digest", lambda: d["source_digest"])
    alg = 1.6e9
    entry = d["kinds"]["inner_pass_b_cols"]
    for v, ratio in entry["variants"].items():
        assert bench.ncu_traffic("inner_pass_b_cols", alg, variant=int(v)) == round(ratio * alg)
    assert bench.ncu_traffic("arnoldi_dots", alg) == round(d["kinds"]["arnoldi_dots"]["dram_over_algorithmic"] * alg)
    # every ratio is a plausible DRAM / algorithmic byte ratio
    for kind, e in d["kinds"].items():
        assert 0.5 < e["dram_over_algorithmic"] < 2.0, kind
    assert bench.ncu_traffic("no_such_kind", alg) is None


def test_traffic_is_null_once_the_kernels_changed(bench, monkeypatch):
    monkeypatch.setattr(bench, "source_digest", lambda: "0" * 16)
    assert bench.ncu_traffic("inner_pass_b_cols", 1.0e9, variant=0) is None


def test_fp64_column_roofline_counts_elements_from_the_profiled_bytes(bench):
    # 3 launches of the FP64 column pass over 10 slot-steps of an N = 64 grid: bytes =
    # 10 x 2 F64 + 3 x (M+2) F64 tables; flops per element 2 x 5 log2 N + 8 (M+1) + 12
    N, M = 64, 2
    f64 = 16.0 * N * N
    nbytes = 10 * 2 * f64 + 3 * (M + 2) * f64
    r = bench.fp64_column_roofline((2.0, 3, nbytes), N, M)
    flop = 10 * N * N * (10 * 6 + 8 * 3 + 12)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["flop_per_launch"] == pytest.approx(flop / 3)
    assert r["achieved"] == pytest.approx(flop / 2e-3 / 1e12, abs=1e-4)
    assert r["peak"] == pytest.approx(152 * 4 * 2.07e9 / 1e12, abs=1e-4)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], abs=1e-3)
