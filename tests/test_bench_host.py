"""Host logic of bench.py that needs no GPU: wave count, per-build stage scaling, roofline."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_host", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_pair_waves_count_unordered_pairs(bench):
    # one k' per wave: (k, k) plus every k' > k, i.e. nk (nk + 1) / 2 waves
    assert bench.pair_waves(216, 8, 64) == 216 * 217 // 2 == 23436
    assert bench.pair_waves(5, 2, 4) == 15
    # three k' per wave: k = 0 has k' = 1..4 in two waves, k = 1 one, k = 2 one, k = 3 one
    assert bench.pair_waves(5, 2, 12) == 5 + 2 + 1 + 1 + 1
    # brute force over small meshes
    for nk in range(1, 9):
        for nkp in range(1, 5):
            expect = sum(1 + len(range(k + 1, nk, nkp)) for k in range(nk))
            assert bench.pair_waves(nk, 3, 9 * nkp) == expect


def test_sampled_pair_stages_scale_to_a_build(bench):
    stages = {"orbitals": {"ms": 600.0, "launches": 3, "units": 3},
              "pair_a": {"ms": 10.0, "launches": 200, "units": 0},
              "pairs": {"ms": 9000.0, "launches": 3, "units": 0}}
    out = bench.stage_ms_per_build(stages, waves=1000, steps=3)
    assert out["orbitals"] == pytest.approx(200.0)        # every launch timed: per step
    assert out["pair_a"] == pytest.approx(50.0)           # 0.05 ms per sampled wave x 1000
    assert out["pairs"] == pytest.approx(3000.0)


def _stages(fields, ms):
    return {"pair_a": {"ms": 2.0, "launches": 4, "units": 256},
            "pair_b": {"ms": 3.0, "launches": 4, "units": 256},
            "pair_c": {"ms": 5.0, "launches": 4, "units": 256},
            "pairs": {"ms": ms, "launches": 1, "units": fields}}


def test_roofline_of_the_fused_mixed_round_trip(bench):
    ng = 60 ** 3
    info = {"fields_per_wave": 64, "precision": 1}
    roof = bench.roofline(_stages(1000.0, 500.0), info, 60, ng, 8, 6000.0, "measured")
    assert roof["achieved"] == pytest.approx(32.0 * ng * 1000.0 / 0.5 / 1e9)
    assert roof["frac"] == pytest.approx(roof["achieved"] / 6000.0)
    assert roof["bytes_per_launch"] == 32.0 * ng * 64
    assert roof["ms_per_launch"] == pytest.approx(500.0 * 64 / 1000.0)
    assert "pass_cd" in roof["kernel"] and "pass_d" not in roof["kernel"].replace("pass_cd", "")
    assert roof["traffic"] == bench.TRAFFIC[("round_trip", 60, 64, "mixed")]
    assert sum(roof["pass_ms_share"].values()) == pytest.approx(1.0)
    assert roof["pass_ms_share"]["pair_c"] == pytest.approx(0.5)


def test_roofline_of_unfused_waves_has_no_borrowed_traffic(bench):
    ng = 60 ** 3
    fp64 = bench.roofline(_stages(10.0, 5.0), {"fields_per_wave": 64, "precision": 0}, 60, ng,
                          8, 6000.0, "measured")
    assert "pass_c + pass_d" in fp64["kernel"] and fp64["traffic"] is None
    wide = bench.roofline(_stages(10.0, 5.0), {"fields_per_wave": 144, "precision": 1}, 60, ng,
                          12, 6000.0, "measured")
    assert "pass_c + pass_d" in wide["kernel"] and wide["traffic"] is None
    assert bench.roofline({"pairs": {"ms": 0.0, "launches": 0, "units": 0}},
                          {"fields_per_wave": 64}, 60, ng, 8, 6000.0, "measured") is None


def test_l2_note_follows_the_field_sizes(bench):
    big = bench.l2_note(216, 8, 60 ** 3)         # 216 x 8 x 216,000 x 8 B = 2.99 GB
    assert big.startswith("no flush") and "3 GB" in big
    small = bench.l2_note(1, 4, 24 ** 3)
    assert small.startswith("fields fit L2")


def test_tensor_roofline_counts_stage_flops_over_gemm_time(bench):
    fps = 3 * 2 * 128 * 192 * 32                   # one stage: three MMAs of M 128, N 192, K 32
    info = {"contraction_tc": 1, "tc_stages": 1_000_000, "tc_flops_per_stage": float(fps)}
    r = bench.tensor_roofline(info, 4.0, 1000.0, "measured", stage_ms=8.0)
    assert r["achieved"] == pytest.approx(fps * 1e6 / 4e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 1000.0)
    assert r["frac_of_stage"] == pytest.approx(r["frac"] / 2.0)   # twice the time, same flops
    assert r["useful_frac"] == pytest.approx(r["frac"] / 3.0)     # only hi.hi is the product
    assert bench.tensor_roofline(info, 4.0, 1000.0, "measured")["frac_of_stage"] is None
    assert bench.tensor_roofline(dict(info, contraction_tc=0), 4.0, 1000.0, "m") is None
    assert bench.tensor_roofline(info, 0.0, 1000.0, "m") is None


def test_alu_roofline_of_the_fp64_pair_loop(bench):
    ng = 8 ** 3
    assert bench.pair_field_flops(ng) == pytest.approx((10.0 * 9 + 24.0) * ng)
    r = bench.alu_roofline(2000.0, ng, 10.0, 1.25, "fp64")
    assert r["achieved"] == pytest.approx(bench.pair_field_flops(ng) * 2000.0 / 0.01 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 1.25) and r["bound"] == "alu"
    assert bench.alu_roofline(2000.0, ng, 10.0, 0.0, "fp64") is None


def test_sweep_slope_and_job_throughput(bench):
    xs = [1, 8, 27, 64, 125, 216]
    assert bench.loglog_slope(xs, [3.0 * x ** 2 for x in xs]) == pytest.approx(2.0)
    assert bench.loglog_slope(xs, [7.0 * x ** 0.5 for x in xs]) == pytest.approx(0.5)
    # replicas: every rank runs `steps` builds; the job's rate is the sum over ranks
    assert bench.job_throughput(4, 3, 1500.0) == pytest.approx(8.0)
    assert bench.max_over_ranks(12.5) == 12.5
