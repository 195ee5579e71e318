"""The pair loop's autotuner (occri_plan_autotune) and its per-shape cache, through the C ABI."""
import numpy as np
import pytest

from workloads import small_workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

occri = pytest.importorskip("paper_2207_09028_gb300")


def _wl(nocc=4, grid=(24, 24, 24), mesh=(2, 2, 2)):
    return small_workload(mesh=mesh, grid=grid, nocc=nocc, counts=(3, 2, 1))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 2e-6)])
def test_autotuned_build_matches_default(prec, tol):
    """The configuration changes the schedule, not the result (beyond rounding)."""
    w = _wl()
    plan = occri.Plan.from_workload(w, precision=prec)
    C = torch.from_numpy(w.C).cuda()
    kc0, _, ex0 = plan.build(C, want_k=False)
    kc0 = kc0.cpu().numpy()
    t = plan.autotune(force=True)
    assert t["candidates"] > 1
    assert 1 <= t["k_per_wave"] <= w.nk and t["streams"] in (1, 2, 3)
    assert t["pass_b_div"] in (1, 2) and t["split_cd"] in (0, 1)
    assert 0 < t["us_per_field"] <= t["us_default"]
    cur = plan.tuning()
    assert cur["k_per_wave"] == t["k_per_wave"] and cur["candidates"] == -1
    kc1, _, ex1 = plan.build(C, want_k=False)
    assert np.abs(kc1.cpu().numpy() - kc0).max() <= tol * np.abs(kc0).max()
    assert abs(float(ex1.cpu()[0]) - float(ex0.cpu()[0])) <= tol * abs(float(ex0.cpu()[0]))
    plan.close()


@pytest.mark.parametrize("cfg", [dict(k_per_wave=1, streams=1, pass_b_div=2, split_cd=1),
                                 dict(k_per_wave=3, streams=2, pass_b_div=1, split_cd=0),
                                 dict(k_per_wave=2, streams=3, pass_b_div=1, split_cd=0),
                                 dict(k_per_wave=2, streams=3, pass_b_div=1, split_cd=0,
                                      wave_tables=1)])
def test_every_configuration_gives_the_same_result(cfg, monkeypatch):
    """Each knob on its own: builds under forced configurations agree with the default."""
    w = _wl(nocc=3, grid=(20, 20, 20))
    plan = occri.Plan.from_workload(w, precision="fp64")
    C = torch.from_numpy(w.C).cuda()
    kc0, _, _ = plan.build(C, want_k=False)
    kc0 = kc0.cpu().numpy()
    plan.force_tuning(**cfg)
    assert {k: plan.tuning()[k] for k in cfg} == {k: min(v, w.nk) if k == "k_per_wave" else v
                                                   for k, v in cfg.items()}
    kc1, _, _ = plan.build(C, want_k=False)
    assert np.abs(kc1.cpu().numpy() - kc0).max() <= 1e-12 * np.abs(kc0).max()
    plan.close()


def test_tuning_is_cached_per_shape():
    w = _wl(nocc=2, grid=(16, 16, 16))
    a = occri.Plan.from_workload(w, precision="mixed")
    t = a.autotune(force=True)
    assert t["candidates"] > 0
    b = occri.Plan.from_workload(w, precision="mixed")       # same shape: taken at creation
    assert b.tuning()["candidates"] == -1
    assert b.tuning()["k_per_wave"] == t["k_per_wave"]
    again = b.autotune()
    assert again["candidates"] == 0 and again["k_per_wave"] == t["k_per_wave"]
    c = occri.Plan.from_workload(w, precision="fp64")        # another precision: not cached yet
    assert c.tuning()["candidates"] in (0, -1)
    for p in (a, b, c):
        p.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
def test_plan_tables_match_wave_tables(prec, tol):
    """The plan's kernel tables (one per integer k - k', formed at creation) and the tables each
    wave forms for itself hold the same values: both builds agree, at the 60^3 grid edge of the
    benchmark and on an uneven mesh (k - k' differs per axis)."""
    w = small_workload(mesh=(3, 2, 1), grid=(60, 60, 60), nocc=3, counts=(2, 1), seed=91)
    plan = occri.Plan.from_workload(w, precision=prec)
    assert plan.tuning()["wave_tables"] == 0          # the plan holds its tables
    C = torch.from_numpy(w.C).cuda()
    kc0, _, ex0 = plan.build(C, want_k=False)
    kc0 = kc0.cpu().numpy()
    cur = plan.tuning()
    plan.force_tuning(cur["k_per_wave"], cur["streams"], cur["pass_b_div"], cur["split_cd"],
                      wave_tables=1)
    assert plan.tuning()["wave_tables"] == 1
    kc1, _, ex1 = plan.build(C, want_k=False)
    assert np.abs(kc1.cpu().numpy() - kc0).max() <= tol * np.abs(kc0).max()
    assert abs(float(ex1.cpu()[0]) - float(ex0.cpu()[0])) <= tol * abs(float(ex0.cpu()[0]))
    plan.close()
