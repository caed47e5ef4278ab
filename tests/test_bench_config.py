"""Host logic of the benchmark (no GPU): both arms describe the workload with
the same `config`, and the reference arm finds the case-sweeps recorded for
the default workload at its current tolerance (so its extrapolation to a
whole solve uses this build's iteration count, not a stale one)."""
import bench


def test_both_arms_share_the_config():
    c = bench.config_of("porous191", 1)
    assert c["workload"] == "porous191" and c["tol"] == bench.WORKLOADS["porous191"]["tol"]
    assert c["voxels"] == 191 ** 3 and c["load_cases"] == 6 and "L2" in c["l2"]


def test_reference_arm_has_a_recorded_case_sweep_count():
    w = bench.WORKLOADS["porous191"]
    rec = bench.recorded_case_sweeps("porous191", w["tol"])
    assert rec is not None and rec["case_sweeps"] > 0
    assert abs(rec["St"] - w["St"]) <= 1e-9 * w["St"], "record taken with another Strouhal number"
    assert bench.recorded_case_sweeps("porous191", 0.5 * w["tol"]) is None
