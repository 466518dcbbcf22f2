"""The JSON-lines metrics records (CPU)."""
import json

from paper_2010_00409_gb300 import metrics


def test_bench_record_keeps_config_rate_bandwidth_roofline_errors_cores(tmp_path):
    line = {"metric": "PSATD cell-steps/s", "value": 2.5e10, "unit": "cell-steps/s", "n_gpus": 1,
            "ms_per_step": 250.0, "dtype": "f32", "config": {"workload": "tight focus 256^3"},
            "roofline": {"kernel": "plane_xy", "achieved": 3400.0, "unit": "GB/s", "peak": 6693.8,
                         "frac": 0.508, "traffic": 7.5e8, "bound": "hbm"},
            "step_hbm": {"achieved_GBps": 3660.0, "frac_of_measured_peak": 0.547},
            "focal_forms": {"stepped_fp32": {"rel_l2_err_vs_fp64": 3.6e-5}},
            "batched_stepped": {"max_rel_l2_err_fp32_stepped_vs_fp64_exact": 2.5e-5},
            "cpu_baseline": {"cores": 1}, "clocks": {"sm_mhz": 2070}}
    rec = metrics.bench_record(line)
    assert rec["config"] == line["config"] and rec["dtype"] == "f32" and rec["value"] == 2.5e10
    assert rec["dominant_kernel"]["frac"] == 0.508 and rec["step_gbs"] == 3660.0 and rec["step_frac"] == 0.547
    assert rec["errors"] == {"focal_forms.stepped_fp32": 3.6e-5,
                             "batched_stepped.max_rel_l2_err_fp32_stepped_vs_fp64_exact": 2.5e-5}
    assert rec["cpu_baseline_cores"] == 1
    path = tmp_path / "m.jsonl"
    metrics.append(str(path), rec)
    metrics.append(str(path), metrics.parity_record("case", 32, 2e-6, 1e-5))
    rows = [json.loads(x) for x in path.read_text().splitlines()]
    assert len(rows) == 2 and rows[0]["kind"] == "bench" and rows[1]["ok"] is True
    assert rows[0]["host_info"]["host_cores"] >= 1 and "time" in rows[1]
