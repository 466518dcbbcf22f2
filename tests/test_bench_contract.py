"""bench.py's reference arm (the float64 oracle on the host) prints one JSON line
with the keys of the benchmark contract; no GPU is needed."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--size", "32",
                        "--steps", "2", "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "PSATD cell-steps/s" and d["unit"] == "cell-steps/s"
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 0 and d["ms_per_step"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["grid"] == [32, 32, 32]


def test_all_cores_oracle_rate_runs_spawned_processes():
    sys.path.insert(0, ROOT)
    import bench
    r = bench.oracle_all_cores_rate(32, procs=2)
    assert r["cores"] == 2 and r["kind"] == "oracle" and r["unit"] == "cell-steps/s" and r["value"] > 0


def test_step_roofline_per_kernel_figures():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2010_00409_gb300 import workloads as W
    g = W.GridSpec(256, 256, 256, 1.0, 1.0, 1.0, 0.0, 0.0, 0.0, 1.0)
    # two steps: two forward + two inverse plane launches of 0.25 ms, two k-space launches of 0.2 ms
    prof = {"plane_xy": (1.0, 4), "kspace_z": (0.4, 2), "init_pulse": (4.0, 1)}
    roof, hbm = bench.step_roofline(prof, g, "real", 256, 6779.0, "measured")
    B = 48 * 256 ** 3
    assert roof["kernel"] == "plane_xy" and roof["avg_launch_ms"] == 0.25
    assert abs(roof["achieved"] - B / 0.25e-3 / 1e9) < 1e-6
    assert hbm["algorithmic_bytes_per_cell_step"] == 144.0 and abs(hbm["ms_per_psatd_step"] - 0.7) < 1e-12
    k = hbm["kernels"]
    assert set(k) == {"plane_xy", "kspace_z"}
    assert abs(k["kspace_z"]["achieved_GBps"] - B / 0.2e-3 / 1e9) < 1e-6
    assert abs(k["kspace_z"]["frac"] - k["kspace_z"]["achieved_GBps"] / 6779.0) < 1e-12
    assert k["kspace_z"]["traffic"] == bench.NCU_TRAFFIC_BYTES[("kspace_z", 256, "real")]
