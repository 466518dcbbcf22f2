"""JSON-lines metrics records: one line per bench run or parity check, with the
configuration, precision, throughput, bandwidth, roofline fraction, error and
the host the number came from.

`append(path, record)` adds one line; `bench_record(line)` condenses the bench's
JSON line; `parity_record(...)` describes one comparison against the CPU oracle
(written by the tests, which are the only callers of the oracle).
"""
from __future__ import annotations

import json
import os
import platform
import time

ENV = "PSATD_METRICS_LOG"


def host_info() -> dict:
    return {"host": platform.node(), "machine": platform.machine(), "host_cores": os.cpu_count()}


def append(path: str, record: dict) -> None:
    """Append one JSON object as a line (created if missing)."""
    rec = dict(record)
    rec.setdefault("time", time.strftime("%Y-%m-%dT%H:%M:%S"))
    rec.setdefault("host_info", host_info())
    line = json.dumps(rec, sort_keys=True)
    with open(path, "a") as fh:
        fh.write(line + "\n")


def bench_record(line: dict) -> dict:
    """The bench's fields that a run log keeps: workload, precision, cell-steps/s,
    achieved bandwidth and roofline fraction of the dominant kernel and of the
    whole step, errors the run measured, and the CPU baseline's cores."""
    roof = line.get("roofline") or {}
    hbm = line.get("step_hbm") or {}
    forms = line.get("focal_forms") or {}
    cpu = line.get("cpu_baseline") or {}
    errs = {}
    for k, v in forms.items():
        if isinstance(v, dict) and "rel_l2_err_vs_fp64" in v:
            errs["focal_forms.%s" % k] = v["rel_l2_err_vs_fp64"]
    for key in ("batched_sweep", "batched_stepped"):
        obj = line.get(key) or {}
        for k, v in obj.items():
            if k.startswith("max_rel_l2_err"):
                errs["%s.%s" % (key, k)] = v
    return {
        "kind": "bench",
        "metric": line.get("metric"), "config": line.get("config"), "dtype": line.get("dtype"),
        "n_gpus": line.get("n_gpus"), "value": line.get("value"), "unit": line.get("unit"),
        "ms_per_step": line.get("ms_per_step"),
        "dominant_kernel": {k: roof.get(k) for k in ("kernel", "achieved", "unit", "peak", "frac", "traffic")},
        "step_gbs": hbm.get("achieved_GBps"), "step_frac": hbm.get("frac_of_measured_peak"),
        "errors": errs, "cpu_baseline_cores": cpu.get("cores"), "clocks": line.get("clocks"),
    }


def parity_record(case: str, precision: int, rel_l2: float, tol: float, **extra) -> dict:
    rec = {"kind": "parity", "case": case, "precision": precision, "rel_l2_vs_oracle": rel_l2, "tol": tol,
           "ok": bool(rel_l2 <= tol)}
    rec.update(extra)
    return rec
