"""bench.py's reference arm on the CPU: it runs only the oracle, so its JSON line is checked here against the
contract (keys, units, the oracle as cpu_baseline, an e2e with no host-device bytes) and against our arm's
description of the same workload."""

import json
import subprocess
import sys

import bench
import workloads

KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
        "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"}


def test_reference_line_follows_the_contract():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "heat1d", "--steps", "2",
                          "--warmup", "3"], cwd=bench.ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert KEYS <= set(line)
    assert line["impl"] == "reference" and line["unit"] == "DoF/s" and line["higher_is_better"] is True
    assert line["n_gpus"] == 1 and line["steps"] == 2 and line["warmup"] == 3 and line["data"] == "synthetic"
    assert line["metric"] == bench.METRIC and line["vs_baseline"] is None
    wl = dict(workloads.WORKLOADS["heat1d"], name="heat1d")
    assert line["config"]["workload"] == bench.workload_desc("heat1d", wl)
    assert line["config"]["n_h"] == 63 and line["config"]["n_t"] == 64
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "DoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["value"] > 0 and line["ms_per_step"] > 0
    assert abs(line["value"] - 63 * 64 / (line["ms_per_step"] * 1e-3)) <= 1e-6 * line["value"]


def test_workload_descriptions_name_the_workload():
    for name, wl in workloads.WORKLOADS.items():
        d = bench.workload_desc(name, dict(wl, name=name))
        assert d.split(":")[0] == (wl.get("kind") or name)
    served = dict(workloads.WORKLOADS["served"], name="served")

    class Args:
        requests, gap_scale = 50, 2.0
    d = bench.workload_desc("served", served, Args())
    assert "50 requests (first 5 warm-up)" in d and f"{2e3 * served['mean_gap_s']:.2f} ms" in d
