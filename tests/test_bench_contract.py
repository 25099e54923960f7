"""The benchmark's reference arm (the FP64 oracle on the host cores) and its
JSON line, run on the CPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "grid32", "--steps", "2", "--warmup", "1"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e", "impl"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "grid32"


def test_clock_summary_parses_nvidia_smi_lines():
    sys.path.insert(0, ROOT)
    import bench
    c = bench.ClockSampler(0)
    c.lines = ["2070, 2070, Not Active, Not Active, Not Active, Not Active",
               "1980, 2070, Not Active, Not Active, Not Active, Active",
               "2070, 2070, Not Active, Not Active, Not Active, Not Active",
               "[N/A], 2070, Not Active, Not Active, Not Active, Not Active",
               "garbage"]
    s = c.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                 "samples": 3}
    c.lines = []
    assert c.summary()["samples"] == 0


def test_roofline_of_the_dominant_kernel():
    sys.path.insert(0, ROOT)
    import bench
    names = ["bbox", "morton_hist", "sort", "radix_tree_scan", "records", "traverse", "gather",
             "controller"]
    ms = [0.008, 0.008, 0.046, 0.018, 0.012, 0.110, 0.021, 0.008]
    prof = {"stage_names": names, "stage_ms": ms, "nnz_S": 2_000_000, "interactions": 4.0e7}
    peaks = {"hbm_gbs": 6784.5, "sm_max_mhz": 2070.0}
    fp32 = (72.5, "measured")
    r = bench.roofline(prof, peaks, "measured", {}, 100_000, workload="rgg100k", fp32=fp32)
    assert r["kernel"] == "traverse" and r["bound"] == "alu"
    assert abs(r["achieved"] - 10 * 4.0e7 / 110e-6 / 1e12) < 1e-9
    assert r["peak"] == 72.5 and r["peak_source"] == "measured"
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert r["traffic"] is None   # no capture of the current kernel stored
    g = r["others"]["gather"]
    assert g["bound"] == "hbm" and abs(g["achieved"] - (100_000 * 32 + 2_000_000 * 8) / 21e-6 / 1e9) < 1e-6
    # an exact-repulsion level counts n (n - 1) pair interactions
    r2 = bench.roofline(prof, peaks, "measured", {}, 1024, exact=True, fp32=fp32)
    assert abs(r2["achieved"] - 10 * 1024 * 1023 / 110e-6 / 1e12) < 1e-9


def test_stored_traffic_is_dropped_once_its_kernel_source_changes(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    rel = "paper_1506_04383_gb300/csrc/k_tree.cu"
    monkeypatch.setitem(bench.NCU_TRAFFIC, ("w", "traverse"), (123.0, rel, bench._src_sha(rel)))
    assert bench.ncu_traffic("w", "traverse") == 123.0
    monkeypatch.setitem(bench.NCU_TRAFFIC, ("w", "traverse"), (123.0, rel, "0" * 16))
    assert bench.ncu_traffic("w", "traverse") is None
    assert bench.ncu_traffic("other", "traverse") is None
