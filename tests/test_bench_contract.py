"""bench.py's JSON contract on the host (no GPU): the reference arm (the
oracle on the host cores) prints one line with the contract's keys, and the
DRAM-traffic figure is reported only while the device code matches the hash
it was captured on."""
import importlib.util
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench_module():
    spec = importlib.util.spec_from_file_location("bench_contract", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 0
    assert line["config"]["workload"] and line["dtype"] == "f64"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == line["value"]
    e2e = line["e2e"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0 and e2e["value"] == line["value"]


def test_traffic_figure_follows_the_device_code_hash():
    b = _bench_module()
    sha = b._kernel_sha()
    assert len(sha) == 64 and sha == b._kernel_sha()
    for prec, (nbytes, captured) in b.TRAFFIC.items():
        assert b._traffic(prec) == (nbytes if captured == sha else None)
    saved = dict(b.TRAFFIC)
    try:
        b.TRAFFIC["fp64"] = (1.0, "0" * 64)
        assert b._traffic("fp64") is None
    finally:
        b.TRAFFIC.clear()
        b.TRAFFIC.update(saved)
