"""bench.py on the CPU: the reference arm's JSON line (the FP64 oracle timed on
the host cores) and the rules of the pair kernel's DRAM traffic table."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "tiny", "--steps", "2", "--warmup", "1"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [x for x in out.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "unit", "dtype", "data", "scaling"):
        assert isinstance(d[k], str) and d[k]
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["config"]["workload"].startswith("tiny")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_traffic_table_rules():
    import bench
    sha = bench._kernel_sha()
    assert len(sha) == 16
    # a workload without a capture has no traffic
    assert bench.env_traffic("loop", 1.0e9) == (None, None)
    for wl, e in bench.ENV_DRAM.items():
        got = bench.env_traffic(wl, 2.0 * e["pairs"])
        if e["sha"] == sha:
            # scaled by the pairs of the timed launch
            assert got == (2.0 * e["bytes"], e["source"])
            assert os.path.exists(os.path.join(ROOT, e["source"]))
        else:
            # counters taken on other kernel sources are not reported
            assert got == (None, None)
