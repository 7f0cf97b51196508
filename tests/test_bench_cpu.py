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
    # an untabulated tuning has no traffic
    assert bench.env_traffic("batch", dict(group=4, max_entries=16, block_threads=128)) == (None, None)
    assert bench.env_traffic("loop", dict(group=2, max_entries=128, block_threads=256)) == (None, None)
    for (wl, g, me, bt), e in bench.ENV_TRAFFIC.items():
        got = bench.env_traffic(wl, dict(group=g, max_entries=me, block_threads=bt))
        if e["sha"] == sha:
            assert got == (e["bytes"], e["source"])
            assert os.path.exists(os.path.join(ROOT, e["source"]))
        else:
            # counters taken on other kernel sources are not reported
            assert got == (None, None)
