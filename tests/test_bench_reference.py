"""The bench's reference arm (the FP64 oracle on the host cores) prints one
JSON line with the contract's keys; run on a small grid (no GPU needed)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n", "40",
                        "--steps", "1", "--warmup", "3"], cwd=ROOT, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "unit", "scaling", "dtype", "data"):
        assert isinstance(d[k], str) and d[k]
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert (d["n_gpus"], d["steps"], d["warmup"]) == (1, 1, 3)
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert cb["cpu"]


def test_traffic_figure_is_reported_only_for_the_measured_sources(monkeypatch):
    """The bench's per-launch DRAM traffic comes from an ncu capture of given
    kernel sources: it is reported (scaled by the point count) while the
    sources hash to the recorded digest, and null once they differ."""
    import hashlib
    sys.path.insert(0, ROOT)
    import bench
    h = hashlib.sha256()
    for rel in bench.TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    monkeypatch.setattr(bench, "TRAFFIC_DIGEST", h.hexdigest())
    for st, b in bench.TRAFFIC_B_PER_POINT.items():
        assert bench.traffic_per_launch(st, 1000) == b * 1000
    assert bench.traffic_per_launch("not_a_stencil", 1000) is None
    monkeypatch.setattr(bench, "TRAFFIC_DIGEST", "0" * 64)
    assert bench.traffic_per_launch("rhombus4_displs", 1000) is None
