"""The reference arm of bench.py (the oracle timed on the host) runs without a GPU
and prints the one JSON line of the benchmark contract, on the GPU arm's workload."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "e2e",
              "cpu_baseline"):
        assert k in line, k
    assert line["impl"] == "reference" and line["unit"] == "queries/s"
    assert line["higher_is_better"] is True and line["value"] > 0
    assert line["config"]["queries_per_frame"] == (1 << 20) + 2 * 10000
    assert line["config"]["faces"] == 200000 and line["config"]["gaussians"] == 600000
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert cb["host"]["nproc"] >= 1 and cb["host"]["cpu_model"]
    assert line["e2e"] == {"value": line["value"], "unit": "queries/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_traffic_record_is_used_only_for_the_captured_sources():
    """The roofline's DRAM / L2 traffic comes from a committed ncu capture; bench.py uses
    it only while the contact kernel's sources hash as they did when it was captured,
    and only for the captured traversal variant."""
    import hashlib
    sys.path.insert(0, ROOT)
    import bench
    p = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    d = json.load(open(p))
    m = hashlib.sha256()
    for f in d["source_files"]:
        m.update(open(os.path.join(ROOT, f), "rb").read())
    current = m.hexdigest()[:16] == d["source_hash"]
    for key, rec in d["by_config"].items():
        got = bench.contact_traffic(key)
        assert got == (rec if current else None)
    assert bench.contact_traffic("L9/v99/b7") is None
    assert bench.traversal_label({"leaf": 2, "lanes": 1, "variant": 3, "block": 64}) == "L2/v3/b64"
    # a counted visit reads a 64-byte node record, or a 128-byte 4-wide record (variant 13)
    assert bench.node_bytes({"lanes": 1, "variant": 13}) == 128
    assert bench.node_bytes({"lanes": 1, "variant": 2}) == 64
    assert bench.node_bytes({"lanes": 4, "variant": 13}) == 64
