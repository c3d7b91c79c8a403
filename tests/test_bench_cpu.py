"""Host logic of bench.py on CPU: the reference arm's JSON line keeps the contract's keys, the
algorithmic-byte formula of the least-model roofline, and the lookup of recorded DRAM traffic
(valid only for the kernel sources it was taken on and, for the least-model kernel, for the row
map it was taken with)."""
import hashlib
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n-atoms", "100000",
                        "--steps", "2", "--warmup", "1", "--ref-iters", "3"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] >= 3
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_algorithmic_bytes_per_iteration():
    # row_ptr (n'+1 int32) and col (nnz int32) read once, x read and y written as bits
    assert bench.alg_bytes_per_iter(64, 100) == 4 * 65 + 4 * 100 + 2 * 8
    assert bench.alg_bytes_per_iter(65, 0) == 4 * 66 + 2 * 9


def _write_record(root, key, kernel, src_text, fields=None):
    os.makedirs(os.path.join(root, "profiles"), exist_ok=True)
    src = os.path.join(root, "k.cu")
    with open(src, "w") as f:
        f.write(src_text)
    rec = {"kernel": kernel, "sources": ["k.cu"], "bytes_per_launch": 123,
           "source_sha": hashlib.sha256(src_text.encode()).hexdigest()[:16]}
    if fields is not None:
        rec["schedule_fields"] = fields
    path = os.path.join(root, "profiles", "traffic.json")
    recs = json.load(open(path)) if os.path.exists(path) else {}
    recs[key] = rec
    json.dump(recs, open(path, "w"))


def test_traffic_lookup_follows_sources_and_row_map(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    fields = {"fixpoint_kernel": 0, "fixpoint_row_split": 1, "fixpoint_chunk_batch": 1, "fixpoint_row_map": 3}
    _write_record(str(tmp_path), "fixpoint_kernel rows3", "fixpoint_kernel", "int x;", fields)
    sched = {"fixpoint_kernel": 0, "fixpoint_blocks_per_sm": 0, "fixpoint_row_split": 0, "fixpoint_chunk_batch": 0,
             "fixpoint_row_map": 3, "stable_tile_words": 0, "stable_blocks_per_sm": 0, "stable_row_split": 0}
    assert bench.measured_traffic("fixpoint_kernel", sched) == 123  # 0 reads as 1 for split / batch
    assert bench.measured_traffic("fixpoint_kernel", dict(sched, fixpoint_row_map=1)) is None
    with open(os.path.join(str(tmp_path), "k.cu"), "w") as f:
        f.write("int y;")  # the kernel changed since the capture
    assert bench.measured_traffic("fixpoint_kernel", sched) is None
    assert bench.measured_traffic("stable_kernel") is None  # no record


def test_traffic_lookup_tells_variants_apart(tmp_path, monkeypatch):
    # the batch kernel's frontier and full-sweep instantiations share a name: a record with a
    # variant answers only a lookup of that variant, a record without one only a plain lookup
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    _write_record(str(tmp_path), "batch frontier", "batch_stable_kernel", "int z;")
    path = os.path.join(str(tmp_path), "profiles", "traffic.json")
    recs = json.load(open(path))
    recs["batch frontier"]["variant"] = "frontier"
    json.dump(recs, open(path, "w"))
    assert bench.measured_traffic("batch_stable_kernel", variant="frontier") == 123
    assert bench.measured_traffic("batch_stable_kernel", variant="full_sweep") is None
    assert bench.measured_traffic("batch_stable_kernel") is None


@pytest.mark.parametrize("key", ["fixpoint_kernel", "stable_kernel", "batch_stable_kernel", "rx_forward_kernel",
                                 "stable_frontier_kernel", "fixpoint_sliced_kernel"])
def test_committed_records_name_existing_sources(key):
    recs = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    assert any(r.get("kernel", k) == key for k, r in recs.items())
    for k, r in recs.items():
        assert r["bytes_per_launch"] == r["dram_bytes_read"] + r["dram_bytes_write"]
        for src in r["sources"]:
            assert os.path.exists(os.path.join(ROOT, src)), src


def test_profile_commands_use_existing_bench_options():
    # every bench.py option that a committed ncu summary's command line uses exists, so the
    # summaries' commands still run
    import re
    src = open(os.path.join(ROOT, "bench.py")).read()
    known = set(re.findall(r'add_argument\("(--[a-z0-9-]+)"', src))
    prof = os.path.join(ROOT, "profiles")
    used = set()
    for name in os.listdir(prof):
        if name.endswith(".md"):
            text = open(os.path.join(prof, name)).read().replace("\\\n", " ")  # join continued lines
            for cmd in re.findall(r"python bench\.py[^\n]*", text):
                used |= set(re.findall(r"(--[a-z0-9-]+)", cmd))
    assert {"--schedule", "--n-atoms", "--no-tune"} <= used  # the continued lines were read
    assert used <= known, sorted(used - known)
