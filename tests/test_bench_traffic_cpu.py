"""The benchmark's DRAM-traffic record (profiles/traffic.json) on CPU: an
entry counts only for the dominant kernel of its kind and only while that
kind's sources are the ones it was captured on; otherwise the line reports
null.  Every entry names a kind the benchmark knows."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _with_record(tmp_path, monkeypatch, record):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.json").write_text(json.dumps(record))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))


def _sources(tmp_path):
    # the hash reads the sources under ROOT: give the temporary root a copy
    src = os.path.join(ROOT, "paper_1803_04880_b300", "csrc")
    dst = tmp_path / "paper_1803_04880_b300" / "csrc"
    dst.mkdir(parents=True)
    for name in os.listdir(src):
        (dst / name).write_bytes(open(os.path.join(src, name), "rb").read())
    return dst


def test_entry_counts_for_its_kind_and_current_sources(tmp_path, monkeypatch):
    csrc = _sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench._kernel_hash(bench.KIND_SOURCES["fused"])
    _with_record(tmp_path, monkeypatch, {"w": {"recover": {"kind": "fused", "kernel_hash": h,
                                                            "dram_bytes_per_launch": 123}}})
    assert bench._traffic("w", "recover", "fused") == 123
    assert bench._traffic("w", "recover", "cipher") is None   # another kernel dominates
    assert bench._traffic("w", "protect", "fused") is None    # no entry for that direction
    assert bench._traffic("x", "recover", "fused") is None    # no entry for that workload
    # a change to one of the kind's sources retires the entry
    (csrc / "swar.cuh").write_bytes((csrc / "swar.cuh").read_bytes() + b"\n")
    assert bench._traffic("w", "recover", "fused") is None


def test_committed_record_names_known_kinds():
    t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for w, v in t.items():
        if w.startswith("_"):
            continue
        for d, e in v.items():
            assert d in ("protect", "recover")
            assert e["kind"] in bench.KIND_SOURCES
            assert e["dram_bytes_per_launch"] == e["read"] + e["write"]
