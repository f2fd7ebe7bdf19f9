"""Host logic of bench.py (no GPU): the committed DRAM-traffic records are
scaled to a launch while the kernel's sources are as captured, and give
null as soon as any of them changes."""
import json
import os

import bench


def _record(root, sources, per_unit):
    os.makedirs(os.path.join(root, "profiles"), exist_ok=True)
    rec = {"k": {"dram_bytes_per_unit": per_unit, "sources": sources,
                 "source_hash": bench.kernel_source_hash(sources)}}
    with open(os.path.join(root, "profiles", "traffic.json"), "w") as f:
        json.dump(rec, f)


def test_recorded_traffic_scales_and_expires(tmp_path, monkeypatch):
    root = str(tmp_path)
    monkeypatch.setattr(bench, "ROOT", root)
    for name, text in (("a.cu", "kernel a"), ("b.cuh", "header b")):
        (tmp_path / name).write_text(text)
    _record(root, ["a.cu", "b.cuh"], 30.5)
    assert bench.recorded_traffic("k", 200) == 30.5 * 200
    assert bench.recorded_traffic("missing", 200) is None
    # the hash covers every listed source, in order
    assert bench.kernel_source_hash(["a.cu", "b.cuh"]) != bench.kernel_source_hash(["b.cuh", "a.cu"])
    (tmp_path / "b.cuh").write_text("header b, edited")
    assert bench.recorded_traffic("k", 200) is None


def test_committed_records_name_existing_sources():
    d = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    for kernel in ("pipeline", "part_scatter"):
        r = d[kernel]
        assert r["dram_bytes_per_unit"] > 0 and r["unit"]
        for f in r["sources"]:
            assert os.path.exists(os.path.join(bench.ROOT, f)), f
        assert os.path.exists(os.path.join(bench.ROOT, r["summary"]))
