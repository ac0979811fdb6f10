"""bench.py reports the roofline's DRAM traffic only for the conv sources it was captured on:
any change to them (or a missing file) turns the figure into null."""
import hashlib
import os
import shutil

import bench


def _tree(tmp_path):
    for rel in bench.CONV_TRAFFIC["sha256"]:
        dst = tmp_path / rel
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copyfile(os.path.join(bench.ROOT, rel), dst)


def test_traffic_follows_the_captured_sources(tmp_path, monkeypatch):
    _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    match = all(hashlib.sha256((tmp_path / rel).read_bytes()).hexdigest() == d
                for rel, d in bench.CONV_TRAFFIC["sha256"].items())
    assert bench.conv_traffic() == (bench.CONV_TRAFFIC["bytes_per_step"] if match else None)


def test_changed_or_missing_source_gives_null(tmp_path, monkeypatch):
    _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    rel = next(iter(bench.CONV_TRAFFIC["sha256"]))
    with open(tmp_path / rel, "ab") as f:
        f.write(b"\n// changed\n")
    assert bench.conv_traffic() is None
    os.remove(tmp_path / rel)
    assert bench.conv_traffic() is None
