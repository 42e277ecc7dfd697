"""Host-side helpers of bench.py that feed its JSON line (no GPU).

roofline.traffic comes from a recorded ncu ratio that is valid only for the CUDA sources it was
measured on: the record names the source hash, and any source change must make the bench report
null instead of a stale figure.
"""
import json
import os

import pytest

import bench


def _tree(tmp_path, sources, record):
    csrc = tmp_path / "paper_2506_03969_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name, text in sources.items():
        (csrc / name).write_text(text)
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "dram_traffic.json").write_text(record)
    return tmp_path


def test_source_hash_is_stable_and_tracks_every_file(tmp_path, monkeypatch):
    root = _tree(tmp_path, {"a.cu": "x", "b.cuh": "y"}, "{}")
    monkeypatch.setattr(bench, "ROOT", str(root))
    h1 = bench.csrc_hash()
    assert len(h1) == 12 and all(c in "0123456789abcdef" for c in h1)
    assert bench.csrc_hash() == h1
    (root / "paper_2506_03969_gb300" / "csrc" / "b.cuh").write_text("y2")
    assert bench.csrc_hash() != h1
    (root / "paper_2506_03969_gb300" / "csrc" / "b.cuh").write_text("y")
    assert bench.csrc_hash() == h1
    os.rename(root / "paper_2506_03969_gb300" / "csrc" / "b.cuh", root / "paper_2506_03969_gb300" / "csrc" / "c.cuh")
    assert bench.csrc_hash() != h1      # file names count too


def test_recorded_traffic_only_for_the_recorded_sources(tmp_path, monkeypatch):
    root = _tree(tmp_path, {"k.cu": "kernel"}, "{}")
    monkeypatch.setattr(bench, "ROOT", str(root))
    h = bench.csrc_hash()
    (root / "profiles" / "dram_traffic.json").write_text(json.dumps({"records": [
        {"kernel": "x_node", "csrc_hash": h, "dram_over_algorithmic": 0.882},
        {"kernel": "web_bias_adj", "csrc_hash": "deadbeef0000", "dram_over_algorithmic": 0.976}]}))
    assert bench.recorded_traffic("x_node", 1000.0) == pytest.approx(882.0)
    assert bench.recorded_traffic("web_bias_adj", 1000.0) is None     # recorded on other sources
    assert bench.recorded_traffic("y_inv", 1000.0) is None            # never recorded
    (root / "paper_2506_03969_gb300" / "csrc" / "k.cu").write_text("kernel, changed")
    assert bench.recorded_traffic("x_node", 1000.0) is None           # sources changed since


def test_recorded_traffic_keyed_to_the_kernels_own_sources(tmp_path, monkeypatch):
    """A record that names its kernel's source files stays valid while only other files change."""
    root = _tree(tmp_path, {"k.cu": "kernel", "k.cuh": "header", "other.cu": "host"}, "{}")
    monkeypatch.setattr(bench, "ROOT", str(root))
    files = ["k.cu", "k.cuh"]
    (root / "profiles" / "dram_traffic.json").write_text(json.dumps({"records": [
        {"kernel": "x_node", "sources": files, "csrc_hash": bench.csrc_hash(files), "dram_over_algorithmic": 0.5}]}))
    assert bench.recorded_traffic("x_node", 10.0) == pytest.approx(5.0)
    (root / "paper_2506_03969_gb300" / "csrc" / "other.cu").write_text("host, changed")
    assert bench.recorded_traffic("x_node", 10.0) == pytest.approx(5.0)
    (root / "paper_2506_03969_gb300" / "csrc" / "k.cuh").write_text("header, changed")
    assert bench.recorded_traffic("x_node", 10.0) is None
    os.remove(root / "paper_2506_03969_gb300" / "csrc" / "k.cuh")
    assert bench.recorded_traffic("x_node", 10.0) is None


def test_recorded_traffic_without_a_record(tmp_path, monkeypatch):
    root = _tree(tmp_path, {"k.cu": "kernel"}, "{}")
    os.remove(root / "profiles" / "dram_traffic.json")
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.recorded_traffic("x_node", 1.0) is None


def test_committed_record_parses():
    """Every record of the committed file has the fields the bench reads."""
    import re
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "profiles", "dram_traffic.json")
    recs = json.load(open(path))["records"]
    assert recs
    for r in recs:
        assert re.fullmatch(r"[0-9a-f]{12}", r["csrc_hash"]) and r["kernel"]
        assert 0.5 < float(r["dram_over_algorithmic"]) < 1.5


def test_workload_config_names_the_small_case():
    """The --small-case profiling run labels its line as the 128^3 case, never as the headline."""
    head = bench.workload_config(1)
    small = bench.workload_config(1, 128)
    assert head["n"] == 256 and "256^3" in head["workload"]
    assert small["n"] == 128 and "not the headline" in small["workload"]
