"""The DRAM traffic bench.py reports beside a roofline comes from a committed ncu record
(profiles/traffic.json) and applies only while the kernel sources hash as they did at the
capture and the launch shape matches: lane layout, tile count, index source and form must
be equal; another row-range count keeps the figure and says so."""
import json
import os
import shutil

import bench

def _record():
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        return json.load(f)


def _shape(kind):
    return dict(_record()["chung_lu_n1e6_k100"][kind]["shape"])


def test_committed_records_match_the_sources():
    for kind in ("cheb_step", "cg_lap"):
        traffic, note = bench.recorded_traffic("chung_lu_n1e6_k100", kind, _shape(kind))
        assert traffic is not None and traffic > 0, note


def test_other_row_range_count_keeps_the_figure_with_a_note():
    sh = _shape("cg_lap")
    exact, _ = bench.recorded_traffic("chung_lu_n1e6_k100", "cg_lap", sh)
    sh["P"] += 1
    traffic, note = bench.recorded_traffic("chung_lu_n1e6_k100", "cg_lap", sh)
    assert traffic == exact and f"this run tuned {sh['P']}" in note


def test_other_lane_layout_or_workload_has_no_figure():
    sh = _shape("cg_lap")
    sh["G"] = 16 if sh["G"] != 16 else 8
    assert bench.recorded_traffic("chung_lu_n1e6_k100", "cg_lap", sh)[0] is None
    assert bench.recorded_traffic("sbm_n1e5_k200", "cg_lap", _shape("cg_lap"))[0] is None


def test_changed_source_has_no_figure(tmp_path, monkeypatch):
    rec = _record()["chung_lu_n1e6_k100"]["cg_lap"]
    os.makedirs(tmp_path / "profiles")
    shutil.copy(os.path.join(bench.ROOT, "profiles", "traffic.json"), tmp_path / "profiles" / "traffic.json")
    for src in rec["sources"]:
        dst = tmp_path / src
        os.makedirs(dst.parent, exist_ok=True)
        shutil.copy(os.path.join(bench.ROOT, src), dst)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("chung_lu_n1e6_k100", "cg_lap", _shape_at(tmp_path))[0] is not None
    with open(tmp_path / rec["sources"][0], "a") as f:
        f.write("\n// edited\n")
    traffic, note = bench.recorded_traffic("chung_lu_n1e6_k100", "cg_lap", _shape_at(tmp_path))
    assert traffic is None and "changed" in note


def _shape_at(root):
    with open(root / "profiles" / "traffic.json") as f:
        return dict(json.load(f)["chung_lu_n1e6_k100"]["cg_lap"]["shape"])
