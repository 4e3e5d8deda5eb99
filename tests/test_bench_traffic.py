"""bench.py reports an ncu DRAM-traffic figure only for the kernel it was captured on: the same
sources (hashed from the files profiles/traffic.json names), the same form and the same tile
shape; anything else reports null."""
import json
import os
import shutil

import bench


def _records(d):
    """(key, record) for every record; a key may hold one record or a list (several tile shapes)."""
    for key, v in d.items():
        for rec in v if isinstance(v, list) else [v]:
            yield key, rec


def _copy_tree(tmp_path):
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    shutil.copy(os.path.join(bench.ROOT, "profiles", "traffic.json"), root / "profiles" / "traffic.json")
    shutil.copytree(os.path.join(bench.ROOT, "paper_1004_5059_gb300", "csrc"), root / "paper_1004_5059_gb300" / "csrc")
    return root


def test_recorded_traffic_for_the_captured_kernel_only():
    d = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    for key, e in _records(d):
        workload, form = key.split("/")
        if e["csrc_sha256"] != bench.csrc_hash(e["csrc_files"]):
            # the kernel changed since its counters were taken: no traffic figure
            assert bench.kernel_traffic(workload, form, e["tile"]) is None
            continue
        assert bench.kernel_traffic(workload, form, e["tile"]) == e["dram_bytes_per_launch"]
        per_step = bench.traffic_per_time_step(workload, form, e["tile"])
        assert per_step == e["dram_bytes_per_launch"] / e["time_steps_per_launch"]
        other = [t + 1 for t in e["tile"]]
        assert bench.kernel_traffic(workload, form, other) is None
    assert bench.kernel_traffic("c1", "plain", None) is None  # no capture of that form


def test_changed_source_voids_the_record(tmp_path, monkeypatch):
    root = _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    d = json.load(open(root / "profiles" / "traffic.json"))
    # as if every record had just been captured on the copied sources
    for _, rec in _records(d):
        rec["csrc_sha256"] = bench.csrc_hash(rec["csrc_files"])
    json.dump(d, open(root / "profiles" / "traffic.json", "w"))
    e = d["c1/flow"]
    assert bench.kernel_traffic("c1", "flow", e["tile"]) == e["dram_bytes_per_launch"]
    # a source the records do not name leaves them valid
    other = root / "paper_1004_5059_gb300" / "csrc" / "tvlbm_mlp.cu"
    other.write_text(other.read_text() + "\n// changed\n")
    for key, rec in _records(d):
        assert "tvlbm_mlp.cu" not in rec["csrc_files"]
        assert bench.kernel_traffic(*key.split("/"), rec["tile"]) == rec["dram_bytes_per_launch"]
    # a named one voids every record built from it
    victim = root / "paper_1004_5059_gb300" / "csrc" / "tvlbm_kernels_q4.cu"
    victim.write_text(victim.read_text() + "\n// changed\n")
    assert bench.kernel_traffic("c1", "flow", e["tile"]) is None
    assert "tvlbm_kernels_q4.cu" not in d["c2/tiled"]["csrc_files"]
    assert bench.kernel_traffic("c2", "tiled", d["c2/tiled"]["tile"]) == d["c2/tiled"]["dram_bytes_per_launch"]
