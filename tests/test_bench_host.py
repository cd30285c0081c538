"""bench.py's host logic on the CPU: the drift-velocity qualifier taken over
the oracle comparisons that resolve 0.5 %, and profile records used only for
the launch form (and kernel sources) they were captured from."""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _w(rel, rel_se, z):
    return {"rel": rel, "rel_se": rel_se, "z": z}


def test_w_qualifier_takes_the_worst_resolved_comparison():
    batched = {"per_swarm": [{"swarm": 3, "W": _w(-0.004, 0.0012, -2.1)},    # resolves 0.5 %
                             {"swarm": 9, "W": _w(0.009, 0.004, 1.5)}]}      # does not
    sweep = {"per_point": [{"E/N_Td": 10.0, "W": _w(0.012, 0.007, 1.7)},     # does not
                           {"E/N_Td": 500.0, "W": _w(0.001, 0.0015, 0.7)}]}  # resolves
    q = bench.w_qualifier(batched, sweep)
    assert q["max_rel_err_W_vs_oracle"] == 0.004
    w = q["w_vs_oracle"]
    assert w["worst_resolved"]["case"] == "batched swarm 3"
    assert (w["resolving_0.5pct"], w["comparisons"], w["within_0.5pct"]) == (2, 4, 2)
    assert w["max_abs_rel_all"] == 0.012 and w["max_abs_z_all"] == 2.1
    # a resolved comparison beyond 0.5 % is reported as it is, not hidden
    sweep["per_point"].append({"E/N_Td": 900.0, "W": _w(0.007, 0.001, 7.0)})
    q = bench.w_qualifier(batched, sweep)
    assert q["max_rel_err_W_vs_oracle"] == 0.007 and q["w_vs_oracle"]["within_0.5pct"] == 2
    # nothing resolves: no qualifier value
    q = bench.w_qualifier(None, {"per_point": [{"E/N_Td": 1.0, "W": _w(0.01, 0.01, 1.0)}]})
    assert q["max_rel_err_W_vs_oracle"] is None and q["w_vs_oracle"]["worst_resolved"] is None
    assert bench.w_qualifier(None, None) == {}


def test_profile_records_apply_to_their_own_launch_form(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1901_08140_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text("kernel v1\n")
    prof = tmp_path / "profiles"
    prof.mkdir()
    sha = hashlib.sha256(b"kernel v1\n").hexdigest()
    rec = {"sources": ["k.cu"], "sources_sha256": sha, "dram_bytes_read": 100, "dram_bytes_write": 900,
           "launch": {"block_threads": 768, "smem_budget": 204800}}
    (prof / "t.json").write_text(json.dumps(rec))
    (prof / "old.json").write_text(json.dumps({k: v for k, v in rec.items() if k != "launch"}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("t", {"block_threads": 768, "smem_budget": 204800}) == 1000
    assert bench.profiled_traffic("t", {"block_threads": 256, "smem_budget": 0}) is None
    assert bench.profiled_traffic("t", {"block_threads": 768, "smem_budget": 0}) is None
    # a record without a launch form is the library default's
    assert bench.profiled_traffic("old", {"block_threads": 256, "smem_budget": 0}) == 1000
    assert bench.profiled_traffic("old", {"block_threads": None, "smem_budget": None}) == 1000
    assert bench.profiled_traffic("old", {"block_threads": 768, "smem_budget": 204800}) is None
    # changed kernel sources void every record
    (csrc / "k.cu").write_text("kernel v2\n")
    assert bench.profiled_traffic("t", {"block_threads": 768, "smem_budget": 204800}) is None
