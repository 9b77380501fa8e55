"""The bench line's `roofline.traffic` comes from a committed ncu record and is dropped once
the measured kernels' sources change (no GPU).

The record names the stage, the workload size it was scaled to, the adjoint kernel it was
taken on and the SHA-256 of the kernels' source files; `bench.profiled_traffic` returns its
bytes per launch only when all of them still hold.
"""
import hashlib
import json
import os
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def write_record(root, sources, **over):
    os.makedirs(os.path.join(root, "profiles"), exist_ok=True)
    h = hashlib.sha256()
    for rel, text in sources.items():
        path = os.path.join(root, rel)
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as f:
            f.write(text)
        h.update(text.encode())
    rec = {"stage": "pair_adjoint", "plan_adjoint": 5, "source_files": list(sources),
           "source_sha256": h.hexdigest(), "scaled_to": {"atoms": 1000}, "bytes_per_launch": 123.0}
    rec.update(over)
    with open(os.path.join(root, "profiles", "traffic_boxT.json"), "w") as f:
        json.dump(rec, f)


@pytest.fixture
def fake_root(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    write_record(str(tmp_path), {"k/a.cu": "kernel a\n", "k/b.cuh": "helper b\n"})
    return tmp_path


W = types.SimpleNamespace(name="boxT@1000atoms")


def test_matching_record_gives_its_bytes(fake_root):
    assert bench.profiled_traffic(W, "pair_adjoint", 1000, {"adjoint_warps": 5}) == 123.0
    assert bench.profiled_traffic(W, "pair_adjoint", 1000) == 123.0


@pytest.mark.parametrize("stage,atoms,plan", [("pair_forward", 1000, None),
                                              ("pair_adjoint", 16000, None),
                                              ("pair_adjoint", 1000, {"adjoint_warps": 3})])
def test_other_stage_size_or_kernel_gives_none(fake_root, stage, atoms, plan):
    assert bench.profiled_traffic(W, stage, atoms, plan) is None


def test_changed_source_gives_none(fake_root):
    with open(os.path.join(str(fake_root), "k", "b.cuh"), "a") as f:
        f.write("// one more line\n")
    assert bench.profiled_traffic(W, "pair_adjoint", 1000) is None


def test_missing_source_or_record_gives_none(fake_root):
    os.remove(os.path.join(str(fake_root), "k", "a.cu"))
    assert bench.profiled_traffic(W, "pair_adjoint", 1000) is None
    assert bench.profiled_traffic(types.SimpleNamespace(name="other"), "pair_adjoint", 1000) is None


def test_committed_record_names_existing_sources():
    """The committed record's kernel sources exist, and it was scaled to the full box."""
    with open(os.path.join(ROOT, "profiles", "traffic_box100k_n10l10.json")) as f:
        rec = json.load(f)
    assert rec["stage"] == "pair_adjoint" and rec["scaled_to"]["atoms"] == 100000
    for rel in rec["source_files"]:
        assert os.path.exists(os.path.join(ROOT, rel)), rel
    cap = rec["captured"]
    per = sum(v["read"] + v["write"] for v in cap["per_kernel"].values())
    assert abs(per - cap["dram_bytes_read_plus_write"]) <= 1e-6 * per
    # the full-size figure keeps four significant digits
    assert abs(rec["bytes_per_launch"] - per * rec["scaled_to"]["factor"]) <= 5e-4 * rec["bytes_per_launch"]
