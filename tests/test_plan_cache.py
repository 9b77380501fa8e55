"""The tile-plan cache of `SoapGap.autotune` against a stand-in library (no GPU).

A complete entry for the batch's problem class is installed through soapgap_set_plan
without timing; a missing, incomplete (written before a plan entry existed), rejected or
unreadable entry makes the library tune, and the new plan replaces that entry while the
other classes' entries stay.
"""
import ctypes
import json
import types

import pytest

from paper_1905_02142_gb300 import _lib as L
from paper_1905_02142_gb300.api import SoapGap

TUNED = [5, 0, 3, 1, 1]
STREAM = types.SimpleNamespace(cuda_stream=0)
BATCH = types.SimpleNamespace(c_batch=lambda: ctypes.c_int(0), pos=None)


class FakeLib:
    """soapgap_autotune writes TUNED; soapgap_set_plan records the plan and answers `accept`."""

    def __init__(self, accept=L.OK):
        self.accept = accept
        self.tuned = 0
        self.installed = []

    def soapgap_autotune(self, h, batch, plan, stream):
        self.tuned += 1
        plan = getattr(plan, "_obj", plan)  # the array, passed directly or by reference
        for i, v in enumerate(TUNED):
            plan[i] = v
        return L.OK

    def soapgap_set_plan(self, h, batch, plan):
        self.installed.append(list(getattr(plan, "_obj", plan)))
        return self.accept

    def soapgap_last_error(self, h):
        return b"stand-in"


def model_with(lib, monkeypatch, key="class-A"):
    m = object.__new__(SoapGap)
    m.lib, m.h, m.precision = lib, None, "mixed"
    monkeypatch.setattr(m, "compute", lambda *a, **k: None, raising=False)
    monkeypatch.setattr(m, "_plan_cache_key", lambda s: key, raising=False)
    return m


def as_dict(vals):
    return dict(zip(SoapGap.PLAN_KEYS, vals))


def test_plan_keys_cover_the_plan():
    assert len(SoapGap.PLAN_KEYS) == L.PLAN_LEN == len(TUNED)


def test_without_a_cache_the_library_tunes(monkeypatch):
    lib = FakeLib()
    got = model_with(lib, monkeypatch).autotune(BATCH, stream=STREAM)
    assert lib.tuned == 1 and not lib.installed
    assert got == dict(as_dict(TUNED), cached=False)


def test_first_call_tunes_and_writes_the_second_installs(tmp_path, monkeypatch):
    cache = str(tmp_path / "sub" / "plans.json")
    lib = FakeLib()
    m = model_with(lib, monkeypatch)
    assert m.autotune(BATCH, stream=STREAM, cache=cache)["cached"] is False
    assert json.load(open(cache)) == {"class-A": as_dict(TUNED)}
    got = m.autotune(BATCH, stream=STREAM, cache=cache)
    assert got == dict(as_dict(TUNED), cached=True)
    assert lib.tuned == 1 and lib.installed == [TUNED]


def test_incomplete_entry_is_tuned_again_and_replaced(tmp_path, monkeypatch):
    cache = tmp_path / "plans.json"
    old = {k: v for k, v in as_dict([2, 1, 0, 2, 0]).items() if k != "pair_forward"}
    other = as_dict([3, 0, 0, 1, 2])
    cache.write_text(json.dumps({"class-A": old, "class-B": other}))
    lib = FakeLib()
    got = model_with(lib, monkeypatch).autotune(BATCH, stream=STREAM, cache=str(cache))
    assert lib.tuned == 1 and not lib.installed and got["cached"] is False
    assert json.loads(cache.read_text()) == {"class-A": as_dict(TUNED), "class-B": other}


def test_rejected_entry_is_tuned_again(tmp_path, monkeypatch):
    cache = tmp_path / "plans.json"
    cache.write_text(json.dumps({"class-A": as_dict([9, 9, 9, 9, 9])}))
    lib = FakeLib(accept=L.E_INVALID_ARG)
    got = model_with(lib, monkeypatch).autotune(BATCH, stream=STREAM, cache=str(cache))
    assert lib.installed == [[9, 9, 9, 9, 9]] and lib.tuned == 1
    assert got == dict(as_dict(TUNED), cached=False)
    assert json.loads(cache.read_text())["class-A"] == as_dict(TUNED)


@pytest.mark.parametrize("text", ["{not json", "[1, 2]", "", '{"class-A": {"adjoint_warps": "x", '
                                  '"gap_forward": 0, "gap_backward": 0, "neighbour_sweep": 0, '
                                  '"pair_forward": null}}'])
def test_unreadable_cache_is_rewritten(tmp_path, monkeypatch, text):
    cache = tmp_path / "plans.json"
    cache.write_text(text)
    lib = FakeLib()
    got = model_with(lib, monkeypatch).autotune(BATCH, stream=STREAM, cache=str(cache))
    assert lib.tuned == 1 and got["cached"] is False
    assert json.loads(cache.read_text()) == {"class-A": as_dict(TUNED)}
