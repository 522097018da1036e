"""Host logic of the autotuner's JSON cache (paper_1206_5214_gb300/tuning.py).

The two library calls are replaced by recorders, so no GPU is needed: a miss runs
the tuner once and stores its answer under a key of GPU name, lattice, Ls,
precision and batch; a hit applies the stored value without tuning; keys that
differ in any part do not collide; an unreadable cache counts as empty.
"""
import json

import pytest

from paper_1206_5214_gb300 import tuning


@pytest.fixture
def calls(monkeypatch):
    log = {"autotune": [], "set": []}

    def fake_autotune(ctx, prec, nrhs):
        log["autotune"].append((ctx, prec, nrhs))
        return 8 if prec == 1 else 4

    def fake_set(ctx, prec, nrhs, sb):
        log["set"].append((ctx, prec, nrhs, sb))

    monkeypatch.setattr(tuning, "mdwf_autotune", fake_autotune)
    monkeypatch.setattr(tuning, "mdwf_set_tuning", fake_set)
    return log


def test_miss_tunes_once_then_hits(tmp_path, calls):
    path = str(tmp_path / "sub" / "tune.json")
    dims = (16, 16, 16, 32)
    assert tuning.tuned("ctx", "GB300", dims, 16, 1, 1, path) == 8
    assert calls["autotune"] == [("ctx", 1, 1)] and calls["set"] == []
    with open(path) as f:
        stored = json.load(f)
    assert stored == {"GB300|16x16x16x32|Ls16|f32|nrhs1": 8}
    assert tuning.tuned("ctx2", "GB300", dims, 16, 1, 1, path) == 8
    assert calls["autotune"] == [("ctx", 1, 1)]
    assert calls["set"] == [("ctx2", 1, 1, 8)]


def test_keys_do_not_collide(tmp_path, calls):
    path = str(tmp_path / "tune.json")
    base = ("GB300", (16, 16, 16, 32), 16, 1, 1)
    variants = [base,
                ("B200",) + base[1:],
                ("GB300", (16, 16, 32, 16)) + base[2:],
                base[:2] + (12,) + base[3:],
                base[:3] + (2,) + base[4:],
                base[:4] + (12,)]
    for v in variants:
        tuning.tuned("ctx", *v, path=path)
    assert len(calls["autotune"]) == len(variants)
    assert len(tuning.load_cache(path)) == len(variants)
    assert calls["set"] == []


def test_unreadable_cache_is_empty(tmp_path, calls):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    assert tuning.load_cache(str(path)) == {}
    assert tuning.load_cache(str(tmp_path / "missing.json")) == {}
    assert tuning.tuned("ctx", "GB300", (4, 4, 4, 4), 8, 0, 1, str(path)) == 4
    assert json.loads(path.read_text()) == {"GB300|4x4x4x4|Ls8|f64|nrhs1": 4}


def test_default_path_from_environment(monkeypatch, tmp_path):
    monkeypatch.setenv("MDWF_TUNE_CACHE", str(tmp_path / "x.json"))
    assert tuning.default_path() == str(tmp_path / "x.json")
    monkeypatch.delenv("MDWF_TUNE_CACHE")
    assert tuning.default_path().endswith("tune.json")
