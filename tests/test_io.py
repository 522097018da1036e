"""Checkpoint files and solve logs (host side, no GPU)."""
import json

import numpy as np
import pytest

from paper_1206_5214_gb300 import io
from paper_1206_5214_gb300 import SolveInfo


def test_field_roundtrip(tmp_path):
    rng = np.random.default_rng(1)
    a = rng.standard_normal((2, 4, 2, 2, 2, 4, 4, 3)) + 1j * rng.standard_normal((2, 4, 2, 2, 2, 4, 4, 3))
    path = str(tmp_path / "x.bin")
    io.save_field(path, a, {"dims": [4, 2, 2, 2], "Ls": 4, "seed": 2001})
    b, meta = io.load_field(path)
    assert np.array_equal(a, b)
    assert meta["seed"] == 2001
    # a truncated file is refused
    with open(path, "r+b") as f:
        f.truncate(100)
    with pytest.raises(ValueError):
        io.load_field(path)


def test_solve_log(tmp_path):
    info = SolveInfo()
    info.status, info.iters, info.true_res = 0, 336, 4e-11
    path = str(tmp_path / "log.jsonl")
    io.log_solve(path, [info, info], lattice="4^4", inner="f32")
    lines = [json.loads(l) for l in open(path)]
    assert len(lines) == 2 and lines[1]["rhs"] == 1 and lines[0]["iters"] == 336
    assert lines[0]["inner"] == "f32"
