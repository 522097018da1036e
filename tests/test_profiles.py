"""The committed profile summaries stay reproducible: each gives the command that
made it, the bench.py arguments in it are ones bench.py accepts, every ncu call
in it leaves the clocks alone (--clock-control none), and profiles/ holds short
text only."""
import glob
import os
import re
import shlex
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SUMMARIES = sorted(glob.glob(os.path.join(ROOT, "profiles", "*")))


def _commands(text):
    """Indented command blocks, with backslash continuations joined."""
    cmds, cur = [], ""
    for line in text.splitlines():
        if line.startswith("    ") and line.strip():
            part = line.strip()
            cur = (cur + " " + part[:-1].strip()) if part.endswith("\\") else (cur + " " + part)
            if not part.endswith("\\"):
                cmds.append(cur.strip())
                cur = ""
    return cmds


def test_profiles_are_short_text():
    assert SUMMARIES, "profiles/ is empty"
    for path in SUMMARIES:
        assert path.endswith((".md", ".txt")), path
        assert os.path.getsize(path) < 32 * 1024, path


@pytest.mark.parametrize("path", SUMMARIES, ids=[os.path.basename(p) for p in SUMMARIES])
def test_summary_commands(path, monkeypatch):
    sys.path.insert(0, ROOT)
    try:
        import bench
    finally:
        sys.path.remove(ROOT)
    text = open(path).read()
    cmds = _commands(text)
    assert any("bench.py" in c for c in cmds), f"{path}: no bench.py command"
    for cmd in cmds:
        for seg in re.split(r"&&|;", cmd):
            words = shlex.split(seg)
            if "ncu" in words:
                assert "--clock-control" in words and words[words.index("--clock-control") + 1] == "none", seg
            if "bench.py" in words:
                args = words[words.index("bench.py") + 1:]
                if ">" in args:
                    args = args[:args.index(">")]
                monkeypatch.setattr(sys, "argv", ["bench.py"] + args)
                bench.parse()


def test_traffic_record_is_keyed_by_the_kernel_sources(tmp_path):
    """A recorded DRAM traffic figure is reported only while the hop kernels'
    sources hash to the value recorded with the capture."""
    sys.path.insert(0, ROOT)
    try:
        import bench
    finally:
        sys.path.remove(ROOT)
    src = tmp_path / "k.cuh"
    src.write_text("kernel A")
    sha_a = bench.kernel_sources_sha256(files=("k.cuh",), root=str(tmp_path))
    assert re.fullmatch(r"[0-9a-f]{64}", sha_a)
    rec = tmp_path / "t.txt"
    rec.write_text('x\n```json\n{"kernels": {"hop_xpay_f32": {"dram_read_bytes": 3e8, "dram_write_bytes": 1e8, '
                   f'"sources_sha256": "{sha_a}"}}}}}}\n```\n')
    assert bench.recorded_traffic("hop_xpay_f32", str(rec), sha_a)[0] == 4e8
    src.write_text("kernel B")
    sha_b = bench.kernel_sources_sha256(files=("k.cuh",), root=str(tmp_path))
    got, note = bench.recorded_traffic("hop_xpay_f32", str(rec), sha_b)
    assert got is None and "stale" in note
    assert bench.recorded_traffic("hop_f32", str(rec), sha_a)[0] is None
    # the committed record, when there is one, names its fields
    if os.path.exists(bench.TRAFFIC_FILE):
        text = open(bench.TRAFFIC_FILE).read()
        import json
        kernels = json.loads(text.split("```json", 1)[1].split("```", 1)[0])["kernels"]
        for k, v in kernels.items():
            assert {"dram_read_bytes", "dram_write_bytes", "sources_sha256", "template"} <= set(v), k
