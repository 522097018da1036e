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
