"""Checkpoint files and solve logs (host side).

A field is stored as its raw little-endian complex128 values in ``path`` with
a JSON sidecar ``path + ".json"`` holding the shape, the dtype and free-form
metadata (lattice, Ls, coefficients, seeds). A solve can resume from a stored
solution with ``mdwf_cgne(..., guess=True)``. Solve statistics are appended to a
JSON-lines log, one line per right-hand side.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np

__all__ = ["save_field", "load_field", "log_solve"]


def save_field(path: str, array, meta: dict | None = None) -> None:
    """Write a complex128 array (numpy, or a torch tensor on any device) and its sidecar."""
    if hasattr(array, "detach"):
        array = array.detach().cpu().numpy()
    a = np.ascontiguousarray(array, dtype=np.complex128)
    tmp = path + ".tmp"
    a.astype("<c16", copy=False).tofile(tmp)
    os.replace(tmp, path)
    side = {"shape": list(a.shape), "dtype": "complex128", "byteorder": "little", "meta": meta or {}}
    with open(path + ".json", "w") as f:
        json.dump(side, f, indent=1, sort_keys=True)


def load_field(path: str):
    """(array, meta) from a file written by save_field; the size is checked against the sidecar."""
    with open(path + ".json") as f:
        side = json.load(f)
    if side.get("dtype") != "complex128":
        raise ValueError(f"{path}: unsupported dtype {side.get('dtype')}")
    shape = tuple(int(n) for n in side["shape"])
    a = np.fromfile(path, dtype="<c16")
    if a.size != int(np.prod(shape)):
        raise ValueError(f"{path}: {a.size} values, the sidecar says {shape}")
    return a.reshape(shape).astype(np.complex128, copy=False), side.get("meta", {})


def log_solve(path: str, infos, **extra) -> None:
    """Append one JSON line per right-hand side: the SolveInfo fields, a time stamp and extra keys."""
    with open(path, "a") as f:
        for r, info in enumerate(infos):
            rec = {"time": time.time(), "rhs": r}
            rec.update(info.as_dict() if hasattr(info, "as_dict") else dict(info))
            rec.update(extra)
            f.write(json.dumps(rec, sort_keys=True) + "\n")
