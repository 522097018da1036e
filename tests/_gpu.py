"""Helpers for the GPU parity tests: run the library through its C ABI on
torch device memory and bring results back as numpy arrays."""
from __future__ import annotations

import numpy as np
import torch

import paper_1206_5214_gb300 as mdwf

PREC_NAME = {mdwf.MDWF_F64: "f64", mdwf.MDWF_F32: "f32", mdwf.MDWF_F16N: "f16n"}


class Ctx:
    def __init__(self, dims, Ls, M5, b5, c5, mf, U: np.ndarray, dense_s: bool = False):
        self.dims, self.Ls = tuple(dims), Ls
        x, y, z, t = dims
        self.Vh = x * y * z * t // 2
        self.h = mdwf.mdwf_create(dims, Ls, M5, b5, c5, mf, dense_s=dense_s)
        Ud = torch.from_numpy(np.ascontiguousarray(U)).cuda()
        mdwf.mdwf_load_gauge(self.h, Ud)
        torch.cuda.synchronize()

    def close(self):
        if self.h:
            mdwf.mdwf_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def alloc(self, prec, nrhs=1):
        nbytes = mdwf.mdwf_field_bytes(self.h, prec, nrhs)
        return torch.empty(nbytes, dtype=torch.uint8, device="cuda")

    def upload(self, odd: np.ndarray, prec, nrhs=1):
        """odd: (nrhs, Ls, Vh, 4, 3) or (Ls, Vh, 4, 3) complex128 -> internal field."""
        buf = self.alloc(prec, nrhs)
        src = torch.from_numpy(np.ascontiguousarray(odd, dtype=np.complex128)).cuda()
        mdwf.mdwf_field_import(self.h, buf, src, prec, nrhs)
        return buf

    def download(self, buf, prec, nrhs=1) -> np.ndarray:
        out = torch.empty((nrhs, self.Ls, self.Vh, 4, 3), dtype=torch.complex128, device="cuda")
        mdwf.mdwf_field_export(self.h, out, buf, prec, nrhs)
        torch.cuda.synchronize()
        return out.cpu().numpy()

    def apply(self, odd: np.ndarray, prec, dagger=False, nrhs=1, masses=None) -> np.ndarray:
        inp = self.upload(odd, prec, nrhs)
        out = self.alloc(prec, nrhs)
        f = mdwf.mdwf_apply_dag if dagger else mdwf.mdwf_apply
        f(self.h, out, inp, prec, nrhs, masses)
        torch.cuda.synchronize()
        return self.download(out, prec, nrhs)


def rel_err(a: np.ndarray, b: np.ndarray) -> tuple[float, float]:
    """(max elementwise |a-b| / max|b|, |a-b|_2 / |b|_2)."""
    d = np.abs(a - b)
    return float(d.max() / np.abs(b).max()), float(np.linalg.norm(a - b) / np.linalg.norm(b))
