"""FP64 CPU oracle for the Moebius domain-wall operator (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package. The
library in ``paper_1206_5214_gb300`` never imports it, and the two share no
code: this is a plain statement of what the paper defines (Eq. D^Wilson,
Eq. MoebiusOp, the red/black Schur complement and the closed-form I_rr^-1 of
Sec. 3), written in C (``mdwf_oracle.c``) and called through ctypes.

Array conventions (numpy complex128, C order):

* gauge ``U``: ``(T, Z, Y, X, 4, 3, 3)``
* full 5d field: ``(Ls, T, Z, Y, X, 4, 3)``
* half (one-parity) 5d field: ``(Ls, V/2, 4, 3)``, sites of that parity in
  lexicographic (x fastest) order.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mdwf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libmdwf_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over sites) into ``oracle/_build``."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fcx-limited-range", "-fopenmp", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int * 4), ("Ls", ctypes.c_int), ("M5", ctypes.c_double),
                ("b5", ctypes.c_double), ("c5", ctypes.c_double), ("mf", ctypes.c_double),
                ("b5s", ctypes.POINTER(ctypes.c_double)), ("c5s", ctypes.POINTER(ctypes.c_double)),
                ("mu", ctypes.c_double)]


@dataclass(frozen=True)
class Params:
    """Physics parameters: dims = (X, Y, Z, T), Ls, wall height M5 (> 0), b5, c5, mf.

    ``b5s`` / ``c5s`` (tuples of Ls values, or None) replace the constant b5 / c5
    by per-slice coefficients b5(s), c5(s): row s of Eq. (MoebiusOp) then uses
    D+ = b5(s) D_W + 1 and D- = c5(s) D_W - 1. ``mu`` is a chemical potential
    on the time links (Sec. 6.6).
    """
    dims: tuple
    Ls: int
    M5: float
    b5: float
    c5: float
    mf: float
    b5s: tuple | None = None
    c5s: tuple | None = None
    mu: float = 0.0

    def c(self) -> _Params:
        p = _Params()
        for k in range(4):
            p.L[k] = int(self.dims[k])
        p.Ls, p.M5, p.b5, p.c5, p.mf = int(self.Ls), float(self.M5), float(self.b5), float(self.c5), float(self.mf)
        p.mu = float(self.mu)
        keep = []
        for name in ("b5s", "c5s"):
            vals = getattr(self, name)
            if vals is not None:
                if len(vals) != self.Ls or self.Ls > 64:
                    raise ValueError(f"{name} needs Ls <= 64 values")
                arr = (ctypes.c_double * self.Ls)(*[float(v) for v in vals])
                keep.append(arr)
                setattr(p, name, ctypes.cast(arr, ctypes.POINTER(ctypes.c_double)))
        p._keep = keep   # the arrays live as long as the struct
        return p

    def with_(self, **kw) -> "Params":
        d = dict(dims=self.dims, Ls=self.Ls, M5=self.M5, b5=self.b5, c5=self.c5, mf=self.mf,
                 b5s=self.b5s, c5s=self.c5s, mu=self.mu)
        d.update(kw)
        return Params(**d)

    @property
    def s_dependent(self) -> bool:
        return self.b5s is not None or self.c5s is not None

    @property
    def V(self) -> int:
        x, y, z, t = self.dims
        return int(x * y * z * t)


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER(_Params)
        vp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)
        dp = ctypes.POINTER(ctypes.c_double)
        sig = {
            "or_gammas": (None, [vp]),
            "or_dw": (None, [vp, vp, vp, ctypes.POINTER(ctypes.c_int), ctypes.c_double, ctypes.c_double,
                             ctypes.c_int]),
            "or_ddw": (None, [vp, vp, vp, P, ctypes.c_int]),
            "or_mee": (None, [vp, vp, P, ctypes.c_int]),
            "or_dhop": (None, [vp, vp, vp, P, ctypes.c_int, ctypes.c_int]),
            "or_mee_inv": (None, [vp, vp, ctypes.c_long, P, ctypes.c_int]),
            "or_m": (None, [vp, vp, vp, P, ctypes.c_int]),
            "or_mdagm": (None, [vp, vp, vp, P]),
            "or_cgne": (ctypes.c_int, [vp, vp, vp, P, ctypes.c_double, ctypes.c_int, ip, dp]),
            "or_prepare": (None, [vp, vp, vp, P]),
            "or_reconstruct": (None, [vp, vp, vp, vp, P]),
            "or_solve": (ctypes.c_int, [vp, vp, vp, P, ctypes.c_double, ctypes.c_int, ip, dp]),
            "or_solve_dag": (ctypes.c_int, [vp, vp, vp, P, ctypes.c_double, ctypes.c_int, ip, dp]),
            "or_dm_dparam": (None, [vp, vp, vp, P, ctypes.c_int]),
            "or_force": (ctypes.c_int, [vp, dp, dp, dp, vp, vp, P, ctypes.c_double, ctypes.c_int, ip]),
            "or_set_threads": (None, [ctypes.c_int]),
            "or_get_threads": (ctypes.c_int, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _c(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def set_threads(n: int) -> None:
    _load().or_set_threads(int(n))


def get_threads() -> int:
    return int(_load().or_get_threads())


def gammas() -> tuple[np.ndarray, np.ndarray]:
    """The oracle's (g_1..g_4 as (4, 4, 4), g5 as (4, 4))."""
    out = np.zeros(80, dtype=np.complex128)
    _load().or_gammas(_ptr(out))
    return out[:64].reshape(4, 4, 4), out[64:].reshape(4, 4)


def dw(psi4: np.ndarray, U: np.ndarray, dims, M5: float, dagger: bool = False, mu: float = 0.0) -> np.ndarray:
    """D_W (Eq. D^Wilson, diagonal 4 - M5) on a 4d field of shape (T, Z, Y, X, 4, 3)."""
    psi4, U = _c(psi4), _c(U)
    out = np.empty_like(psi4)
    L = (ctypes.c_int * 4)(*[int(d) for d in dims])
    _load().or_dw(_ptr(out), _ptr(psi4), _ptr(U), L, float(M5), float(mu), int(dagger))
    return out


def ddw(psi: np.ndarray, U: np.ndarray, p: Params, dagger: bool = False) -> np.ndarray:
    """Full 5d D_DW(m) (Eq. MoebiusOp), or its adjoint, on a full 5d field."""
    psi, U = _c(psi), _c(U)
    out = np.empty_like(psi)
    _load().or_ddw(_ptr(out), _ptr(psi), _ptr(U), ctypes.byref(p.c()), int(dagger))
    return out


def mee(psi_h: np.ndarray, p: Params, dagger: bool = False) -> np.ndarray:
    """Site-diagonal red/black block I_rr (Eq. D_5d_matrix) on a half field."""
    psi_h = _c(psi_h)
    out = np.empty_like(psi_h)
    _load().or_mee(_ptr(out), _ptr(psi_h), ctypes.byref(p.c()), int(dagger))
    return out


def mee_inv(psi_h: np.ndarray, p: Params, dagger: bool = False) -> np.ndarray:
    """I_rr^-1 (or I_rr^-dag) by the closed form of Sec. 3 on a half field."""
    psi_h = _c(psi_h)
    out = np.empty_like(psi_h)
    nsites = psi_h.size // (12 * p.Ls)
    _load().or_mee_inv(_ptr(out), _ptr(psi_h), nsites, ctypes.byref(p.c()), int(dagger))
    return out


def dhop(psi_h: np.ndarray, U: np.ndarray, p: Params, out_parity: int, dagger: bool = False) -> np.ndarray:
    """Hopping block into parity ``out_parity`` (D_rb for 0, D_br for 1)."""
    psi_h, U = _c(psi_h), _c(U)
    out = np.empty_like(psi_h)
    _load().or_dhop(_ptr(out), _ptr(psi_h), _ptr(U), ctypes.byref(p.c()), int(out_parity), int(dagger))
    return out


def m(psi_o: np.ndarray, U: np.ndarray, p: Params, dagger: bool = False) -> np.ndarray:
    """Preconditioned operator M = 1 - I^-1 D_br I^-1 D_rb (or M^dag) on an odd half field."""
    psi_o, U = _c(psi_o), _c(U)
    out = np.empty_like(psi_o)
    _load().or_m(_ptr(out), _ptr(psi_o), _ptr(U), ctypes.byref(p.c()), int(dagger))
    return out


def mdagm(psi_o: np.ndarray, U: np.ndarray, p: Params) -> np.ndarray:
    psi_o, U = _c(psi_o), _c(U)
    out = np.empty_like(psi_o)
    _load().or_mdagm(_ptr(out), _ptr(psi_o), _ptr(U), ctypes.byref(p.c()))
    return out


def cgne(bprime: np.ndarray, U: np.ndarray, p: Params, tol: float = 1e-10, maxiter: int = 10000,
         x0: np.ndarray | None = None):
    """CG on M^dag M x = M^dag b'. Returns (x, status, iterations, true relative residual)."""
    bprime, U = _c(bprime), _c(U)
    x = np.zeros_like(bprime) if x0 is None else _c(x0).copy()
    it, rel = ctypes.c_int(0), ctypes.c_double(0)
    st = _load().or_cgne(_ptr(x), _ptr(bprime), _ptr(U), ctypes.byref(p.c()), float(tol), int(maxiter),
                         ctypes.byref(it), ctypes.byref(rel))
    return x, int(st), int(it.value), float(rel.value)


def prepare(b_full: np.ndarray, U: np.ndarray, p: Params) -> np.ndarray:
    """b'_o = I^-1 (b_o - D_br I^-1 b_e) as an odd half field."""
    b_full, U = _c(b_full), _c(U)
    out = np.empty((p.Ls, p.V // 2, 4, 3), dtype=np.complex128)
    _load().or_prepare(_ptr(out), _ptr(b_full), _ptr(U), ctypes.byref(p.c()))
    return out


def reconstruct(x_odd: np.ndarray, b_full: np.ndarray, U: np.ndarray, p: Params) -> np.ndarray:
    """Full x from x_o: x_e = I^-1 (b_e - D_rb x_o)."""
    x_odd, b_full, U = _c(x_odd), _c(b_full), _c(U)
    out = np.empty_like(b_full)
    _load().or_reconstruct(_ptr(out), _ptr(x_odd), _ptr(b_full), _ptr(U), ctypes.byref(p.c()))
    return out


def solve(b_full: np.ndarray, U: np.ndarray, p: Params, tol: float = 1e-10, maxiter: int = 10000):
    """Full D_DW(m) x = b via prepare / CGNE / reconstruct. Returns (x, status, iters, rel)."""
    b_full, U = _c(b_full), _c(U)
    x = np.empty_like(b_full)
    it, rel = ctypes.c_int(0), ctypes.c_double(0)
    st = _load().or_solve(_ptr(x), _ptr(b_full), _ptr(U), ctypes.byref(p.c()), float(tol), int(maxiter),
                          ctypes.byref(it), ctypes.byref(rel))
    return x, int(st), int(it.value), float(rel.value)


def dm_dparam(X: np.ndarray, U: np.ndarray, p: Params, which: str) -> np.ndarray:
    """dM/db5 X (which='b5') or dM/dc5 X (which='c5'); constant b5, c5 only."""
    if p.s_dependent:
        raise ValueError("dM/db5, dM/dc5 are defined for constant b5, c5 only")
    X, U = _c(X), _c(U)
    out = np.empty_like(X)
    _load().or_dm_dparam(_ptr(out), _ptr(X), _ptr(U), ctypes.byref(p.c()), {"b5": 0, "c5": 1}[which])
    return out


def solve_dag(b: np.ndarray, U: np.ndarray, p: Params, tol: float = 1e-12, maxiter: int = 20000):
    """x = D_DW(m)^-dag b on a full 5d field by CG on D D^dag (no red/black split).
    Returns (x, status, iters, |D^dag x - b| / |b|)."""
    b, U = _c(b), _c(U)
    x = np.empty_like(b)
    it, rel = ctypes.c_int(0), ctypes.c_double(0)
    st = _load().or_solve_dag(_ptr(x), _ptr(b), _ptr(U), ctypes.byref(p.c()), float(tol), int(maxiter),
                              ctypes.byref(it), ctypes.byref(rel))
    return x, int(st), int(it.value), float(rel.value)


def force(phi: np.ndarray, U: np.ndarray, p: Params, tol: float = 1e-12, maxiter: int = 20000):
    """S = phi^dag (M^dag M)^-1 phi and dS/dU, dS/db5, dS/dc5 (with a chemical
    potential when p.mu is set).

    dS/dU has the gauge field's shape; a variation dU changes S by
    Re sum(conj(dSdU) * dU). With per-slice coefficients dSdb5 and dSdc5 are arrays of
    Ls values, dS/db5(s) and dS/dc5(s). Returns (S, dSdU, dSdb5, dSdc5, status, iters).
    """
    phi, U = _c(phi), _c(U)
    G = np.zeros_like(U)
    n = p.Ls if p.s_dependent else 1
    S, db5, dc5 = ctypes.c_double(0), (ctypes.c_double * n)(), (ctypes.c_double * n)()
    it = ctypes.c_int(0)
    st = _load().or_force(_ptr(G), db5, dc5, ctypes.byref(S), _ptr(phi), _ptr(U),
                          ctypes.byref(p.c()), float(tol), int(maxiter), ctypes.byref(it))
    if p.s_dependent:
        return float(S.value), G, np.array(db5[:]), np.array(dc5[:]), int(st), int(it.value)
    return float(S.value), G, float(db5[0]), float(dc5[0]), int(st), int(it.value)


# ------------------------------------------------------------- layout helpers

def parity_mask(dims) -> np.ndarray:
    """Boolean (T, Z, Y, X) mask of odd sites."""
    x, y, z, t = (int(d) for d in dims)
    tt, zz, yy, xx = np.meshgrid(np.arange(t), np.arange(z), np.arange(y), np.arange(x), indexing="ij")
    return ((xx + yy + zz + tt) & 1) == 1


def split(full: np.ndarray, dims) -> tuple[np.ndarray, np.ndarray]:
    """Full 5d field (..., Ls, T, Z, Y, X, 4, 3) -> (even, odd) half fields (..., Ls, V/2, 4, 3)."""
    mask = parity_mask(dims).reshape(-1)
    lead = full.shape[:-7]
    Ls = full.shape[-7]
    f = full.reshape(lead + (Ls, -1, 4, 3))
    return np.ascontiguousarray(f[..., ~mask, :, :]), np.ascontiguousarray(f[..., mask, :, :])


def join(even: np.ndarray, odd: np.ndarray, dims) -> np.ndarray:
    """Inverse of :func:`split`."""
    x, y, z, t = (int(d) for d in dims)
    mask = parity_mask(dims).reshape(-1)
    lead = even.shape[:-3]
    out = np.empty(lead + (x * y * z * t, 4, 3), dtype=np.complex128)
    out[..., ~mask, :, :] = even
    out[..., mask, :, :] = odd
    return out.reshape(lead + (t, z, y, x, 4, 3))
