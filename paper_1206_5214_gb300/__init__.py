"""Python binding of libmdwf, the GB300 (sm_103a) Moebius domain-wall operator.

The functions here carry the names of the C entry points in ``include/mdwf.h``
and only marshal arguments: every step of the operator and the solve runs in
the library's CUDA kernels. Buffers are passed as ``torch.Tensor`` (device or
host) or ``numpy.ndarray`` (host); their pointers go straight to the C call.
There is no CPU fallback: if ``libmdwf.so`` cannot be loaded every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

__all__ = [
    "MDWF_F64", "MDWF_F32", "MDWF_F16N", "MdwfError", "lib_path", "load",
    "mdwf_create", "mdwf_destroy", "mdwf_create_slab", "mdwf_slab_face_bytes", "mdwf_slab_stage",
    "mdwf_bounds_status", "mdwf_set_stream", "mdwf_set_s_coefficients", "mdwf_get_s_coefficients",
    "mdwf_set_chemical_potential",
    "mdwf_load_gauge", "mdwf_field_bytes",
    "mdwf_field_import", "mdwf_field_export", "mdwf_apply", "mdwf_apply_dag", "mdwf_cgne",
    "mdwf_apply_full", "mdwf_overlap_apply", "mdwf_pv_reconstruct", "mdwf_gw_violation", "mdwf_force4d",
    "mdwf_strerror", "mdwf_force", "mdwf_apply_noalloc", "mdwf_autotune", "mdwf_set_tuning",
    "mdwf_get_tuning", "mdwf_set_staging", "mdwf_get_staging", "mdwf_device_status", "mdwf_selftest_wait",
    "mdwf_profile_enable", "mdwf_profile_read", "mdwf_counters", "SolveParams", "SolveInfo", "KernelStat",
    "MDWF_OK", "MDWF_EINVAL", "MDWF_ENOMEM", "MDWF_ECUDA", "MDWF_ENOCONV", "MDWF_EBREAKDOWN", "MDWF_ETIMEOUT",
    "MDWF_ENOGAUGE", "STAGE_AUTO", "STAGE_CP_ASYNC", "STAGE_BULK", "STAGE_PREFETCH", "STAGE_REGISTERS",
]

MDWF_F64, MDWF_F32, MDWF_F16N = 0, 1, 2
MDWF_HOST, MDWF_DEVICE = 0, 1
MDWF_OK, MDWF_EINVAL, MDWF_ENOMEM, MDWF_ECUDA, MDWF_ENOCONV, MDWF_EBREAKDOWN, MDWF_ETIMEOUT, MDWF_ENOGAUGE = range(8)
_lib = None


class MdwfError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = f"{where}: {mdwf_strerror(status)}"
        if _lib is not None:
            extra = _lib.mdwf_last_error().decode()
            if extra:
                msg += f" ({extra})"
        super().__init__(msg)
        self.status = status


class _Opts(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_void_p), ("device", ctypes.c_int), ("dense_s", ctypes.c_int),
                ("autotune", ctypes.c_int)]


class SolveParams(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxiter", ctypes.c_int), ("inner_prec", ctypes.c_int),
                ("delta", ctypes.c_double), ("check_every", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("guess", ctypes.c_int)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("launches", ctypes.c_longlong), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("flops", ctypes.c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("reliable_updates", ctypes.c_int),
                ("true_res", ctypes.c_double), ("res_m", ctypes.c_double), ("seconds", ctypes.c_double),
                ("restarts", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libmdwf.so (building it with nvcc if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise OSError(f"libmdwf.so not found at {path}; run paper_1206_5214_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, ip, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    dp = ctypes.POINTER(ctypes.c_double)
    sig = {
        "mdwf_create": (ip, [ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int), ip, ctypes.c_double,
                             ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.POINTER(_Opts)]),
        "mdwf_destroy": (ip, [vp]),
        "mdwf_create_slab": (ip, [ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int), ip, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.POINTER(_Opts)]),
        "mdwf_slab_face_bytes": (sz, [vp, ip, ip]),
        "mdwf_bounds_status": (ip, [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), ip]),
        "mdwf_slab_stage": (ip, [vp, ip, vp, vp, ip, ip, dp, ip, vp, vp]),
        "mdwf_set_stream": (ip, [vp, vp]),
        "mdwf_set_s_coefficients": (ip, [vp, dp, dp]),
        "mdwf_set_chemical_potential": (ip, [vp, ctypes.c_double]),
        "mdwf_get_s_coefficients": (ip, [vp, dp, dp, ctypes.POINTER(ctypes.c_int)]),
        "mdwf_load_gauge": (ip, [vp, vp, ip]),
        "mdwf_field_bytes": (sz, [vp, ip, ip]),
        "mdwf_field_import": (ip, [vp, vp, vp, ip, ip, ip]),
        "mdwf_field_export": (ip, [vp, vp, vp, ip, ip, ip]),
        "mdwf_apply": (ip, [vp, vp, vp, ip, ip, dp]),
        "mdwf_apply_dag": (ip, [vp, vp, vp, ip, ip, dp]),
        "mdwf_cgne": (ip, [vp, vp, vp, ip, dp, ip, ctypes.POINTER(SolveParams), ctypes.POINTER(SolveInfo)]),
        "mdwf_apply_noalloc": (ip, [vp, vp, vp, ip, ip, dp, ip]),
        "mdwf_apply_full": (ip, [vp, vp, vp, ip, dp, ip, ip]),
        "mdwf_overlap_apply": (ip, [vp, vp, vp, ip, dp, ip, ctypes.POINTER(SolveParams), ctypes.POINTER(SolveInfo)]),
        "mdwf_pv_reconstruct": (ip, [vp, vp, vp, ip, dp, ip, ctypes.POINTER(SolveParams), ctypes.POINTER(SolveInfo)]),
        "mdwf_gw_violation": (ip, [vp, vp, vp, ip, dp, ip, ctypes.POINTER(SolveParams), ctypes.POINTER(SolveInfo)]),
        "mdwf_force4d": (ip, [vp, vp, dp, vp, ip, ctypes.POINTER(SolveParams), ctypes.POINTER(SolveInfo)]),
        "mdwf_force": (ip, [vp, vp, dp, dp, dp, vp, ip, ctypes.POINTER(SolveParams), ctypes.POINTER(SolveInfo)]),
        "mdwf_profile_enable": (ip, [vp, ip]),
        "mdwf_profile_read": (ip, [vp, ctypes.POINTER(KernelStat), ip, ctypes.POINTER(ctypes.c_int), ip]),
        "mdwf_counters": (ip, [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
        "mdwf_autotune": (ip, [vp, ip, ip, ctypes.POINTER(ctypes.c_int)]),
        "mdwf_set_tuning": (ip, [vp, ip, ip, ip]),
        "mdwf_get_tuning": (ip, [vp, ip, ip, ctypes.POINTER(ctypes.c_int)]),
        "mdwf_set_staging": (ip, [vp, ip, ip]),
        "mdwf_get_staging": (ip, [vp, ip, ctypes.POINTER(ctypes.c_int)]),
        "mdwf_device_status": (ip, [vp]),
        "mdwf_get_geometry": (ip, [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
        "mdwf_selftest_wait": (ip, [vp, ip]),
        "mdwf_strerror": (ctypes.c_char_p, [ip]),
        "mdwf_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status: int, where: str) -> None:
    if status != 0:
        raise MdwfError(status, where)


def _ptr_where(a) -> tuple[int, int]:
    """(pointer, MDWF_HOST / MDWF_DEVICE) of a torch tensor or numpy array."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy buffers must be C-contiguous")
        return a.ctypes.data, MDWF_HOST
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr(), (MDWF_DEVICE if a.is_cuda else MDWF_HOST)
    raise TypeError(f"unsupported buffer type {type(a)}")


def _masses(mf_per_rhs):
    if mf_per_rhs is None:
        return None
    arr = (ctypes.c_double * len(mf_per_rhs))(*[float(m) for m in mf_per_rhs])
    return arr


def mdwf_strerror(status: int) -> str:
    return load().mdwf_strerror(int(status)).decode()


def mdwf_create(dims, Ls: int, M5: float, b5: float, c5: float, mf: float, stream=None, device: int = -1,
                dense_s: bool = False, autotune: bool = False):
    """Create a context; returns an opaque handle (int). ``stream``: torch.cuda.Stream, raw handle or None.
    ``dense_s``: apply the Ls x Ls factors as dense matrices instead of the closed-form elimination."""
    lib = load()
    h = ctypes.c_void_p()
    d = (ctypes.c_int * 4)(*[int(x) for x in dims])
    opts = _Opts(_stream_handle(stream), int(device), int(bool(dense_s)), int(bool(autotune)))
    _check(lib.mdwf_create(ctypes.byref(h), d, int(Ls), float(M5), float(b5), float(c5), float(mf),
                           ctypes.byref(opts)), "mdwf_create")
    return h.value


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def mdwf_create_slab(local_dims, Ls: int, M5: float, b5: float, c5: float, mf: float, stream=None,
                     device: int = -1, dense_s: bool = False):
    """Context of one t-slab of a lattice split along t (local_dims = (X, Y, Z, T/n))."""
    lib = load()
    h = ctypes.c_void_p()
    d = (ctypes.c_int * 4)(*[int(x) for x in local_dims])
    opts = _Opts(_stream_handle(stream), int(device), int(bool(dense_s)), 0)
    _check(lib.mdwf_create_slab(ctypes.byref(h), d, int(Ls), float(M5), float(b5), float(c5), float(mf),
                                ctypes.byref(opts)), "mdwf_create_slab")
    return h.value


def mdwf_slab_face_bytes(ctx, prec: int, nrhs: int = 1) -> int:
    return int(load().mdwf_slab_face_bytes(ctx, int(prec), int(nrhs)))


def mdwf_slab_stage(ctx, stage: int, out, inp, prec: int, nrhs: int = 1, mf_per_rhs=None, dagger: bool = False,
                    send=None, recv=None) -> None:
    """One of the three stages of M (or M^dag) on a t-slab; send / recv: face buffers (device)."""
    ptr = lambda t: None if t is None else _ptr_where(t)[0]
    _check(load().mdwf_slab_stage(ctx, int(stage), ptr(out), ptr(inp), int(prec), int(nrhs), _masses(mf_per_rhs),
                                  int(bool(dagger)), ptr(send), ptr(recv)), "mdwf_slab_stage")


def mdwf_bounds_status(reset: bool = False) -> tuple[bool, bool]:
    """(checked, violated): whether the loaded library is the bounds-checked debug build,
    and whether one of its kernels computed an index out of range since the last reset."""
    checked, bad = ctypes.c_int(), ctypes.c_int()
    _check(load().mdwf_bounds_status(ctypes.byref(checked), ctypes.byref(bad), int(bool(reset))),
           "mdwf_bounds_status")
    return bool(checked.value), bool(bad.value)


def mdwf_destroy(ctx) -> None:
    _check(load().mdwf_destroy(ctx), "mdwf_destroy")


def mdwf_set_stream(ctx, stream) -> None:
    _check(load().mdwf_set_stream(ctx, _stream_handle(stream)), "mdwf_set_stream")


def mdwf_set_s_coefficients(ctx, b5s, c5s) -> None:
    """Per-slice b5(s), c5(s) (Ls values each, slice order s = 0..Ls-1), or both None
    for the constant b5, c5 given at creation."""
    if (b5s is None) != (c5s is None):
        raise ValueError("give both b5s and c5s, or neither")
    if b5s is None:
        _check(load().mdwf_set_s_coefficients(ctx, None, None), "mdwf_set_s_coefficients")
        return
    b = (ctypes.c_double * len(b5s))(*[float(v) for v in b5s])
    c = (ctypes.c_double * len(c5s))(*[float(v) for v in c5s])
    _check(load().mdwf_set_s_coefficients(ctx, b, c), "mdwf_set_s_coefficients")


def mdwf_set_chemical_potential(ctx, mu: float) -> None:
    """Chemical potential on the time links (e^{+mu} forward, e^{-mu} backward); 0 turns it off."""
    _check(load().mdwf_set_chemical_potential(ctx, float(mu)), "mdwf_set_chemical_potential")


def mdwf_get_geometry(ctx) -> tuple[tuple[int, int, int, int], int]:
    """((x, y, z, t), Ls) of the context."""
    d = (ctypes.c_int * 4)()
    Ls = ctypes.c_int(0)
    _check(load().mdwf_get_geometry(ctx, d, ctypes.byref(Ls)), "mdwf_get_geometry")
    return tuple(d), Ls.value


def mdwf_get_s_coefficients(ctx, Ls: int):
    """(b5s, c5s, per_slice): the Ls coefficients in force and whether they are per-slice."""
    b = (ctypes.c_double * Ls)()
    c = (ctypes.c_double * Ls)()
    flag = ctypes.c_int(0)
    _check(load().mdwf_get_s_coefficients(ctx, b, c, ctypes.byref(flag)), "mdwf_get_s_coefficients")
    return list(b), list(c), bool(flag.value)


def mdwf_load_gauge(ctx, U) -> None:
    p, where = _ptr_where(U)
    _check(load().mdwf_load_gauge(ctx, p, where), "mdwf_load_gauge")


def mdwf_field_bytes(ctx, prec: int, nrhs: int = 1) -> int:
    return int(load().mdwf_field_bytes(ctx, int(prec), int(nrhs)))


def mdwf_field_import(ctx, dst, src, prec: int, nrhs: int = 1) -> None:
    pd, wd = _ptr_where(dst)
    if wd != MDWF_DEVICE:
        raise ValueError("internal fields live in device memory")
    ps, ws = _ptr_where(src)
    _check(load().mdwf_field_import(ctx, pd, ps, int(prec), int(nrhs), ws), "mdwf_field_import")


def mdwf_field_export(ctx, dst, src, prec: int, nrhs: int = 1) -> None:
    pd, wd = _ptr_where(dst)
    ps, ws = _ptr_where(src)
    if ws != MDWF_DEVICE:
        raise ValueError("internal fields live in device memory")
    _check(load().mdwf_field_export(ctx, pd, ps, int(prec), int(nrhs), wd), "mdwf_field_export")


def mdwf_apply(ctx, out, inp, prec: int, nrhs: int = 1, mf_per_rhs=None) -> None:
    po, _ = _ptr_where(out)
    pi, _ = _ptr_where(inp)
    _check(load().mdwf_apply(ctx, po, pi, int(prec), int(nrhs), _masses(mf_per_rhs)), "mdwf_apply")


def mdwf_apply_dag(ctx, out, inp, prec: int, nrhs: int = 1, mf_per_rhs=None) -> None:
    po, _ = _ptr_where(out)
    pi, _ = _ptr_where(inp)
    _check(load().mdwf_apply_dag(ctx, po, pi, int(prec), int(nrhs), _masses(mf_per_rhs)), "mdwf_apply_dag")


def mdwf_cgne(ctx, x, b, nrhs: int = 1, mf_per_rhs=None, tol: float = 1e-10, maxiter: int = 20000,
              inner_prec: int = MDWF_F64, delta: float = 0.0, check_every: int = 8, use_graph: bool = True,
              raise_on_error: bool = True, guess: bool = False):
    """Solve D_DW(m) x = b (full 5d fields, complex128, user order). Returns (status, [SolveInfo per rhs]).
    guess=True starts the CG from the odd part of the x passed in."""
    px, wx = _ptr_where(x)
    pb, wb = _ptr_where(b)
    if wx != wb:
        raise ValueError("x and b must both be host or both be device buffers")
    prm = SolveParams(float(tol), int(maxiter), int(inner_prec), float(delta), int(check_every), int(bool(use_graph)),
                      int(bool(guess)))
    infos = (SolveInfo * int(nrhs))()
    st = load().mdwf_cgne(ctx, px, pb, int(nrhs), _masses(mf_per_rhs), wb, ctypes.byref(prm), infos)
    if raise_on_error and st not in (0,):
        raise MdwfError(st, "mdwf_cgne")
    return st, list(infos)


def mdwf_apply_full(ctx, out, inp, nrhs: int = 1, mf_per_rhs=None, dagger: bool = False) -> None:
    """out = D_DW(m) in (or its adjoint) on full 5d fields (complex128, user order), FP64."""
    po, wo = _ptr_where(out)
    pi, wi = _ptr_where(inp)
    if wo != wi:
        raise ValueError("out and in must both be host or both be device buffers")
    _check(load().mdwf_apply_full(ctx, po, pi, int(nrhs), _masses(mf_per_rhs), wi, int(bool(dagger))),
           "mdwf_apply_full")


def _pv_call(fn, name, ctx, out, psi, nrhs, mf_per_rhs, tol, maxiter, raise_on_error, inner_prec=MDWF_F64):
    po, wo = _ptr_where(out)
    pp, wp = _ptr_where(psi)
    if wo != wp:
        raise ValueError("both buffers must be host or both device")
    prm = SolveParams(float(tol), int(maxiter), int(inner_prec), 0.0, 8, 1)
    infos = (SolveInfo * int(nrhs))()
    st = fn(ctx, po, pp, int(nrhs), _masses(mf_per_rhs), wp, ctypes.byref(prm), infos)
    if raise_on_error and st != 0:
        raise MdwfError(st, name)
    return st, list(infos)


def mdwf_overlap_apply(ctx, out4, psi4, nrhs: int = 1, mf_per_rhs=None, tol: float = 1e-12, maxiter: int = 20000,
                       raise_on_error: bool = True, inner_prec: int = MDWF_F64):
    """out4 = D_ov(m) psi4 through a Pauli-Villars solve; returns (status, [SolveInfo])."""
    return _pv_call(load().mdwf_overlap_apply, "mdwf_overlap_apply", ctx, out4, psi4, nrhs, mf_per_rhs, tol,
                    maxiter, raise_on_error, inner_prec)


def mdwf_pv_reconstruct(ctx, Psi5, psi4, nrhs: int = 1, mf_per_rhs=None, tol: float = 1e-12, maxiter: int = 20000,
                        raise_on_error: bool = True, inner_prec: int = MDWF_F64):
    """5d Psi (Sec. 2.3) from the 4d overlap solution psi4; returns (status, [SolveInfo])."""
    return _pv_call(load().mdwf_pv_reconstruct, "mdwf_pv_reconstruct", ctx, Psi5, psi4, nrhs, mf_per_rhs, tol,
                    maxiter, raise_on_error, inner_prec)


def mdwf_gw_violation(ctx, out4, psi4, nrhs: int = 1, mf_per_rhs=None, tol: float = 1e-12, maxiter: int = 20000,
                      raise_on_error: bool = True, inner_prec: int = MDWF_F64):
    """out4 = Delta_Ls psi4 = (1 - eps^2) psi4 / 4 through two overlap applications."""
    return _pv_call(load().mdwf_gw_violation, "mdwf_gw_violation", ctx, out4, psi4, nrhs, mf_per_rhs, tol, maxiter,
                    raise_on_error, inner_prec)


def mdwf_apply_noalloc(ctx, out, inp, prec: int, nrhs: int = 1, mf_per_rhs=None, dagger: bool = False) -> None:
    """M (or M^dag) like mdwf_apply, with the intermediates in the library's fixed scratch (no allocation)."""
    po, _ = _ptr_where(out)
    pi, _ = _ptr_where(inp)
    _check(load().mdwf_apply_noalloc(ctx, po, pi, int(prec), int(nrhs), _masses(mf_per_rhs), int(bool(dagger))),
           "mdwf_apply_noalloc")


def mdwf_force(ctx, dSdU, phi, tol: float = 1e-12, maxiter: int = 40000, inner_prec: int = MDWF_F64,
               use_graph: bool = True, raise_on_error: bool = True):
    """S = phi^dag (M^dag M)^-1 phi, dS/dU (written into dSdU, gauge layout) and dS/db5, dS/dc5.

    Returns (S, dSdb5, dSdc5, status, SolveInfo); with per-slice coefficients dSdb5 and
    dSdc5 are arrays of Ls values (dS/db5(s), dS/dc5(s))."""
    pp, wp = _ptr_where(phi)
    if dSdU is None:
        pg = None
    else:
        pg, wg = _ptr_where(dSdU)
        if wg != wp:
            raise ValueError("dSdU and phi must both be host or both be device buffers")
    prm = SolveParams(float(tol), int(maxiter), int(inner_prec), 0.0, 8, int(bool(use_graph)))
    info = SolveInfo()
    _, Ls = mdwf_get_geometry(ctx)
    per_slice = mdwf_get_s_coefficients(ctx, Ls)[2]
    n = Ls if per_slice else 1
    S, db5, dc5 = ctypes.c_double(0), (ctypes.c_double * n)(), (ctypes.c_double * n)()
    derivs = dSdU is not None
    st = load().mdwf_force(ctx, pg, db5 if derivs else None, dc5 if derivs else None,
                           ctypes.byref(S), pp, wp, ctypes.byref(prm), ctypes.byref(info))
    if raise_on_error and st != 0:
        raise MdwfError(st, "mdwf_force")
    if per_slice:
        return S.value, np.array(db5[:]), np.array(dc5[:]), st, info
    return S.value, db5[0], dc5[0], st, info


def mdwf_force4d(ctx, dSdU, phi4, tol: float = 1e-12, maxiter: int = 40000, raise_on_error: bool = True,
                 inner_prec: int = MDWF_F64):
    """S = |D(1)^dag D(m)^-dag P phi|^2 for a 4d wall pseudofermion and dS/dU (into dSdU, or
    None for S only). Returns (S, status, SolveInfo)."""
    pp, wp = _ptr_where(phi4)
    pg = None
    if dSdU is not None:
        pg, wg = _ptr_where(dSdU)
        if wg != wp:
            raise ValueError("dSdU and phi must both be host or both be device buffers")
    prm = SolveParams(float(tol), int(maxiter), int(inner_prec), 0.0, 8, 1)
    info = SolveInfo()
    S = ctypes.c_double(0)
    st = load().mdwf_force4d(ctx, pg, ctypes.byref(S), pp, wp, ctypes.byref(prm), ctypes.byref(info))
    if raise_on_error and st != 0:
        raise MdwfError(st, "mdwf_force4d")
    return S.value, st, info


def mdwf_profile_enable(ctx, enable: bool = True) -> None:
    _check(load().mdwf_profile_enable(ctx, int(bool(enable))), "mdwf_profile_enable")


def mdwf_profile_read(ctx, reset: bool = False) -> list[dict]:
    """Per-kernel launches, total ms (CUDA events) and algorithmic bytes / flops."""
    out = (KernelStat * 64)()
    n = ctypes.c_int(0)
    _check(load().mdwf_profile_read(ctx, out, 64, ctypes.byref(n), int(bool(reset))), "mdwf_profile_read")
    return [{"name": out[i].name.decode(), "launches": out[i].launches, "ms": out[i].ms,
             "bytes": out[i].bytes, "flops": out[i].flops} for i in range(n.value)]


STAGE_AUTO, STAGE_CP_ASYNC, STAGE_BULK, STAGE_PREFETCH, STAGE_REGISTERS = 0, 1, 2, 3, 4


def mdwf_set_staging(ctx, prec: int, staged: int) -> None:
    """Neighbour loads of the FP32 / FP16 hop kernels: 0 the default (register prefetch except
    in the fused residual update), 1 through shared memory with per-thread cp.async, 2 whole
    neighbour columns by bulk copies (TMA), 3 register prefetch everywhere, 4 plain register
    loads everywhere."""
    _check(load().mdwf_set_staging(ctx, int(prec), int(staged)), "mdwf_set_staging")


def mdwf_get_staging(ctx, prec: int) -> int:
    v = ctypes.c_int(0)
    _check(load().mdwf_get_staging(ctx, int(prec), ctypes.byref(v)), "mdwf_get_staging")
    return v.value


def mdwf_device_status(ctx) -> int:
    """Synchronise the context's stream; MDWF_ETIMEOUT if a bounded device wait gave up since
    the last report (the mark is cleared), else MDWF_OK (a CUDA error raises)."""
    st = load().mdwf_device_status(ctx)
    if st not in (MDWF_OK, MDWF_ETIMEOUT):
        _check(st, "mdwf_device_status")
    return st


def mdwf_selftest_wait(ctx, arrivals: int) -> int:
    """Bounded-wait self-test: MDWF_ETIMEOUT unless both expected arrivals are made."""
    st = load().mdwf_selftest_wait(ctx, int(arrivals))
    if st not in (MDWF_OK, MDWF_ETIMEOUT):
        _check(st, "mdwf_selftest_wait")
    return st


def mdwf_counters(ctx) -> tuple[int, list[int]]:
    """(kernel launches, [M/M^dag applications in F64, F32, F16N]) since mdwf_create."""
    launches = ctypes.c_longlong(0)
    applies = (ctypes.c_longlong * 3)()
    _check(load().mdwf_counters(ctx, ctypes.byref(launches), applies), "mdwf_counters")
    return int(launches.value), [int(a) for a in applies]


def mdwf_autotune(ctx, prec: int, nrhs: int = 1) -> int:
    """Tune the hop kernels' block shape for (prec, nrhs); returns the chosen 4d sites per block."""
    sb = ctypes.c_int(0)
    _check(load().mdwf_autotune(ctx, int(prec), int(nrhs), ctypes.byref(sb)), "mdwf_autotune")
    return int(sb.value)


def mdwf_set_tuning(ctx, prec: int, nrhs: int, sites_per_block: int) -> None:
    _check(load().mdwf_set_tuning(ctx, int(prec), int(nrhs), int(sites_per_block)), "mdwf_set_tuning")


def mdwf_get_tuning(ctx, prec: int, nrhs: int = 1) -> int:
    sb = ctypes.c_int(0)
    _check(load().mdwf_get_tuning(ctx, int(prec), int(nrhs), ctypes.byref(sb)), "mdwf_get_tuning")
    return int(sb.value)
