#!/usr/bin/env python
"""Benchmark of the red/black Moebius domain-wall hot path on GB300.

Workload (one "step"): a full solve D_DW(m) x = b on a 16^3 x 32 lattice,
Ls = 16, M5 = 1.8, mf = 0.01, b5 = 1.5, c5 = 0.5 (alpha = b5 + c5 = 2,
b5 - c5 = 1), SU(3) links exp(i 0.2 H), one Gaussian source: red/black source
preparation, CGNE on M^dag M to a true FP64 residual of 1e-10 with the
operator in FP32 (mixed precision, FP64 reliable updates), reconstruction.

metric: Moebius Dslash GFLOP/s over the solve = (M and M^dag applications
x 3120 flops per odd 5d site) / step time, inputs resident in HBM. Extra keys
report the per-precision Dslash rate, the time to solution of the mixed and
plain FP64 solves, the roofline of the dominant kernel (CUDA events around
each launch in one profiled solve of the same workload), the FP64 oracle on
the host cores, and the end-to-end rate through mdwf_cgne with host buffers.

Multi-GPU: every rank solves its own source (independent problems, no
collective on the data path); value = all ranks' flops / max rank time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = (16, 16, 16, 32)
LS, M5, B5, C5, MF, EPS = 16, 1.8, 1.5, 0.5, 0.01, 0.2
GAUGE_SEED, SOURCE_SEED = 1002, 2002
FLOPS_PER_SITE = 3120.0      # per odd 5d site and M (or M^dag) application
# DRAM bytes (read + write) per launch of a kernel in this workload's solve come from one
# ncu capture, recorded (a JSON block) in a text file under profiles/ with the SHA-256 of the
# kernel's sources at capture time; a record whose hash differs from the sources as they
# are now is stale and is not reported.
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic_cgne_f32_16x16x16x32_Ls16.txt")
KERNEL_SOURCES = ("paper_1206_5214_gb300/csrc/hop_kernel.cuh", "paper_1206_5214_gb300/csrc/mdwf_internal.cuh",
                  "paper_1206_5214_gb300/csrc/mbarrier.cuh")
METRIC = "Moebius Dslash GFLOP/s in CGNE to 1e-10 (mixed FP32/FP64)"
# spectrum bounds of the Zolotarev coefficients of the per-slice solve: the upper one is
# lambda_max = (8 - M5) / (10 - M5) of the Shamir kernel at M5 = 1.8 (Sec. 2)
ZOLO_RANGE = (0.05, 0.756)
# the force workload: the same lattice and links, mf = 0.02, its own Gaussian phi
FORCE_MF, FORCE_SEED = 0.02, 2004
# the 4d field of the overlap application and the wall force, and the chemical potential
OVERLAP_SEED, CHEM_MU = 2005, 0.1
N5 = DIMS[0] * DIMS[1] * DIMS[2] * DIMS[3] // 2 * LS
# the batched workloads: 12 spin-colour point sources on 24^3 x 64, Ls = 12 (mixed FP32), and
# 8 Gaussian sources at 8 masses on 32^3 x 64, Ls = 16 (mixed FP16+norm, autotuned tiles)
BATCHED = {
    "c3_12_point_sources": {"dims": (24, 24, 24, 64), "Ls": 12, "mf": [0.005] * 12, "eps": 0.2, "cfg": 3,
                            "inner": "f32", "sources": "point", "autotune": False, "buffers": "device"},
    # 8 x 6.4 GB sources and solutions do not fit in HBM beside the solver's FP64 fields:
    # they stay in host memory and the library moves them (timed)
    "c5_8_masses": {"dims": (32, 32, 32, 64), "Ls": 16,
                    "mf": [0.001, 0.002, 0.005, 0.01, 0.02, 0.03, 0.04, 0.05], "eps": 0.15, "cfg": 5,
                    "inner": "f16n", "sources": "gaussian", "autotune": True, "buffers": "host"},
}


def workload_config(inner: str) -> dict:
    return {"workload": "mdwf-cgne 16^3x32 Ls=16 M5=1.8 mf=0.01 b5=1.5 c5=0.5 eps=0.2",
            "lattice": list(DIMS), "Ls": LS, "M5": M5, "b5": B5, "c5": C5, "mf": MF, "eps": EPS,
            "nrhs": 1, "tol": 1e-10, "inner": inner,
            "l2": "256 MB buffer written between timed steps (L2 129 MB); each step streams > 1 GB"}


def kernel_sources_sha256(files=KERNEL_SOURCES, root=ROOT) -> str:
    """SHA-256 over the hop kernels' source files, in a fixed order."""
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(root, f), "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read() + b"\0")
    return h.hexdigest()


def recorded_traffic(name: str, path: str = TRAFFIC_FILE, current_sha: str | None = None) -> tuple:
    """(DRAM bytes per launch, note) of kernel `name` from the capture record, or
    (None, why) when there is no record or the sources changed since the capture."""
    try:
        text = open(path).read()
        block = text.split("```json", 1)[1].split("```", 1)[0]
        rec = json.loads(block)["kernels"].get(name)
    except (OSError, ValueError, KeyError, IndexError):
        return None, "no capture record"
    if not rec:
        return None, f"no capture of {name}"
    sha = current_sha or kernel_sources_sha256()
    if rec.get("sources_sha256") != sha:
        return None, "stale: the kernel sources changed since the capture"
    return rec["dram_read_bytes"] + rec["dram_write_bytes"], f"ncu capture, {rec.get('summary', '')}"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["mdwf", "reference"], default="mdwf")
    ap.add_argument("--inner", choices=["f32", "f16n"], default="f32")
    ap.add_argument("--no-f64", action="store_true", help="skip the plain FP64 solve comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--quick", action="store_true", help="small lattice, for debugging only")
    ap.add_argument("--solve-only", action="store_true",
                    help="only the warm-up and timed solves (a short, fixed launch sequence for ncu)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the per-precision Dslash loops, the second inner precision and the e2e leg")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the full-size batched solves (12 point sources at 24^3x64 Ls=12, 8 masses at "
                         "32^3x64 Ls=16)")
    ap.add_argument("--apply-only", choices=["f64", "f32", "f16n"], default=None,
                    help="only time M applications in this precision (a fixed launch sequence for ncu)")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.gpu_id is not None:
                cmd += ["-i", self.gpu_id]
            self.proc = subprocess.Popen(cmd, stdout=self.file, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        if self.proc is None or self.file is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), float(parts[3]) if parts[3] not in ("[N/A]", "N/A") else 0.0,
                                 parts[5:9]))
                except ValueError:
                    continue
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(rows), "reasons": reasons}


def gpu_identifier(torch) -> str | None:
    try:
        u = torch.cuda.get_device_properties(torch.cuda.current_device()).uuid
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        return vis.split(",")[0] if vis else None


# ------------------------------------------------------------ oracle (CPU)

def cpu_baseline(dims, Ls) -> dict:
    """The FP64 oracle on this host's cores: a bounded sample of the same
    workload, six CG iterations' worth of operator work (M and M^dag six times,
    about 10 s on 16 Grace cores)."""
    import numpy as np
    import oracle
    import synthetic as sy
    oracle.build()
    p = oracle.Params(dims, Ls, M5, B5, C5, MF)
    U = sy.gauge_field(dims, EPS, GAUGE_SEED)
    _, xo = oracle.split(sy.gaussian_field(dims, Ls, SOURCE_SEED), dims)
    t0 = time.perf_counter()
    v = xo
    reps = 6
    for _ in range(reps):
        v = oracle.m(v, U, p)
        v = oracle.m(v, U, p, dagger=True)
    dt = time.perf_counter() - t0
    n5 = int(np.prod(dims)) // 2 * Ls
    gf = 2 * reps * FLOPS_PER_SITE * n5 / dt / 1e9
    cores = oracle.get_threads()
    # one host thread: one M application
    oracle.set_threads(1)
    try:
        t1 = time.perf_counter()
        v = oracle.m(xo, U, p)
        dt1 = time.perf_counter() - t1
    finally:
        oracle.set_threads(cores)
    return {"value": gf, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
            "sample": f"{2 * reps} applications (M, M^dag alternating) of the FP64 oracle on the full "
                      f"workload lattice, {dt:.1f} s",
            "single_thread": {"value": FLOPS_PER_SITE * n5 / dt1 / 1e9, "unit": "GFLOP/s", "cores": 1,
                              "sample": f"one M application on the same lattice, {dt1:.1f} s"}}


def run_reference(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    dims, Ls = DIMS, LS
    import numpy as np
    import oracle
    import synthetic as sy
    oracle.build()
    p = oracle.Params(dims, Ls, M5, B5, C5, MF)
    U = sy.gauge_field(dims, EPS, GAUGE_SEED)
    _, xo = oracle.split(sy.gaussian_field(dims, Ls, SOURCE_SEED), dims)
    # one step = one CG iteration's operator work (M then M^dag) on the workload
    def step(v):
        return oracle.m(oracle.m(v, U, p), U, p, dagger=True)
    v = xo
    for _ in range(args.warmup):
        v = step(v)
        v = v / np.linalg.norm(v)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v = step(v)
        v = v / np.linalg.norm(v)
    dt = time.perf_counter() - t0
    n5 = int(np.prod(dims)) // 2 * Ls
    val = 2 * FLOPS_PER_SITE * n5 * args.steps / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args.inner),
            "cpu_baseline": {"value": val, "unit": "GFLOP/s", "cores": oracle.get_threads(), "kind": "oracle",
                             "sample": "each step: M then M^dag of the FP64 oracle on the full workload lattice"},
            "e2e": {"value": val, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------- multi-rank logic

def rank_source_seed(rank: int) -> int:
    """Every rank solves its own source (independent problems, no data exchange)."""
    return SOURCE_SEED + 100 * rank


def combine_ranks(ms: float, flops: float, dist=None, device: str = "cpu") -> tuple[float, float]:
    """Whole-job timing: the slowest rank's time and the sum of all ranks' flops."""
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    f = torch.tensor([flops], dtype=torch.float64, device=device)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(f, op=dist.ReduceOp.SUM)
    return float(t.item()), float(f.item())


# --------------------------------------------------------------- GPU arm

def apply_only(args, h, b, dims, Ls, n5, flush) -> None:
    """warmup + steps applications of M on resident fields of one precision."""
    import numpy as np
    import torch
    import paper_1206_5214_gb300 as mdwf
    prec = {"f64": mdwf.MDWF_F64, "f32": mdwf.MDWF_F32, "f16n": mdwf.MDWF_F16N}[args.apply_only]
    Vh = int(np.prod(dims)) // 2
    src = torch.from_numpy(np.ascontiguousarray(b.reshape(Ls, -1, 4, 3)[:, :Vh])).cuda()
    fi = torch.empty(mdwf.mdwf_field_bytes(h, prec, 1), dtype=torch.uint8, device="cuda")
    fo = torch.empty_like(fi)
    mdwf.mdwf_field_import(h, fi, src, prec)
    for _ in range(args.warmup):
        mdwf.mdwf_apply(h, fo, fi, prec)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        mdwf.mdwf_apply(h, fo, fi, prec)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"apply_only": args.apply_only, "ms_per_M": ms,
                      "GFLOPs": FLOPS_PER_SITE * n5 / (ms * 1e-3) / 1e9}), flush=True)


def main() -> None:
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch

    import paper_1206_5214_gb300 as mdwf
    import synthetic as sy

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    dims, Ls = ((8, 8, 8, 8), 8) if args.quick else (DIMS, LS)
    n5 = dims[0] * dims[1] * dims[2] * dims[3] // 2 * Ls
    inner = mdwf.MDWF_F32 if args.inner == "f32" else mdwf.MDWF_F16N
    U = sy.gauge_field(dims, EPS, GAUGE_SEED)
    b = sy.gaussian_field(dims, Ls, rank_source_seed(rank))
    h = mdwf.mdwf_create(dims, Ls, M5, B5, C5, MF)
    Ud = torch.from_numpy(U).cuda()
    mdwf.mdwf_load_gauge(h, Ud)
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()

    def solve(prec, use_graph=True):
        st, info = mdwf.mdwf_cgne(h, xd, bd, tol=1e-10, inner_prec=prec, use_graph=use_graph)
        return info[0]

    if args.apply_only:
        apply_only(args, h, b, dims, Ls, n5, flush)
        mdwf.mdwf_destroy(h)
        return

    for _ in range(args.warmup):
        flush.zero_()
        solve(inner)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()

    # ---------------- timed region: K solves, device-resident inputs
    launches0, applies0 = mdwf.mdwf_counters(h)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    infos = []
    with ClockSampler(gpu_identifier(torch)) as clocks:
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record()
            infos.append(solve(inner))
            ev[k][1].record()
        torch.cuda.synchronize()
    launches1, applies1 = mdwf.mdwf_counters(h)
    ms = sum(a.elapsed_time(bb) for a, bb in ev)
    if args.solve_only:
        print(json.dumps({"solve_only": args.inner, "ms_per_solve": ms / args.steps, "iters": infos[-1].iters,
                          "true_res": infos[-1].true_res, "launches_per_solve": (launches1 - launches0) / args.steps}),
              flush=True)
        mdwf.mdwf_destroy(h)
        return
    applies = sum(applies1) - sum(applies0)
    flops = applies * FLOPS_PER_SITE * n5
    ms_max, flops_all = combine_ranks(ms, flops, dist, device="cuda")
    value = flops_all / (ms_max * 1e-3) / 1e9

    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        mdwf.mdwf_destroy(h)
        return

    # ---------------- dominant kernel: per-launch CUDA events in one profiled solve
    mdwf.mdwf_profile_read(h, reset=True)
    mdwf.mdwf_profile_enable(h, True)
    flush.zero_()
    prof_info = solve(inner, use_graph=False)
    stats = mdwf.mdwf_profile_read(h, reset=True)
    mdwf.mdwf_profile_enable(h, False)
    total_ms = sum(s["ms"] for s in stats)
    top = max(stats, key=lambda s: s["ms"])
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    achieved = top["bytes"] / top["launches"] / (top["ms"] / top["launches"] * 1e-3) / 1e9
    traffic, traffic_note = recorded_traffic(top["name"])
    roofline = {"kernel": top["name"], "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "peak_source": peak_src,
                "traffic": traffic, "traffic_source": traffic_note,
                "launches": top["launches"], "avg_us": 1e3 * top["ms"] / top["launches"],
                "share_of_solve_kernel_time": top["ms"] / total_ms,
                "algorithmic_bytes_per_launch": top["bytes"] / top["launches"]}
    # the whole inner iteration (its four hops, the vector update and the scalar
    # reductions, in the inner precision): algorithmic bytes over device time
    inner_tag = "_" + args.inner
    it = [st for st in stats if st["name"].endswith(inner_tag)]
    it_bytes, it_ms = sum(st["bytes"] for st in it), sum(st["ms"] for st in it)
    roofline_iteration = {"kernels": [st["name"] for st in it], "bound": "hbm",
                          "achieved": it_bytes / (it_ms * 1e-3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                          "frac": it_bytes / (it_ms * 1e-3) / 1e9 / hbm_peak,
                          "share_of_solve_kernel_time": it_ms / total_ms} if it and it_ms > 0 else None
    # the FP64 operator of the reliable updates, preparation and reconstruction is bound by
    # the FP64 pipe (GB300 runs FP64 at 1/64 of the FP32 rate): its roofline is the FP64
    # peak measured here by cuBLAS DGEMM
    f64 = [st for st in stats if st["name"].startswith("hop") and st["name"].endswith("_f64")]
    peak64 = fp64_peak_tflops()
    roofline_fp64 = None
    if f64 and peak64:
        fl, tm = sum(st["flops"] for st in f64), sum(st["ms"] for st in f64)
        ach = fl / (tm * 1e-3) / 1e12
        roofline_fp64 = {"kernels": [st["name"] for st in f64], "bound": "fp64_alu", "achieved": ach,
                         "peak": peak64, "unit": "TFLOP/s", "frac": ach / peak64,
                         "peak_source": "measured in this run: cuBLAS DGEMM 4096^3 through torch, best of 5",
                         "flops_model": "1320 per 5d site and hop + the s-operator and xpay terms",
                         "share_of_solve_kernel_time": tm / total_ms}
    kernels = [{"name": s["name"], "launches": s["launches"], "ms": round(s["ms"], 3),
                "share": round(s["ms"] / total_ms, 4),
                "GBps": round(s["bytes"] / (s["ms"] * 1e-3) / 1e9, 1) if s["ms"] > 0 else None}
               for s in sorted(stats, key=lambda s: -s["ms"])]

    # ---------------- end to end through the C ABI with host buffers (right after the timed
    # solves, with the context in the same state)
    e2e = None
    if not args.no_extras:
        e2e = end_to_end(args, h, b, inner, n5, flush, lambda: solve(inner))

    # ---------------- Dslash alone per precision (M applications on resident fields)
    dslash = {}
    precs = () if args.no_extras else (("f64", mdwf.MDWF_F64), ("f32", mdwf.MDWF_F32), ("f16n", mdwf.MDWF_F16N))
    x_, y_, z_, t_ = dims
    Vh = x_ * y_ * z_ * t_ // 2
    src_odd = torch.from_numpy(np.ascontiguousarray(
        b.reshape(Ls, -1, 4, 3)[:, :Vh])).cuda()   # any field of the right size
    for name, prec in precs:
        nbytes = mdwf.mdwf_field_bytes(h, prec, 1)
        fi = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        fo = torch.empty_like(fi)
        mdwf.mdwf_field_import(h, fi, src_odd, prec)
        reps = 4 if name == "f64" else 20
        for _ in range(3):
            mdwf.mdwf_apply(h, fo, fi, prec)
        torch.cuda.synchronize()
        mdwf.mdwf_profile_enable(h, True)
        mdwf.mdwf_profile_read(h, reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        e0.record()
        for _ in range(reps):
            mdwf.mdwf_apply(h, fo, fi, prec)
        e1.record()
        torch.cuda.synchronize()
        st = mdwf.mdwf_profile_read(h, reset=True)
        mdwf.mdwf_profile_enable(h, False)
        ms_apply = e0.elapsed_time(e1) / reps
        hop = [s for s in st if s["name"].startswith("hop")]
        hop_bytes = sum(s["bytes"] for s in hop) / reps
        dslash[name] = {"ms_per_M": ms_apply, "GFLOPs": FLOPS_PER_SITE * n5 / (ms_apply * 1e-3) / 1e9,
                        "GBps": hop_bytes / (ms_apply * 1e-3) / 1e9,
                        "hbm_frac": hop_bytes / (ms_apply * 1e-3) / 1e9 / hbm_peak,
                        "kernels": {s["name"]: round(1e3 * s["ms"] / s["launches"], 2) for s in st}}
        del fi, fo

    # ---------------- batching: M on 12 right-hand sides in one launch against 1 (FP32)
    batched = None
    if not args.no_extras:
        per_rhs = {}
        for nr in (1, 12):
            nbytes = mdwf.mdwf_field_bytes(h, mdwf.MDWF_F32, nr)
            fi = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            fo = torch.empty_like(fi)
            mdwf.mdwf_field_import(h, fi, src_odd.unsqueeze(0).expand(nr, *src_odd.shape).contiguous(),
                                   mdwf.MDWF_F32, nr)
            for _ in range(3):
                mdwf.mdwf_apply(h, fo, fi, mdwf.MDWF_F32, nr)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 10
            flush.zero_()
            e0.record()
            for _ in range(reps):
                mdwf.mdwf_apply(h, fo, fi, mdwf.MDWF_F32, nr)
            e1.record()
            torch.cuda.synchronize()
            per_rhs[nr] = e0.elapsed_time(e1) / reps / nr
            del fi, fo
        batched = {"prec": "f32", "nrhs": 12, "ms_per_M_per_rhs": per_rhs[12], "ms_per_M_nrhs1": per_rhs[1],
                   "GFLOPs": FLOPS_PER_SITE * n5 / (per_rhs[12] * 1e-3) / 1e9,
                   "speedup_per_rhs": per_rhs[1] / per_rhs[12]}

    # ---------------- time to solution: mixed (both inner precisions) and plain FP64
    cg = {"mixed_" + args.inner: {"ms": ms / args.steps, "iters": infos[-1].iters,
                                  "reliable_updates": infos[-1].reliable_updates,
                                  "true_res": infos[-1].true_res, "res_m": infos[-1].res_m}}
    other = "f16n" if args.inner == "f32" else "f32"
    legs = () if args.no_extras else ((f"mixed_{other}", mdwf.MDWF_F16N if other == "f16n" else mdwf.MDWF_F32),)
    legs += () if args.no_f64 else (("f64", mdwf.MDWF_F64),)
    for name, prec in legs:
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        inf = solve(prec)
        e1.record()
        torch.cuda.synchronize()
        cg[name] = {"ms": e0.elapsed_time(e1), "iters": inf.iters, "reliable_updates": inf.reliable_updates,
                    "true_res": inf.true_res, "res_m": inf.res_m}

    # ---------------- the same solve with per-slice (Zolotarev) b5(s), c5(s): dense s-operators
    if not args.no_extras:
        from paper_1206_5214_gb300 import zolotarev
        b5s, c5s = zolotarev.zolotarev_coefficients(Ls, *ZOLO_RANGE)
        mdwf.mdwf_set_s_coefficients(h, list(b5s), list(c5s))
        solve(inner)  # tables and graph
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        inf = solve(inner)
        e1.record()
        torch.cuda.synchronize()
        cg[f"mixed_{args.inner}_zolotarev"] = {
            "ms": e0.elapsed_time(e1), "iters": inf.iters, "reliable_updates": inf.reliable_updates,
            "true_res": inf.true_res, "ms_per_iter": e0.elapsed_time(e1) / max(inf.iters, 1),
            "lambda_range": list(ZOLO_RANGE)}
        mdwf.mdwf_set_s_coefficients(h, None, None)

    # ---------------- the constructions around the solve, mixed precision to 1e-10: D_ov(m) psi
    # (one Pauli-Villars solve, Sec. 2.2), the wall-pseudofermion action and its force (two
    # solves, Sec. 2.4), and the solve with a chemical potential on the time links (Sec. 6.6)
    around = None
    if not args.no_extras:
        around = {}
        psi4 = torch.from_numpy(np.ascontiguousarray(sy.gaussian_field(dims, 1, OVERLAP_SEED)[0])).cuda()
        out4 = torch.empty_like(psi4)
        G4 = torch.empty(U.shape, dtype=torch.complex128, device="cuda")

        def timed(fn):
            fn()  # warm-up
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            r = fn()
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1), r

        ms, (st, infs) = timed(lambda: mdwf.mdwf_overlap_apply(h, out4, psi4, tol=1e-10, inner_prec=inner))
        around["overlap_apply"] = {"ms": ms, "pv_iters": infs[0].iters, "status": st}
        ms, (S4, st, inf4) = timed(lambda: mdwf.mdwf_force4d(h, G4, psi4, tol=1e-10, inner_prec=inner))
        around["wall_force"] = {"ms": ms, "second_solve_iters": inf4.iters, "status": st}
        mdwf.mdwf_set_chemical_potential(h, CHEM_MU)
        ms, inf = timed(lambda: solve(inner))
        around["mixed_" + args.inner + "_chemical_potential"] = {
            "ms": ms, "mu": CHEM_MU, "iters": inf.iters, "reliable_updates": inf.reliable_updates,
            "true_res": inf.true_res}
        mdwf.mdwf_set_chemical_potential(h, 0.0)
        del psi4, out4, G4

    # ---------------- the force on the same lattice at mf = 0.02 (dS/dU, dS/db5, dS/dc5; one solve)
    force = None
    if not args.no_extras:
        # a Gaussian odd field (any field of the odd-field shape serves)
        phi = np.ascontiguousarray(sy.gaussian_field(dims, Ls, FORCE_SEED).reshape(Ls, -1, 4, 3)[:, :Vh])
        hf = mdwf.mdwf_create(dims, Ls, M5, B5, C5, FORCE_MF)
        mdwf.mdwf_load_gauge(hf, Ud)
        phid = torch.from_numpy(phi).cuda()
        G = torch.empty(U.shape, dtype=torch.complex128, device="cuda")
        mdwf.mdwf_force(hf, G, phid, tol=1e-10, inner_prec=inner)  # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        S, db5, dc5, fst, finfo = mdwf.mdwf_force(hf, G, phid, tol=1e-10, inner_prec=inner)
        e1.record()
        torch.cuda.synchronize()
        force = {"ms": e0.elapsed_time(e1), "mf": FORCE_MF, "tol": 1e-10, "inner": args.inner,
                 "iters": finfo.iters, "true_res": finfo.true_res, "status": fst}
        mdwf.mdwf_destroy(hf)
        del G, phid

    batched_solves = None
    if not args.no_extras and not args.no_batched and not args.quick:
        del flush
        torch.cuda.empty_cache()
        batched_solves = {name: batched_solve(name, cfg) for name, cfg in BATCHED.items()}

    cpu = None if args.no_cpu else cpu_baseline(dims, Ls)

    line = {"metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.inner == "f32" else "f16n",
            "data": "synthetic", "config": workload_config(args.inner),
            "gpu_launches": launches1 - launches0,
            "applies_per_step": applies / args.steps,
            "roofline": roofline, "roofline_iteration": roofline_iteration, "roofline_fp64": roofline_fp64,
            "clocks": clocks.summary(), "e2e": e2e, "cpu_baseline": cpu,
            "cgne": cg, "dslash": dslash, "batched_apply": batched, "batched_solves": batched_solves,
            "force": force, "around_the_solve": around,
            "kernels": kernels,
            "profiled_solve": {"iters": prof_info.iters, "true_res": prof_info.true_res}}
    print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    mdwf.mdwf_destroy(h)


def fp64_peak_tflops(n: int = 4096, reps: int = 5) -> float | None:
    """FP64 throughput of cuBLAS DGEMM (2 n^3 flops per product), best of reps."""
    import torch
    try:
        a = torch.randn(n, n, dtype=torch.float64, device="cuda")
        b = torch.randn(n, n, dtype=torch.float64, device="cuda")
        c = torch.matmul(a, b)
        best = None
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        del a, b, c
        return 2.0 * n ** 3 / (best * 1e-3) / 1e12
    except RuntimeError:
        return None


def batched_solve(name: str, cfg: dict) -> dict:
    """Time to solution of one batched workload: all right-hand sides in one solve
    (one launch per kernel over the batch), FP64 reliable updates, to a true FP64
    residual of 1e-10 per right-hand side; the wall time of the mdwf_cgne call,
    which synchronises. The sources and solutions are device buffers where they fit
    beside the solver's fields and host buffers otherwise (the library's copies are
    then inside the timed call). The plain FP64
    solve of the same batch would take minutes, so its time is extrapolated: the
    time per FP64 CG iteration (the difference of two capped FP64 solves of the
    whole batch, or of a quarter of it when the whole batch does not fit beside
    its workspace, then scaled by the batch size, since the FP64 operator is
    bound by the FP64 pipe and its time grows in proportion) times the
    iterations of the mixed solve, plus the capped solve's fixed costs."""
    import torch
    import paper_1206_5214_gb300 as mdwf
    import synthetic as sy
    dims, Ls, mf = cfg["dims"], cfg["Ls"], cfg["mf"]
    nrhs = len(mf)
    inner = mdwf.MDWF_F32 if cfg["inner"] == "f32" else mdwf.MDWF_F16N
    out = {"lattice": list(dims), "Ls": Ls, "nrhs": nrhs, "masses": mf, "b5": B5, "c5": C5, "M5": M5,
           "eps": cfg["eps"], "inner": cfg["inner"], "sources": cfg["sources"], "tol": 1e-10,
           "autotune": cfg["autotune"], "buffers": cfg["buffers"]}
    t0 = time.perf_counter()
    U = sy.gauge_field(dims, cfg["eps"], sy.config_seed("gauge", cfg["cfg"]))
    if cfg["sources"] == "point":
        b = sy.point_sources_device(dims, Ls)
    else:
        b = sy.gaussian_field_device(dims, Ls, sy.config_seed("source", cfg["cfg"]), nrhs)
    if cfg["buffers"] == "host":
        bh = torch.empty(b.shape, dtype=b.dtype)
        bh.copy_(b)
        del b
        torch.cuda.empty_cache()
        b = bh
    x = torch.zeros_like(b)
    out["input_setup_s"] = round(time.perf_counter() - t0, 1)
    Ud = torch.from_numpy(U).cuda()
    del U
    n5 = dims[0] * dims[1] * dims[2] * dims[3] // 2 * Ls

    def run(h, prec, maxiter, sub=None):
        bb, xx, mm = (b, x, mf) if sub is None else (b[:sub], x[:sub], mf[:sub])
        xx.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        st, info = mdwf.mdwf_cgne(h, xx, bb, nrhs=len(mm), mf_per_rhs=mm, tol=1e-10, inner_prec=prec,
                                  maxiter=maxiter, raise_on_error=False)
        torch.cuda.synchronize()
        return 1e3 * (time.perf_counter() - t), st, info

    h = mdwf.mdwf_create(dims, Ls, M5, B5, C5, mf[0], autotune=cfg["autotune"])
    try:
        mdwf.mdwf_load_gauge(h, Ud)
        run(h, inner, 16)  # warm-up: tables, autotuned tiles, the iteration's CUDA graph
        a0 = sum(mdwf.mdwf_counters(h)[1])
        ms, st, info = run(h, inner, 40000)
        a1 = sum(mdwf.mdwf_counters(h)[1])
    finally:
        mdwf.mdwf_destroy(h)
    iters = [i.iters for i in info]
    out["mixed"] = {"ms": ms, "status": st, "iters": iters, "reliable_updates": [i.reliable_updates for i in info],
                    "true_res": [i.true_res for i in info], "res_m": [i.res_m for i in info],
                    "GFLOPs": (a1 - a0) * nrhs * FLOPS_PER_SITE * n5 / (ms * 1e-3) / 1e9}
    # plain FP64: per-iteration time from two capped solves
    m1, m2 = 4, 12
    est = None
    for sub in (None, max(1, nrhs // 4)):
        h = mdwf.mdwf_create(dims, Ls, M5, B5, C5, mf[0])
        try:
            mdwf.mdwf_load_gauge(h, Ud)
            t1, s1, _ = run(h, mdwf.MDWF_F64, m1, sub)
            t2, s2, _ = run(h, mdwf.MDWF_F64, m2, sub)
        finally:
            mdwf.mdwf_destroy(h)
        if s1 in (0, 4) and s2 in (0, 4):  # MDWF_OK or MDWF_ENOCONV (capped)
            scale = nrhs / (sub or nrhs)
            per_iter = (t2 - t1) / (m2 - m1) * scale
            est = {"ms_per_iter": per_iter, "measured_nrhs": sub or nrhs, "capped_at": [m1, m2],
                   "capped_ms": [t1, t2], "iters_assumed": max(iters),
                   "ms_estimated": t1 * scale + per_iter * (max(iters) - m1)}
            break
        torch.cuda.empty_cache()
    out["f64_extrapolated"] = est
    if est:
        out["mixed_speedup_over_f64"] = est["ms_estimated"] / ms
    del b, x, Ud
    torch.cuda.empty_cache()
    return out


def end_to_end(args, h, b, inner, n5, flush, solve_device) -> dict:
    """The same solve through mdwf_cgne with pinned host buffers: H2D of b and D2H of x timed.
    Each step is followed by the device-buffer solve in the same state (not counted), whose
    wall time shows what the copies add."""
    import torch
    import paper_1206_5214_gb300 as mdwf
    bh = torch.from_numpy(b).pin_memory()
    xh = torch.zeros_like(bh).pin_memory()
    for _ in range(2):  # warm-up: the first transfers from freshly pinned pages are slower
        mdwf.mdwf_cgne(h, xh, bh, tol=1e-10, inner_prec=inner)
    e2e_times, dev_times = [], []
    applies = 0
    for _ in range(max(1, min(args.steps, 5))):
        flush.zero_()
        torch.cuda.synchronize()
        a0 = sum(mdwf.mdwf_counters(h)[1])
        t0 = time.perf_counter()
        mdwf.mdwf_cgne(h, xh, bh, tol=1e-10, inner_prec=inner)
        e2e_times.append(time.perf_counter() - t0)
        applies += sum(mdwf.mdwf_counters(h)[1]) - a0
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        solve_device()
        torch.cuda.synchronize()
        dev_times.append(time.perf_counter() - t0)
    e2e_flops = applies / len(e2e_times) * FLOPS_PER_SITE * n5
    e2e_s = sum(e2e_times) / len(e2e_times)
    bytes_field = b.nbytes
    return {"value": e2e_flops / e2e_s / 1e9, "unit": "GFLOP/s", "h2d_bytes_per_step": bytes_field,
            "d2h_bytes_per_step": bytes_field, "ms_per_step": 1e3 * e2e_s,
            "ms_each": [round(1e3 * t, 2) for t in e2e_times],
            "device_buffers_wall_ms_each": [round(1e3 * t, 2) for t in dev_times]}


if __name__ == "__main__":
    main()
