"""Benchmark of the hot path: mixed-precision even-odd CG solves of the Wilson
twisted-mass clover operator on a 24^3x64 lattice (the MILC12/RBC11 shape of
Table 1), to an FP64 true residual of 1e-10, on synthetic seeded fields.

One step = one complete solve (source preparation, mixed-precision CGNR with
FP64 reliable updates, reconstruction of the odd sites, FP64 true residual).
Printed as one JSON line (rank 0). Beside the headline solves/s it reports:
  * roofline: the dominant kernel's algorithmic HBM bytes per launch over its
    CUDA-event duration inside the timed region, against the measured copy peak;
  * fp64: the plain FP64 single-precision-free CGNR solver on the same system,
    and the speedup of the mixed solver over it;
  * e2e: the same solves through the C ABI with host buffers (pinned), copies
    included;
  * cpu_baseline: the FP64 CPU oracle on a bounded sample of the same workload;
  * clocks sampled with nvidia-smi during the timed region;
  * with --with-configs (default): the 36-RHS 32^3x96 workload, the 48^3x144 HISQ
    multi-shift workload and a short serving trace (p50/p99 latency, solves/s).
--impl reference times the oracle itself (the reference arm).
Multi-GPU (torchrun): every rank runs independent replicas of the same solve.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import signal
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = (24, 24, 24, 64)
C_SW, MASS, MU = 1.05, 0.05, 0.01
GAUGE_SEED, SOURCE_SEED = 102, 202
TOL = 1e-10
METRIC = "mixed-precision CG solves/s at true residual 1e-10 (Wilson twisted-mass clover 24^3x64, even-odd)"
WORKLOAD = "wilson_tm_clover_24x24x24x64_eo_mixed_cg"

# Algorithmic bytes per output site of the hopping kernels (compulsory traffic, one pass):
#   spinor in (neighbours counted once) + 8 links + epilogue operands + spinor out.
#   FP16 spinor = 24 x 2 B + 4 B norm = 52 B; FP32 spinor 96 B; FP64 192 B. A link is
#   `recon` reals (18 / 12 / 8) of 2 / 4 B; the FP64 kernels always read R18 (144 B).
#   AINV epilogue reads A^{-1} (144 reals + FP16 norm); XPAY reads the clover (72 reals
#   + FP16 norm) and y.
KERNELS = ["wilson_dslash_f16_ainv", "wilson_dslash_f16_xpay", "wilson_dslash_f32_ainv", "wilson_dslash_f32_xpay",
           "wilson_dslash_f64_ainv", "wilson_dslash_f64_xpay"]
_SPINOR = {"f16": 52, "f32": 96, "f64": 192}
_REAL = {"f16": 2, "f32": 4, "f64": 8}


def bytes_per_site(name, recon=12):
    prec, epi = name.split("_")[2:4]
    sp, rb = _SPINOR[prec], _REAL[prec]
    link = rb * (18 if prec == "f64" else recon)
    norm = 4 if prec == "f16" else 0
    if epi == "ainv":
        return sp + 8 * link + 144 * rb + norm + sp
    return sp + 8 * link + 72 * rb + norm + sp + sp


FLOPS_PER_SITE = {"hop": 1320, "ainv": 1320 + 2 * 6 * 6 * 8, "xpay": 1320 + 2 * 36 * 8 + 48}

# The sources of the FP16 Wilson kernels: an ncu traffic figure is used only while their
# hash is the one the capture was taken with.
KERNEL_SOURCES = ["core.cuh", "wilson.cuh", "wilson_x2.cuh", "dslash.cu", "dslash_launch.cuh"]


def kernel_source_hash():
    import hashlib
    h = hashlib.sha1()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2201_09004_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def ncu_traffic(kernel):
    """dram__bytes_read.sum + dram__bytes_write.sum per launch of `kernel` from a committed
    ncu summary (a line 'traffic: <kernel> <source hash> <bytes>' in profiles/*.md) taken
    with the current kernel sources; None if there is none."""
    import glob
    want = kernel_source_hash()
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for line in open(path):
            parts = line.strip().strip("`").split()
            if len(parts) == 4 and parts[0] == "traffic:" and parts[1] == kernel and parts[2] == want:
                return int(parts[3])
    return None

REASONS = {
    0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap", 0x8: "hw_slowdown",
    0x10: "sync_boost", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
    0x80: "hw_power_brake_slowdown", 0x100: "display_clock_setting",
}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6400.0)), "measured"
    return 6400.0, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    def __init__(self):
        self.proc = None
        self.path = None

    def start(self, index):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active"
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL,
                                         start_new_session=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        try:
            os.killpg(self.proc.pid, signal.SIGTERM)
        except OSError:
            pass
        self.proc.wait(timeout=10)
        sm, mx, reasons = [], 0.0, set()
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 5:
                continue
            try:
                s, m = float(parts[1]), float(parts[2])
                act = int(parts[4], 16) if parts[4].startswith("0x") else int(parts[4])
            except ValueError:
                continue
            sm.append(s)
            mx = max(mx, m)
            for bit, name in REASONS.items():
                if act & bit and name != "gpu_idle":
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- workload
def setup_gpu(dev):
    import torch
    from paper_2201_09004_b300 import lib, synth
    U = synth.thin_links(DIMS, GAUGE_SEED, device=dev)
    b = synth.z2_source(DIMS, SOURCE_SEED, device=dev)
    lat = lib.Lattice(DIMS, -1)
    lat.load_gauge(lib.THIN, U)
    lat.load_clover(C_SW)
    del U
    torch.cuda.synchronize()
    return lat, b


def job_rate(local_seconds, units_per_rank, world, device="cpu"):
    """Whole-job throughput of `world` replicas: every rank processed
    units_per_rank units; the job took the slowest rank's time (max over ranks).
    Returns (units per second, max seconds)."""
    import torch
    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    s = float(t.item())
    return world * units_per_rank / s, s


def gpu_arm(args):
    import torch
    import torch.distributed as dist
    from paper_2201_09004_b300 import lib

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    lat, b = setup_gpu(dev)
    op = lib.op_params(lib.WILSON_TM_CLOVER, MASS, MU, c_sw=C_SW)
    sp = lib.solve_params(solver=lib.MIXED_CGNR, tol=TOL, delta=0.1, prec_sloppy=args.prec, recon_sloppy=args.recon,
                          graph_iters=args.graph_iters)
    stream = torch.cuda.current_stream()
    x = torch.empty_like(b)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        lat.solve(op, sp, [b], stream=stream, out=[x])
    barrier()
    sampler = ClockSampler()
    if rank == 0:
        sampler.start(local)
    lib.profile_enable(False)
    launches0 = lib.launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    infos, lat_ms = [], []
    barrier()
    ev0.record(stream)
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _, info = lat.solve(op, sp, [b], stream=stream, out=[x])
        lat_ms.append((time.perf_counter() - t0) * 1e3)
        infos.append(info[0])
    ev1.record(stream)
    barrier()
    launches = lib.launch_count() - launches0
    clocks = sampler.stop() if rank == 0 else None
    value, s_max = job_rate(ev0.elapsed_time(ev1) * 1e-3, args.steps, world, dev)
    ms_max = s_max * 1e3

    # second timed pass over the same steps with a CUDA event pair around every
    # launch of the library (on its stream): per-kernel times for the roofline
    lib.profile_reset()
    lib.profile_enable(True)
    ep0 = torch.cuda.Event(enable_timing=True)
    ep1 = torch.cuda.Event(enable_timing=True)
    barrier()
    ep0.record(stream)
    for _ in range(args.steps):
        lat.solve(op, sp, [b], stream=stream, out=[x])
    ep1.record(stream)
    barrier()
    lib.profile_enable(False)
    profiled_ms = ep0.elapsed_time(ep1) / args.steps

    # dominant kernel and its roofline, from the events recorded in the timed region
    kernels = {}
    for name in KERNELS:
        n, tot = lib.profile_query(name)
        if n:
            kernels[name] = (n, tot)
    all_n, all_t = lib.profile_query("")
    dom = max(kernels, key=lambda k: kernels[k][1])
    n, tot = kernels[dom]
    vh = int(np.prod(DIMS)) // 2
    avg_s = tot / n * 1e-3
    byts = bytes_per_site(dom, args.recon) * vh
    peak, peak_kind = measured_peaks()
    achieved = byts / avg_s / 1e9
    epi = dom.rsplit("_", 1)[1]
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_source": peak_kind, "frac_of_nominal_8tbs": round(achieved / 8000.0, 4),
                "algorithmic_bytes_per_launch": byts, "avg_launch_us": round(avg_s * 1e6, 2),
                "gflops": round(FLOPS_PER_SITE[epi] * vh / avg_s / 1e9, 1),
                "share_of_kernel_time": round(tot / all_t, 4),
                "traffic": ncu_traffic(dom) if args.recon == 12 else None, "kernel_source_hash": kernel_source_hash(),
                "pass": "second timed pass of the same steps with per-launch CUDA events",
                "profiled_ms_per_step": round(profiled_ms, 3)}
    per_kernel = {k: {"launches": v[0], "ms": round(v[1], 3),
                      "gbs": round(bytes_per_site(k, args.recon) * vh / (v[1] / v[0] * 1e-3) / 1e9, 1)} for k, v in kernels.items()}
    # device time per solve of every kernel family in the timed region
    breakdown = {}
    for name in ["wilson_dslash_f16", "wilson_dslash_f32x2", "wilson_dslash_f32_", "wilson_ainv_site", "blas_cg_s", "blas_cg_xp",
                 "blas_finalize", "blas_norm2", "blas_copy", "blas_axpy", "blas_xmy_norm", "blas_zero",
                 "import_field", "export_field"]:
        n_, t_ = lib.profile_query(name)
        if n_:
            breakdown[name] = {"launches_per_solve": round(n_ / args.steps, 1), "ms_per_solve": round(t_ / args.steps, 3)}
    breakdown["all_kernels_ms_per_solve"] = round(all_t / args.steps, 3)

    # plain FP64 CGNR on the same system (the comparator of the mixed solver)
    sp64 = lib.solve_params(solver=lib.CGNR, tol=TOL, prec_sloppy=lib.F64)
    fp64 = None
    if args.fp64_steps > 0:
        lat.solve(op, sp64, [b], stream=stream, out=[x])  # tunes the FP64 kernels
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        i64 = None
        for _ in range(args.fp64_steps):
            _, i64 = lat.solve(op, sp64, [b], stream=stream, out=[x])
        e1.record(stream)
        torch.cuda.synchronize()
        s64 = e0.elapsed_time(e1) * 1e-3 / args.fp64_steps
        fp64 = {"solves_per_s": round(1.0 / s64, 3), "iters": i64[0]["iters"],
                "true_rel_residual": i64[0]["true_rel_residual"], "speedup_mixed_over_fp64": round(value / world * s64, 2)}

    # mixed-precision BiCGStab directly on the Schur operator (the same system and tolerance)
    bicg = None
    if args.bicgstab_steps > 0:
        spb = lib.solve_params(solver=lib.BICGSTAB, tol=TOL, delta=0.1, prec_sloppy=args.prec,
                               recon_sloppy=args.recon, graph_iters=args.graph_iters)
        lat.solve(op, spb, [b], stream=stream, out=[x])  # tunes the BiCGStab kernels
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ib = None
        for _ in range(args.bicgstab_steps):
            _, ib = lat.solve(op, spb, [b], stream=stream, out=[x])
        e1.record(stream)
        torch.cuda.synchronize()
        sb = e0.elapsed_time(e1) * 1e-3 / args.bicgstab_steps
        bicg = {"solves_per_s": round(1.0 / sb, 3), "iters": ib[0]["iters"],
                "reliable_updates": ib[0]["reliable_updates"], "operator_applications": ib[0]["operator_applications"],
                "true_rel_residual": ib[0]["true_rel_residual"], "speedup_over_mixed_cgnr": round(1.0 / (sb * value / world), 2)}

    # mixed-precision restarted GCR directly on the Schur operator (same system and tolerance)
    gcr = None
    if args.gcr_steps > 0:
        spg = lib.solve_params(solver=lib.GCR, tol=TOL, delta=0.1, prec_sloppy=args.prec, recon_sloppy=args.recon,
                               restart=args.gcr_restart)
        lat.solve(op, spg, [b], stream=stream, out=[x])
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ig = None
        for _ in range(args.gcr_steps):
            _, ig = lat.solve(op, spg, [b], stream=stream, out=[x])
        e1.record(stream)
        torch.cuda.synchronize()
        sg = e0.elapsed_time(e1) * 1e-3 / args.gcr_steps
        gcr = {"solves_per_s": round(1.0 / sg, 3), "iters": ig[0]["iters"], "restart": args.gcr_restart or 12,
               "defect_corrections": ig[0]["reliable_updates"], "operator_applications": ig[0]["operator_applications"],
               "true_rel_residual": ig[0]["true_rel_residual"], "speedup_over_mixed_cgnr": round(1.0 / (sg * value / world), 2)}

    # the same solve with the reliable updates below 1e-4 |bhat| in correction form with the
    # FP32 operator (update_f32_below; the final residual still recomputed from b)
    late_f32 = None
    if args.bicgstab_steps > 0:
        spc = lib.solve_params(solver=lib.MIXED_CGNR, tol=TOL, delta=0.1, prec_sloppy=args.prec,
                               recon_sloppy=args.recon, update_f32_below=1e-4)
        lat.solve(op, spc, [b], stream=stream, out=[x])
        torch.cuda.synchronize()
        lib.profile_reset()
        lib.profile_enable(True)
        lat.solve(op, spc, [b], stream=stream, out=[x])
        torch.cuda.synchronize()
        lib.profile_enable(False)
        n_df, t_df = lib.profile_query("wilson_dslash_f32x2")
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ic = None
        for _ in range(args.bicgstab_steps):
            _, ic = lat.solve(op, spc, [b], stream=stream, out=[x])
        e1.record(stream)
        torch.cuda.synchronize()
        sc_ = e0.elapsed_time(e1) * 1e-3 / args.bicgstab_steps
        late_f32 = {"solves_per_s": round(1.0 / sc_, 3), "update_f32_below": 1e-4, "iters": ic[0]["iters"],
                    "reliable_updates": ic[0]["reliable_updates"], "true_rel_residual": ic[0]["true_rel_residual"],
                    "double_float_operator": {"launches_per_solve": n_df, "ms_per_solve": round(t_df, 3)},
                    "speedup_over_mixed_cgnr": round(1.0 / (sc_ * value / world), 2)}

    # the same solve with its inner CG iterations in one persistent cooperative kernel
    # (k iterations per launch), against CUDA-graph replay of 1 and 4 iterations per graph
    persistent = None
    if args.persistent_steps > 0:
        def rate(spx, steps):
            lat.solve(op, spx, [b], stream=stream, out=[x])
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            inf = None
            for _ in range(steps):
                _, inf = lat.solve(op, spx, [b], stream=stream, out=[x])
            e1.record(stream)
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) * 1e-3 / steps
            return {"solves_per_s": round(1.0 / sec, 3), "iters": inf[0]["iters"],
                    "reliable_updates": inf[0]["reliable_updates"], "true_rel_residual": inf[0]["true_rel_residual"]}
        persistent = {}
        for k in (1, 4):
            persistent[f"persistent_{k}_iters_per_launch"] = rate(
                lib.solve_params(solver=lib.MIXED_CGNR, tol=TOL, delta=0.1, prec_sloppy=args.prec,
                                 recon_sloppy=args.recon, persistent=k), args.persistent_steps)
            persistent[f"graph_{k}_iters_per_graph"] = rate(
                lib.solve_params(solver=lib.MIXED_CGNR, tol=TOL, delta=0.1, prec_sloppy=args.prec,
                                 recon_sloppy=args.recon, graph_iters=k), args.persistent_steps)

    # end to end through the C ABI with pinned host buffers
    bh = b.cpu().pin_memory()
    xh = torch.empty_like(bh).pin_memory()
    lat.solve(op, sp, [bh], out=[xh])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        lat.solve(op, sp, [bh], out=[xh])
    e2e_rate, _ = job_rate(time.perf_counter() - t0, args.steps, world, dev)
    e2e = {"value": round(e2e_rate, 3), "unit": "solves/s",
           "h2d_bytes_per_step": int(bh.numel() * 16), "d2h_bytes_per_step": int(xh.numel() * 16)}

    if rank == 0:
        iters = [i["iters"] for i in infos]
        res = max(i["true_rel_residual"] for i in infos)
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {0: "f64", 1: "f32", 2: "f16-storage/f32"}[args.prec],
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "dims": list(DIMS), "action": "wilson twisted-mass clover",
                       "c_sw": C_SW, "m": MASS, "mu": MU, "gauge_seed": GAUGE_SEED, "source_seed": SOURCE_SEED,
                       "tol": TOL, "sloppy_precision": args.prec, "recon": args.recon, "delta": 0.1,
                       "graph_iters": args.graph_iters,
                       "parallelism": f"replicas{world}",
                       "l2": "inputs larger than L2 (clover inverse, clover and links ~0.3 GB per step)"},
            "iters": int(np.median(iters)), "reliable_updates": infos[-1]["reliable_updates"],
            "true_rel_residual_max": res,
            "latency_ms": {"p50": round(float(np.percentile(lat_ms, 50)), 3),
                           "p99": round(float(np.percentile(lat_ms, 99)), 3)},
            "roofline": roofline, "kernels": per_kernel, "time_breakdown": breakdown, "fp64": fp64,
            "bicgstab": bicg, "gcr": gcr, "persistent": persistent, "late_updates_f32": late_f32, "e2e": e2e,
            "gpu_launches": int(launches), "clocks": clocks,
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline()
        # the other single-GPU configurations, measured in the same run: 36 right-hand
        # sides at 32^3x96 (multi-RHS kernels, mixed CGNR) and the 48^3x144 HISQ multi-shift
        if args.with_configs and world == 1:
            lat.close()
            del b, x
            torch.cuda.empty_cache()
            line["multirhs_32x32x32x96"] = run_multirhs(args)
            line["hisq_48x48x48x144"] = run_hisq(args)
            if args.serving_requests > 0:  # the serving pattern's p50/p99 on a short Poisson trace
                sargs = argparse.Namespace(**{**vars(args), "requests": args.serving_requests, "fifo_requests": 0})
                line["serving_sample"] = run_serving(sargs)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


# ------------------------------------------------------- other workloads
def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _kernel_table(names, vh, bytes_per_site):
    from paper_2201_09004_b300 import lib
    out = {}
    for name in names:
        n, tot = lib.profile_query(name)
        if n:
            us = tot / n * 1e3
            out[name] = {"launches": n, "ms": round(tot, 3), "avg_us": round(us, 2)}
            if name in bytes_per_site:
                out[name]["gbs"] = round(bytes_per_site[name] * vh / (us * 1e-6) / 1e9, 1)
    return out


def run_multirhs(args):
    """32^3x96 twisted-mass clover (c_sw 1.04, m 0.04): 12 spin-colour point sources at a
    seeded site x 3 twisted masses = 36 right-hand sides, solved 12 at a time (one mass
    per call) through the fused multi-right-hand-side kernels, mixed precision to 1e-10.
    Compared with the plain FP64 single-right-hand-side solver (timed on one source
    and scaled to 36)."""
    import torch
    from paper_2201_09004_b300 import lib, synth
    dims, csw, m, mus = (32, 32, 32, 96), 1.04, 0.04, [0.004, 0.008, 0.016]
    torch.cuda.set_device(0)
    U = synth.thin_links(dims, 103, device="cuda")
    lat = lib.Lattice(dims)
    lat.load_gauge(lib.THIN, U)
    lat.load_clover(csw)
    del U
    site = synth.seeded_site(dims, 303)
    srcs = [synth.point_source(dims, site, sp, c, device="cuda") for sp in range(4) for c in range(3)]
    xs = [torch.empty_like(srcs[0]) for _ in srcs]
    tp0 = time.perf_counter()
    sp = lib.solve_params(solver=lib.MIXED_CGNR, tol=TOL, prec_sloppy=args.prec, recon_sloppy=args.recon)
    ops = [lib.op_params(lib.WILSON_TM_CLOVER, m, mu, c_sw=csw) for mu in mus]
    for op in ops:  # warm-up: clover inverses per mass, tuning of the NB = 4 kernels
        lat.solve(op, sp, srcs[:4], out=xs[:4])
    torch.cuda.synchronize()
    lib.profile_reset()
    lib.profile_enable(True)
    e0, e1 = _events()
    e0.record()
    infos = []
    for op in ops:
        _, inf = lat.solve(op, sp, srcs, out=xs)
        infos += inf
    e1.record()
    torch.cuda.synchronize()
    lib.profile_enable(False)
    tts = e0.elapsed_time(e1) * 1e-3
    vh = int(np.prod(dims)) // 2
    # algorithmic bytes per site of one launch over the 12 right-hand sides of a call: the
    # spinors per right-hand side, the links and the clover (inverse) record once per group
    # of 4 right-hand sides (the threads of one site; the 3 groups meet them in L2 at best)
    n = len(srcs)
    groups = (n + 3) // 4
    bps = {"wilson_dslash_f16_ainv": n * 52 + groups * (8 * 24 + (144 * 2 + 4)) + n * 52,
           "wilson_dslash_f16_xpay": n * 52 + groups * (8 * 24 + (72 * 2 + 4)) + n * 52 + n * 52}
    kern = _kernel_table(list(bps) + ["wilson_dslash_f32x2_ainv", "wilson_dslash_f32x2_xpay"], vh, bps)
    for k in ("wilson_dslash_f16_ainv", "wilson_dslash_f16_xpay"):
        if k in kern:
            kern[k]["gbs_per_rhs"] = round(kern[k]["gbs"] / n, 1)
    # the batching gain alone: the same mixed-precision solver one right-hand side per call
    single = []
    for op in ops:
        lat.solve(op, sp, [srcs[0]], out=[xs[0]])  # tunes the single-RHS kernels of this mass
        torch.cuda.synchronize()
        e0, e1 = _events()
        e0.record()
        for j in range(2):
            _, inf = lat.solve(op, sp, [srcs[4 * j + 1]], out=[xs[0]])
        e1.record()
        torch.cuda.synchronize()
        single.append(e0.elapsed_time(e1) * 1e-3 / 2)
    t_single36 = 12 * sum(single)
    # device time per right-hand side of each kernel family, batched (12 per call) and single
    families = ["wilson_dslash_f16", "wilson_dslash_f32x2", "blas_cg_s", "blas_cg_xp", "blas_finalize", "blas_",
                "import_field", "export_field", "wilson_ainv_site"]
    per_rhs = {"batched_12": {}, "single": {}}
    for f in families:
        n_, t_ = lib.profile_query(f)
        if n_:
            per_rhs["batched_12"][f] = round(t_ / 36, 3)
    lib.profile_reset()
    lib.profile_enable(True)
    _, inf1 = lat.solve(ops[1], sp, [srcs[2]], out=[xs[0]])
    torch.cuda.synchronize()
    lib.profile_enable(False)
    for f in families:
        n_, t_ = lib.profile_query(f)
        if n_:
            per_rhs["single"][f] = round(t_, 3)
    per_rhs["note"] = "ms of device time per right-hand side (profiled; 'blas_' is every BLAS kernel)"
    per_rhs["single_iters"] = inf1[0]["iters"]
    # the same 36 right-hand sides with mixed-precision BiCGStab on the Schur operator
    spb = lib.solve_params(solver=lib.BICGSTAB, tol=TOL, prec_sloppy=args.prec, recon_sloppy=args.recon)
    lat.solve(ops[0], spb, srcs[:4], out=xs[:4])
    torch.cuda.synchronize()
    e0, e1 = _events()
    e0.record()
    binfos = []
    for op in ops:
        _, inf = lat.solve(op, spb, srcs, out=xs)
        binfos += inf
    e1.record()
    torch.cuda.synchronize()
    tts_b = e0.elapsed_time(e1) * 1e-3
    sp64 = lib.solve_params(solver=lib.CGNR, tol=TOL, prec_sloppy=lib.F64)
    e0, e1 = _events()
    e0.record()
    _, i64 = lat.solve(ops[1], sp64, [srcs[0]], out=[xs[0]])
    e1.record()
    torch.cuda.synchronize()
    t64 = e0.elapsed_time(e1) * 1e-3
    line = {"workload": "multirhs", "metric": "time to solution of 36 right-hand sides at true residual 1e-10",
            "value": round(tts, 3), "unit": "s", "higher_is_better": False,
            "config": {"dims": list(dims), "c_sw": csw, "m": m, "mus": mus, "nrhs": 36, "site": list(site),
                       "sloppy_precision": args.prec, "recon": args.recon, "rhs_per_call": 12},
            "iters_max": max(i["iters"] for i in infos),
            "true_rel_residual_max": max(i["true_rel_residual"] for i in infos),
            "all_converged": all(i["status"] == 0 for i in infos),
            "fp64_single_rhs": {"seconds_per_solve": round(t64, 3), "iters": i64[0]["iters"],
                                "seconds_for_36_extrapolated": round(36 * t64, 3)},
            "speedup_vs_fp64_single_rhs": round(36 * t64 / tts, 2),
            "mixed_single_rhs": {"seconds_per_solve_per_mass": [round(t, 4) for t in single],
                                 "seconds_for_36_extrapolated": round(t_single36, 3),
                                 "sample": "2 point sources per mass, one per call, times 12"},
            "batching_gain_vs_mixed_single_rhs": round(t_single36 / tts, 2),
            "device_ms_per_rhs": per_rhs,
            "wall_seconds_incl_setup": round(time.perf_counter() - tp0, 1),
            "bicgstab": {"seconds": round(tts_b, 3), "iters_max": max(i["iters"] for i in binfos),
                         "true_rel_residual_max": max(i["true_rel_residual"] for i in binfos),
                         "all_converged": all(i["status"] == 0 for i in binfos),
                         "speedup_vs_fp64_single_rhs": round(36 * t64 / tts_b, 2)},
            "kernels": kern}
    lat.close()
    torch.cuda.empty_cache()
    return line


def run_delta(args):
    """The reliable-update threshold delta against the sloppy precision on the headline
    system (24^3x64 twisted-mass clover, mixed CGNR to 1e-10): iterations, reliable
    updates, time to solution and the device time of the double-float operator, per
    (delta, precision) pair."""
    import torch
    from paper_2201_09004_b300 import lib
    torch.cuda.set_device(0)
    lat, b = setup_gpu("cuda")
    op = lib.op_params(lib.WILSON_TM_CLOVER, MASS, MU, c_sw=C_SW)
    x = torch.empty_like(b)
    rows = []
    for prec in (lib.F16, lib.F32):
        for delta in (0.1, 0.05, 0.02, 0.01):
            sp = lib.solve_params(solver=lib.MIXED_CGNR, tol=TOL, delta=delta, prec_sloppy=prec, recon_sloppy=12)
            lat.solve(op, sp, [b], out=[x])
            torch.cuda.synchronize()
            lib.profile_reset()
            lib.profile_enable(True)
            e0, e1 = _events()
            e0.record()
            reps = 3
            for _ in range(reps):
                _, inf = lat.solve(op, sp, [b], out=[x])
            e1.record()
            torch.cuda.synchronize()
            lib.profile_enable(False)
            n_df, t_df = lib.profile_query("wilson_dslash_f32x2")
            rows.append({"sloppy": {lib.F16: "f16", lib.F32: "f32"}[prec], "delta": delta,
                         "iters": inf[0]["iters"], "reliable_updates": inf[0]["reliable_updates"],
                         "ms_per_solve": round(e0.elapsed_time(e1) / reps, 2),
                         "double_float_operator_ms_per_solve": round(t_df / reps, 2),
                         "true_rel_residual": inf[0]["true_rel_residual"]})
    line = {"workload": "delta", "metric": "mixed CGNR against the reliable-update threshold and sloppy precision",
            "config": {"dims": list(DIMS), "tol": TOL, "note": "timed with per-launch events (profiling on)"},
            "rows": rows}
    print(json.dumps(line), flush=True)


def run_dslash(args):
    """The operator kernels alone on resident fields (24^3x64, one output parity per
    launch): FP16 / FP32 hopping term, the FP16 A^-1 D and A y - D kernels of the
    Schur operator, and the HISQ FP16 hopping term on the same volume, each with R12
    and with R8 links (thin Wilson / long HISQ links); the 12-right-hand-side Schur
    operator; the FP16 hop and Schur operator on 32^3x96. L2 is flushed
    (a 256 MB write, then a 256 MB read) before every timed launch; each launch is timed alone with CUDA
    events on its stream. Reports algorithmic GB/s against the measured copy peak
    and the nominal 8 TB/s."""
    import torch
    from paper_2201_09004_b300 import lib, synth
    torch.cuda.set_device(0)
    dims = DIMS
    vh = int(np.prod(dims)) // 2
    U = synth.thin_links(dims, GAUGE_SEED, device="cuda")
    lat = lib.Lattice(dims)
    lat.load_gauge(lib.THIN, U)
    lat.load_clover(C_SW)
    del U
    V = synth.fat_links(dims, 104, device="cuda")
    lat.load_gauge(lib.FAT, V)
    del V
    W = synth.long_links(dims, 105, device="cuda")
    lat.load_gauge(lib.LONG, W)
    del W
    # L2 flush before every timed launch: a 256 MB write, then a 256 MB read of another
    # buffer, which evicts the write's dirty lines so that their write-back to HBM does
    # not fall into the timed launch
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    clean = torch.ones(256 << 20, dtype=torch.uint8, device="cuda")
    peak, peak_kind = measured_peaks()
    stream = torch.cuda.current_stream()
    reps = max(args.steps, 10)

    def timed(fn):
        fn()
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            flush.zero_()
            clean.sum(dtype=torch.int32)
            e0, e1 = _events()
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e3)
        return float(np.median(ts))

    out = {}
    psi = synth.gaussian_field(dims, 206, device="cuda")
    chi = synth.gaussian_field(dims, 207, ncomp=3, device="cuda")
    cases = []
    for r in (12, 8):
        cases += [(f"wilson_hop_f16_r{r}", lib.F16, 52 + 8 * 2 * r + 52, "hop", r),
                  (f"wilson_hop_f32_r{r}", lib.F32, 96 + 8 * 4 * r + 96, "hop", r),
                  (f"wilson_schur_f16_r{r} (A^-1 D + A y - D)", lib.F16,
                   (52 + 8 * 2 * r + 292 + 52) + (52 + 8 * 2 * r + 148 + 52 + 52), "schur", r),
                  (f"hisq_hop_f16_long_r{r}", lib.F16, 16 + 8 * 36 + 8 * 2 * r + 16, "hisq", r)]
    for name, prec, bps, kind, r in cases:
        opw = lib.op_params(lib.WILSON_TM_CLOVER, MASS, MU, c_sw=C_SW, recon=r)
        oph = lib.op_params(lib.HISQ, 0.01, recon=r)
        if kind == "hisq":
            fi = lib.Field(lat, lib.STAGGERED_FIELD, prec)
            fo = lib.Field(lat, lib.STAGGERED_FIELD, prec)
            fi.load(0, 1, chi)
            us = timed(lambda: lib.dslash_field(lat, oph, 0, fi, fo, stream=stream))
            launches = 1
        else:
            fi = lib.Field(lat, lib.WILSON_FIELD, prec)
            fo = lib.Field(lat, lib.WILSON_FIELD, prec)
            if kind == "hop":
                fi.load(0, 1, psi)
                us = timed(lambda: lib.dslash_field(lat, opw, 0, fi, fo, stream=stream))
                launches = 1
            else:
                ft = lib.Field(lat, lib.WILSON_FIELD, prec)
                fi.load(0, 0, psi)
                us = timed(lambda: lib.schur_field(lat, opw, fi, fo, ft, stream=stream))
                launches = 2
        gbs = bps * vh / (us * 1e-6) / 1e9
        out[name] = {"us": round(us, 2), "launches": launches, "bytes_per_site": bps, "GB_s": round(gbs, 1),
                     "frac_of_measured": round(gbs / peak, 4), "frac_of_nominal_8tbs": round(gbs / 8000.0, 4)}
    # the fused multi-right-hand-side kernels: the Schur operator on 12 right-hand sides in
    # one call (three groups of four threads per site); the algorithmic bytes count the
    # spinors per right-hand side and the links and clover records once per group
    nr = 12
    opw = lib.op_params(lib.WILSON_TM_CLOVER, MASS, MU, c_sw=C_SW, recon=12)
    fi, fo, ft = (lib.Field(lat, lib.WILSON_FIELD, lib.F16, nr) for _ in range(3))
    for k in range(nr):
        fi.load(k, 0, synth.gaussian_field(dims, 220 + k, device="cuda"))
    us = timed(lambda: lib.schur_field(lat, opw, fi, fo, ft, stream=stream))
    groups = (nr + 3) // 4
    bps = nr * (52 + 52 + 52 + 52 + 52) + groups * ((8 * 24 + 292) + (8 * 24 + 148))
    gbs = bps * vh / (us * 1e-6) / 1e9
    single = out["wilson_schur_f16_r12 (A^-1 D + A y - D)"]["us"]
    out["wilson_schur_f16_r12_12rhs (A^-1 D + A y - D, 3 groups of 4 per site)"] = {
        "us": round(us, 2), "us_per_rhs": round(us / nr, 2), "launches": 2, "bytes_per_site": bps,
        "GB_s": round(gbs, 1), "frac_of_measured": round(gbs / peak, 4),
        "per_rhs_speedup_over_single_rhs": round(single / (us / nr), 3)}
    del fi, fo, ft
    # the same FP16 kernels on the multi-right-hand-side workload's 32^3x96 lattice
    # (3.5x the sites: launch tails and block start-up weigh less)
    dims2 = (32, 32, 32, 96)
    vh2 = int(np.prod(dims2)) // 2
    U2 = synth.thin_links(dims2, 103, device="cuda")
    lat2 = lib.Lattice(dims2)
    lat2.load_gauge(lib.THIN, U2)
    lat2.load_clover(1.04)
    del U2
    op2 = lib.op_params(lib.WILSON_TM_CLOVER, 0.04, 0.008, c_sw=1.04, recon=12)
    psi2 = synth.gaussian_field(dims2, 230, device="cuda")
    fi, fo, ft = (lib.Field(lat2, lib.WILSON_FIELD, lib.F16) for _ in range(3))
    for name, kind, bps in (("wilson_hop_f16_r12_32x32x32x96", "hop", 296),
                            ("wilson_schur_f16_r12_32x32x32x96 (A^-1 D + A y - D)", "schur", 1084)):
        if kind == "hop":
            fi.load(0, 1, psi2)
            us = timed(lambda: lib.dslash_field(lat2, op2, 0, fi, fo, stream=stream))
        else:
            fi.load(0, 0, psi2)
            us = timed(lambda: lib.schur_field(lat2, op2, fi, fo, ft, stream=stream))
        gbs = bps * vh2 / (us * 1e-6) / 1e9
        out[name] = {"us": round(us, 2), "launches": 1 if kind == "hop" else 2, "bytes_per_site": bps,
                     "GB_s": round(gbs, 1), "frac_of_measured": round(gbs / peak, 4),
                     "frac_of_nominal_8tbs": round(gbs / 8000.0, 4)}
    del fi, fo, ft, psi2
    lat2.close()
    line = {"workload": "dslash", "metric": "Dslash HBM GB/s vs roofline (algorithmic bytes, L2 flushed)",
            "config": {"dims": list(dims), "sites_per_parity": vh, "peak_gbs": peak, "peak_source": peak_kind,
                       "reps": reps, "l2": "flushed (256 MB write, then 256 MB read) before every timed launch"},
            "kernels": out}
    print(json.dumps(line), flush=True)


def run_hisq(args):
    """48^3x144 HISQ (fat + long links), multi-shift CG over m in {0.002, 0.01, 0.02, 0.05},
    one Z2 source, mixed precision with double-float refinement to 1e-10 for every mass."""
    import torch
    from paper_2201_09004_b300 import lib, synth
    dims, masses = (48, 48, 48, 144), [0.002, 0.01, 0.02, 0.05]
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    lat = lib.Lattice(dims)
    V = synth.fat_links(dims, 104, device="cuda")
    lat.load_gauge(lib.FAT, V)
    del V
    W = synth.long_links(dims, 105, device="cuda")
    lat.load_gauge(lib.LONG, W)
    del W
    torch.cuda.empty_cache()
    b = synth.z2_source(dims, 204, ncomp=3, device="cuda")
    gen_s = time.perf_counter() - t0
    xs = [torch.empty_like(b) for _ in masses]
    op = lib.op_params(lib.HISQ, masses[0])
    sp = lib.solve_params(solver=lib.MULTISHIFT_CG, tol=TOL, prec_sloppy=args.prec, recon_sloppy=args.recon,
                          masses=masses)
    # warm-up on a lattice of the same volume is the solve itself; tune with a short solve
    lat.solve(op, lib.solve_params(solver=lib.MULTISHIFT_CG, tol=1e-3, prec_sloppy=args.prec,
                                   recon_sloppy=args.recon, masses=masses), [b], out=xs, check=False)
    torch.cuda.synchronize()
    # the multi-shift stage alone (its sloppy tolerance is ~1e-3 in FP16, so a 1e-3 solve
    # adds almost no refinement): the time split between the stages of the full solve
    e0, e1 = _events()
    e0.record()
    _, info_ms = lat.solve(op, lib.solve_params(solver=lib.MULTISHIFT_CG, tol=1e-3, prec_sloppy=args.prec,
                                                recon_sloppy=args.recon, masses=masses), [b], out=xs, check=False)
    e1.record()
    torch.cuda.synchronize()
    ms_stage = {"seconds": round(e0.elapsed_time(e1) * 1e-3, 3), "iters": info_ms[0]["iters"]}
    lib.profile_reset()
    lib.profile_enable(True)
    e0, e1 = _events()
    e0.record()
    _, info = lat.solve(op, sp, [b], out=xs)
    e1.record()
    torch.cuda.synchronize()
    lib.profile_enable(False)
    tts = e0.elapsed_time(e1) * 1e-3
    vh = int(np.prod(dims)) // 2
    # FP16: fat R18 (36 B), long R12 (24 B), colour vector 12 B + 4 B norm
    bps = {"hisq_dslash_f16_hop": 16 + 8 * 36 + 8 * 24 + 16, "hisq_dslash_f16_xpay": 16 + 8 * 36 + 8 * 24 + 16 + 16,
           "hisq_dslash_f32_hop": 24 + 8 * 72 + 8 * 48 + 24, "hisq_dslash_f32_xpay": 24 + 8 * 72 + 8 * 48 + 24 + 24}
    kern = _kernel_table(list(bps) + ["hisq_dslash_f32x2_hop", "hisq_dslash_f32x2_xpay"], vh, bps)
    line = {"workload": "hisq", "metric": "time to solution, multi-shift over 4 masses at true residual 1e-10",
            "value": round(tts, 3), "unit": "s", "higher_is_better": False,
            "config": {"dims": list(dims), "masses": masses, "c_naik": -1.0 / 24.0, "sloppy_precision": args.prec,
                       "recon_long": args.recon},
            "iters": info[0]["iters"], "reliable_updates": info[0]["reliable_updates"],
            "true_rel_residual_max_over_shifts": info[0]["true_rel_residual"], "status": info[0]["status"],
            "setup_seconds": round(gen_s, 1), "multishift_stage_to_1e-3": ms_stage, "kernels": kern}
    lat.close()
    del b, xs
    torch.cuda.empty_cache()
    return line


def run_hisq_propagator(args):
    """A HISQ 3-column propagator (the workload of the paper's HISQ timings, Sec. 2.2:
    24^3x64 with m = 0.0102): three colour point sources at one seeded site, solved
    together (one RHS per thread lane, shared link loads) by the mixed-precision CG
    to a true residual of 1e-10; compared with the same three solves one at a time
    in plain FP64 on the GPU."""
    import torch
    from paper_2201_09004_b300 import lib, synth
    dims, m = DIMS, 0.0102
    torch.cuda.set_device(0)
    lat = lib.Lattice(dims)
    V = synth.fat_links(dims, 104, device="cuda")
    lat.load_gauge(lib.FAT, V)
    del V
    W = synth.long_links(dims, 105, device="cuda")
    lat.load_gauge(lib.LONG, W)
    del W
    site = synth.seeded_site(dims, 304)
    srcs = [synth.point_source(dims, site, None, c, device="cuda") for c in range(3)]
    xs = [torch.empty_like(srcs[0]) for _ in srcs]
    op = lib.op_params(lib.HISQ, m)
    sp = lib.solve_params(solver=lib.MIXED_CGNR, tol=TOL, prec_sloppy=args.prec, recon_sloppy=args.recon)
    lat.solve(op, sp, srcs, out=xs)  # tunes
    torch.cuda.synchronize()
    e0, e1 = _events()
    e0.record()
    _, info = lat.solve(op, sp, srcs, out=xs)
    e1.record()
    torch.cuda.synchronize()
    tts = e0.elapsed_time(e1) * 1e-3
    sp64 = lib.solve_params(solver=lib.CGNR, tol=TOL, prec_sloppy=lib.F64)
    lat.solve(op, sp64, srcs[:1], out=xs[:1])
    torch.cuda.synchronize()
    e0, e1 = _events()
    e0.record()
    i64 = []
    for k in range(3):
        _, inf = lat.solve(op, sp64, srcs[k:k + 1], out=xs[k:k + 1])
        i64 += inf
    e1.record()
    torch.cuda.synchronize()
    t64 = e0.elapsed_time(e1) * 1e-3
    line = {"workload": "hisq_propagator", "metric": "time to solution of a HISQ 3-column propagator at true residual 1e-10",
            "value": round(tts, 3), "unit": "s", "higher_is_better": False,
            "config": {"dims": list(dims), "m": m, "c_naik": -1.0 / 24.0, "site": list(site), "nrhs": 3,
                       "sloppy_precision": args.prec, "recon_long": args.recon, "fat_seed": 104, "long_seed": 105},
            "iters_max": max(i["iters"] for i in info), "true_rel_residual_max": max(i["true_rel_residual"] for i in info),
            "all_converged": all(i["status"] == 0 for i in info),
            "fp64_one_at_a_time": {"seconds": round(t64, 3), "iters_max": max(i["iters"] for i in i64)},
            "speedup_vs_fp64": round(t64 / tts, 2),
            "paper_context": "17 s on 4 V100 (one node) for MILC12 24^3x64, m = 0.0102, residual not stated"}
    print(json.dumps(line), flush=True)


def run_twisted_multimass(args):
    """Twisted mass without clover on 24^3x64 (m = 0.05), one Z2 source and the three
    twisted masses of the multi-right-hand-side workload, mu in {0.004, 0.008, 0.016}:
    one multi-shift solve (full-lattice multi-shift CG on M0^+ M0 + mu^2, then a mixed
    CGNR refinement per mass) against three separate mixed CGNR solves."""
    import torch
    from paper_2201_09004_b300 import lib, synth
    torch.cuda.set_device(0)
    dims, m, mus = DIMS, MASS, [0.004, 0.008, 0.016]
    U = synth.thin_links(dims, GAUGE_SEED, device="cuda")
    lat = lib.Lattice(dims)
    lat.load_gauge(lib.THIN, U)
    del U
    b = synth.z2_source(dims, SOURCE_SEED, device="cuda")
    xs = [torch.empty_like(b) for _ in mus]
    op = lib.op_params(lib.WILSON_TM, m, mus[0])
    spm = lib.solve_params(solver=lib.MULTISHIFT_CG, tol=TOL, prec_sloppy=args.prec, recon_sloppy=args.recon,
                           masses=mus)
    lat.solve(op, spm, [b], out=xs)
    torch.cuda.synchronize()
    e0, e1 = _events()
    e0.record()
    _, info = lat.solve(op, spm, [b], out=xs)
    e1.record()
    torch.cuda.synchronize()
    t_ms = e0.elapsed_time(e1) * 1e-3
    sps = lib.solve_params(solver=lib.MIXED_CGNR, tol=TOL, prec_sloppy=args.prec, recon_sloppy=args.recon)
    e0, e1 = _events()
    e0.record()
    iters = []
    for i, mu in enumerate(mus):
        _, inf = lat.solve(lib.op_params(lib.WILSON_TM, m, mu), sps, [b], out=xs[i:i + 1])
        iters.append(inf[0]["iters"])
    e1.record()
    torch.cuda.synchronize()
    t_sep = e0.elapsed_time(e1) * 1e-3
    line = {"workload": "twisted_multimass", "metric": "time to solution of three twisted masses at true residual 1e-10",
            "value": round(t_ms, 3), "unit": "s", "higher_is_better": False,
            "config": {"dims": list(dims), "m": m, "mus": mus, "sloppy_precision": args.prec, "recon": args.recon,
                       "gauge_seed": GAUGE_SEED, "source_seed": SOURCE_SEED},
            "iters": info[0]["iters"], "true_rel_residual_max": info[0]["true_rel_residual"],
            "status": info[0]["status"],
            "separate_mixed_cgnr": {"seconds": round(t_sep, 3), "iters": iters},
            "speedup_vs_separate": round(t_sep / t_ms, 2)}
    print(json.dumps(line), flush=True)


def run_overlap(args):
    """Overlap building blocks on 24^3x64 (the RBC11 shape of the paper's overlap runs):
    50 applications of the fused g5 D_w(-rho), rho = 1.5, on the full lattice (the
    paper's Sec. 3 comparison: 0.025 s for 50 D_w with QUDA on one node of 4 V100),
    and one application of the Chebyshev/Clenshaw sign function eps(g5 D_w(-rho)) on
    the spectrum interval [0.1, 10.5] to a deviation of 1e-5 (the bound of the
    paper's Fig. 2), FP64 and double-float."""
    import torch
    from paper_2201_09004_b300 import lib, synth
    torch.cuda.set_device(0)
    dims, rho = DIMS, 1.5
    U = synth.thin_links(dims, GAUGE_SEED, device="cuda")
    lat = lib.Lattice(dims)
    lat.load_gauge(lib.THIN, U)
    del U
    v = synth.gaussian_field(dims, 208, device="cuda")
    out = {}
    vh = int(np.prod(dims)) // 2
    for name, prec in (("f64", lib.F64), ("f32x2", lib.F32X2), ("f32", lib.F32)):
        lat.gamma5_dw_apply(rho, v, prec=prec)
        torch.cuda.synchronize()
        e0, e1 = _events()
        e0.record()
        for _ in range(50):
            lat.gamma5_dw_apply(rho, v, prec=prec)
        e1.record()
        torch.cuda.synchronize()
        s50 = e0.elapsed_time(e1) * 1e-3
        out["g5dw_50_" + name] = round(s50, 4)
    # the device-resident kernel time of one full g5 D_w (both parities) inside the sign function
    lib.profile_reset()
    lib.profile_enable(True)
    res = {}
    for name, prec in (("f64", lib.F64), ("f32x2", lib.F32X2)):
        e0, e1 = _events()
        e0.record()
        _, info = lat.overlap_sign_apply(rho, 0.1, 10.5, 1e-5, v, prec=prec)
        e1.record()
        torch.cuda.synchronize()
        res[name] = {"seconds": round(e0.elapsed_time(e1) * 1e-3, 3), "order": info["order"],
                     "max_deviation": info["max_deviation"]}
    lib.profile_enable(False)
    kern = {}
    for name in ("wilson_dslash_f64_xpay", "wilson_dslash_f32x2_xpay"):
        n, t = lib.profile_query(name)
        if n:
            kern[name] = {"launches": n, "avg_us": round(t / n * 1e3, 2)}
    line = {"workload": "overlap", "metric": "g5 D_w(-rho) applications and the Chebyshev sign function, 24^3x64",
            "config": {"dims": list(dims), "rho": rho, "gauge_seed": GAUGE_SEED, "spectrum": [0.1, 10.5],
                       "deviation": 1e-5, "note": "seconds of 50 full-lattice applications include the host-array "
                                                  "copies of lq_gamma5_dw_apply; the kernel times are per parity"},
            "g5dw_50_applications_s": out, "sign_apply": res, "kernels": kern,
            "paper_context": "50 D_w on RBC11 24^3x64: 0.025 s (QUDA), 0.088 s (GWU-code), one node of 4 V100"}
    print(json.dumps(line), flush=True)


def run_eigen(args):
    """Low modes of H_w = g5 D_w(-rho), rho = 1.5, on --eig-dims (default 8^3x16;
    24^3x64 is the RBC11 shape of the paper's overlap runs, Sec. 2.3): the
    Chebyshev-filtered thick-restart Arnoldi eigensolver to |H_w z - lambda z| <= tol,
    then the sign function on one vector with those modes deflated against the same
    function without deflation (lambda_min below the lowest mode), both in
    double-float. On the synthetic near-unit fields the low spectrum is a dense band
    from |lambda| ~ 0.52 up; its density grows with the volume, so the filter edge
    and basis that resolve the lowest modes on 8^3x16 do not on 24^3x64."""
    import torch
    from paper_2201_09004_b300 import lib, synth
    torch.cuda.set_device(0)
    dims, rho, lmax = tuple(args.eig_dims), 1.5, 10.5
    U = synth.thin_links(dims, GAUGE_SEED, device="cuda")
    lat = lib.Lattice(dims)
    lat.load_gauge(lib.THIN, U)
    del U
    v = synth.gaussian_field(dims, 209, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev, Z, info = lat.hw_eigensolve(rho, args.nev, args.lambda_cut, lmax, tol=args.eig_tol, nkv=args.nkv,
                                    degree=args.degree, max_restarts=args.max_restarts, like=v, check=False)
    torch.cuda.synchronize()
    t_eig = time.perf_counter() - t0
    lmin_defl = float(np.max(np.abs(ev)))
    lmin_plain = 0.95 * float(np.min(np.abs(ev)))
    eig = {"converged": info["converged"], "restarts": info["restarts"],
           "hw_applications": info["operator_applications"], "max_residual": info["max_residual"],
           "wall_s": round(t_eig, 3), "abs_lambda_range": [float(np.min(np.abs(ev))), lmin_defl],
           "evals": [round(float(x), 10) for x in ev]}
    config = {"dims": list(dims), "rho": rho, "nev": args.nev, "nkv": args.nkv, "degree": args.degree,
              "lambda_cut": args.lambda_cut, "lambda_max": lmax, "tol": args.eig_tol,
              "gauge_seed": GAUGE_SEED, "precision": "double-float"}
    metric = "time to the nev lowest eigenpairs of g5 D_w(-rho), and the deflated sign function"
    if not info["converged"]:  # the deflated sign function needs converged eigenpairs
        print(json.dumps({"workload": "eigen", "metric": metric, "value": round(info["seconds"], 3), "unit": "s",
                          "higher_is_better": False, "config": config, "eigensolver": eig}), flush=True)
        return
    e0, e1 = _events()
    e0.record()
    sd, infod = lat.overlap_sign_apply_deflated(rho, lmin_defl, lmax, 1e-8, ev, Z, v)
    e1.record()
    torch.cuda.synchronize()
    t_defl = e0.elapsed_time(e1) * 1e-3
    # the same function without deflation must cover the lowest mode; a mode near zero
    # can make that polynomial longer than the library allows (65536 terms)
    try:
        e0, e1 = _events()
        e0.record()
        sp, infop = lat.overlap_sign_apply(rho, lmin_plain, lmax, 1e-8, v, prec=lib.F32X2)
        e1.record()
        torch.cuda.synchronize()
        plain = {"seconds": round(e0.elapsed_time(e1) * 1e-3, 3), "order": infop["order"], "lambda_min": lmin_plain}
        diff = float(torch.linalg.vector_norm(sd - sp) / torch.linalg.vector_norm(sp))
    except lib.LqError as e:
        plain = {"lambda_min": lmin_plain, "error": str(e)}
        diff = None
    line = {"workload": "eigen", "metric": metric,
            "value": round(info["seconds"], 3), "unit": "s", "higher_is_better": False,
            "config": config, "eigensolver": eig,
            "sign_function": {"deflated": {"seconds": round(t_defl, 3), "order": infod["order"],
                                           "lambda_min": lmin_defl},
                              "plain": plain, "relative_difference": diff, "deviation_bound": 1e-8}}
    print(json.dumps(line), flush=True)


def run_serving(args):
    """Poisson stream of solve requests (sizes 8^3x16, 16^3x32, 24^3x64, 32^3x64; twisted-mass
    clover with 12 point sources, or HISQ with one Z2 source; masses drawn from [0.005, 0.05];
    two gauge seeds per size cached on the device) through the continuous-batching server
    (mixed precision, 4 slots, HBM-budget admission), and the same trace through a FIFO
    one-at-a-time FP64 server. Rate = 0.8 x the mixed server's measured capacity."""
    import torch
    from paper_2201_09004_b300 import lib, synth
    torch.cuda.set_device(0)
    sizes = [(8, 8, 8, 16), (16, 16, 16, 32), (24, 24, 24, 64), (32, 32, 32, 64)]
    rng = np.random.default_rng(505)
    lats, srcs = {}, {}
    for si, d in enumerate(sizes):
        for g in range(2):
            lat = lib.Lattice(d)
            lat.load_gauge(lib.THIN, synth.thin_links(d, 600 + 10 * si + g, device="cuda"))
            lat.load_clover(1.05)
            lat.load_gauge(lib.FAT, synth.fat_links(d, 700 + 10 * si + g, device="cuda"))
            lat.load_gauge(lib.LONG, synth.long_links(d, 800 + 10 * si + g, device="cuda"))
            lats[(si, g)] = lat
        site = synth.seeded_site(d, 303)
        srcs[(si, "tmc")] = [synth.point_source(d, site, sp, c).numpy() for sp in range(4) for c in range(3)]
        srcs[(si, "hisq")] = [synth.z2_source(d, 204, ncomp=3).numpy()]
    torch.cuda.empty_cache()

    def make_requests(n):
        reqs = []
        for _ in range(n):
            si = int(rng.integers(0, len(sizes)))
            g = int(rng.integers(0, 2))
            kind = "tmc" if rng.random() < 0.5 else "hisq"
            mass = float(rng.uniform(0.005, 0.05))
            reqs.append((si, g, kind, mass))
        return reqs

    def params(kind, mass, fp64):
        if kind == "tmc":
            op = lib.op_params(lib.WILSON_TM_CLOVER, 0.05, mass, c_sw=1.05)
        else:
            op = lib.op_params(lib.HISQ, mass)
        if fp64:
            sp = lib.solve_params(solver=lib.CGNR, tol=TOL, prec_sloppy=lib.F64)
        else:
            sp = lib.solve_params(solver=lib.MIXED_CGNR, tol=TOL, prec_sloppy=lib.F16, recon_sloppy=args.recon)
        return op, sp

    def serve(reqs, arrivals, fp64, slots):
        srv = lib.Server(200 << 30, slots)
        t_start = time.perf_counter()
        outstanding, done = [], {}

        def collect(timeout_ms):
            # finished solutions are fetched (and dropped) as soon as they are ready, so the
            # server's host copies of large multi-RHS results never pile up
            for t in list(outstanding):
                if not srv.wait(t, timeout_ms):
                    continue
                _, info, times, code = srv.poll(t)
                done[t] = (times["finished"] - times["submitted"], code)
                outstanding.remove(t)

        tickets = []
        for (si, g, kind, mass), ta in zip(reqs, arrivals):
            while time.perf_counter() - t_start < ta:
                collect(0)
                time.sleep(0.0005)
            op, sp = params(kind, mass, fp64)
            t = srv.submit(lats[(si, g)], op, sp, srcs[(si, kind)])
            tickets.append(t)
            outstanding.append(t)
        while outstanding:
            collect(3600 * 1000)
        wall = time.perf_counter() - t_start
        srv.close()
        return (np.array([done[t][0] for t in tickets]), wall, [done[t][1] for t in tickets])

    def serve_fifo(reqs, arrivals):
        """The FP64 comparator: one request at a time in arrival order. Request i is
        submitted once it has arrived and request i-1 has finished (the queue waits
        on the client, so it holds no copies of sources in the server); its latency
        is that wait plus the server's submit-to-finish time."""
        srv = lib.Server(200 << 30, 1)
        t_start = time.perf_counter()
        lat_s, statuses = [], []
        for (si, g, kind, mass), ta in zip(reqs, arrivals):
            while time.perf_counter() - t_start < ta:
                time.sleep(0.0005)
            op, sp = params(kind, mass, True)
            queued = time.perf_counter() - t_start - ta
            t = srv.submit(lats[(si, g)], op, sp, srcs[(si, kind)])
            srv.wait(t, 3600 * 1000)
            _, info, times, code = srv.poll(t)
            lat_s.append(queued + times["finished"] - times["submitted"])
            statuses.append(code)
        wall = time.perf_counter() - t_start
        srv.close()
        return np.array(lat_s), wall, statuses

    # warm-up (tuning, clover inverses) on one request of every (size, kind)
    warm = [(si, 0, k, 0.02) for si in range(len(sizes)) for k in ("tmc", "hisq")]
    serve(warm, [0.0] * len(warm), False, 1)
    serve_fifo(warm[:2], [0.0] * 2)
    ms = lambda a, q: round(float(np.percentile(a, q)) * 1e3, 1)

    def summary(lat_s, wall, st, n):
        return {"p50_ms": ms(lat_s, 50), "p99_ms": ms(lat_s, 99), "solves_per_s": round(n / wall, 3),
                "all_ok": all(c == 0 for c in st)}

    # capacity of the mixed server: back-to-back service of a calibration batch
    calib = make_requests(16)
    _, wall_c, _ = serve(calib, [0.0] * len(calib), False, 4)
    capacity = len(calib) / wall_c
    rate = 0.8 * capacity
    reqs = make_requests(args.requests)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=len(reqs)))
    arrivals -= arrivals[0]
    lat_mixed, wall_mixed, st_mixed = serve(reqs, arrivals, False, 4)
    line = {"workload": "serving", "metric": "p50/p99 request latency and solves/s on a Poisson trace",
            "requests": len(reqs), "rate_per_s": round(rate, 3), "capacity_calibration_per_s": round(capacity, 3),
            "mixed_continuous_batching": dict(summary(lat_mixed, wall_mixed, st_mixed, len(reqs)), slots=4),
            "config": {"sizes": [list(d) for d in sizes], "actions": ["wilson_tm_clover 12 rhs", "hisq 1 rhs"],
                       "mass_range": [0.005, 0.05], "gauge_seeds_per_size": 2, "tol": TOL, "trace_seed": 505}}
    # both servers on one trace at a rate the FIFO FP64 server sustains (0.8 x its own
    # measured capacity), so that its latencies measure solves rather than an ever-growing queue
    if args.fifo_requests > 0:
        calib_f = make_requests(6)
        t0 = time.perf_counter()
        serve_fifo(calib_f, [0.0] * len(calib_f))
        cap_f = len(calib_f) / (time.perf_counter() - t0)
        rate_f = 0.8 * cap_f
        reqs_f = make_requests(args.fifo_requests)
        arr_f = np.cumsum(rng.exponential(1.0 / rate_f, size=len(reqs_f)))
        arr_f -= arr_f[0]
        lm, wm, sm = serve(reqs_f, arr_f, False, 4)
        lf, wf, sf = serve_fifo(reqs_f, arr_f)
        line["at_fifo_sustainable_rate"] = {
            "requests": len(reqs_f), "rate_per_s": round(rate_f, 4), "fifo_capacity_calibration_per_s": round(cap_f, 4),
            "mixed_continuous_batching": summary(lm, wm, sm, len(reqs_f)),
            "fifo_fp64_one_at_a_time": summary(lf, wf, sf, len(reqs_f)),
            "p50_ratio_fifo_over_mixed": round(float(np.percentile(lf, 50) / np.percentile(lm, 50)), 2),
            "p99_ratio_fifo_over_mixed": round(float(np.percentile(lf, 99) / np.percentile(lm, 99)), 2)}
    for lat in lats.values():
        lat.close()
    return line


# ---------------------------------------------------------- oracle (CPU) arm
def oracle_iterations():
    p = os.path.join(ROOT, "tests", "golden", "oracle_cgnr_24x24x24x64.json")
    with open(p) as f:
        return int(json.load(f)["iterations"])


_ORACLE = {}


def oracle_setup():
    if not _ORACLE:
        import oracle
        from paper_2201_09004_b300 import synth
        U = synth.thin_links(DIMS, GAUGE_SEED).numpy()
        C = oracle.clover(DIMS, U, C_SW)
        _ORACLE["W"] = oracle.Wilson(DIMS, U, MASS, MU, clover=C)
        _ORACLE["b"] = synth.z2_source(DIMS, SOURCE_SEED).numpy()
    return _ORACLE["W"], _ORACLE["b"]


def oracle_seconds_per_iteration(threads, n1, n2, reps=1):
    """Seconds per FP64 CGNR iteration of the oracle on the full 24^3x64 system with
    `threads` OpenMP threads, taken differentially: runs of n1 and n2 iterations are
    timed and (t2 - t1) / (n2 - n1) is returned, so the setup that every run repeats
    (allocation, the first M^+ b, the final residual) cancels; with reps > 1 the median
    of that many such pairs (the host's other load makes single pairs noisy)."""
    import oracle
    W, b = oracle_setup()
    oracle.set_threads(threads)
    per, spent = [], 0.0
    for _ in range(reps):
        ts = []
        for n in (n1, n2):
            t0 = time.perf_counter()
            W.cgnr_fixed(b, n)
            ts.append(time.perf_counter() - t0)
        per.append((ts[1] - ts[0]) / (n2 - n1))
        spent += sum(ts)
    return float(np.median(per)), spent


# iterations of the two timed runs per core count, and the pairs whose median is taken:
# about 25 s of host time in all
ORACLE_SAMPLE = {1: (1, 2), "all": (2, 6)}
ORACLE_REPS = {1: 1, "all": 3}


def cpu_baseline_runs(n1_all=None, n2_all=None):
    """The oracle timed on 1 core and on all host cores, each as solves/s scaled by
    the oracle's own iteration count for a complete solve."""
    full = oracle_iterations()
    out = []
    for cores in (1, os.cpu_count() or 1):
        n1, n2 = ORACLE_SAMPLE[1] if cores == 1 else (n1_all or ORACLE_SAMPLE["all"][0], n2_all or ORACLE_SAMPLE["all"][1])
        reps = ORACLE_REPS[1] if cores == 1 else ORACLE_REPS["all"]
        per_it, spent = oracle_seconds_per_iteration(cores, n1, n2, reps)
        med = f"median of {reps} pairs of " if reps > 1 else ""
        out.append({"value": round(1.0 / (per_it * full), 6), "unit": "solves/s", "cores": cores, "kind": "oracle",
                    "seconds_per_iteration": round(per_it, 4),
                    "sample": f"FP64 CGNR of the oracle on the full 24^3x64 lattice: {med}runs of {n1} and {n2} "
                              f"iterations ({spent:.1f} s), per iteration (t{n2} - t{n1}) / {n2 - n1}, scaled to its "
                              f"{full} iterations per solve"})
    return out


def cpu_baseline():
    """cpu_baseline of the bench line: the all-core number, with the 1-core one beside it."""
    one, allc = cpu_baseline_runs()
    line = dict(allc)
    line["one_core"] = one
    return line


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle_setup()
    full = oracle_iterations()
    cores = os.cpu_count() or 1
    oracle_seconds_per_iteration(cores, 1, 2)  # warm-up (page-in, thread pool)
    t0 = time.perf_counter()
    per_it = []
    for _ in range(max(args.steps, 1)):
        pi, _ = oracle_seconds_per_iteration(cores, 1, 1 + args.ref_iters)
        per_it.append(pi)
    s = time.perf_counter() - t0
    per_solve = float(np.median(per_it)) * full
    value = 1.0 / per_solve
    one = cpu_baseline_runs()[0]
    sample = (f"each step: FP64 CGNR runs of 1 and {1 + args.ref_iters} iterations of the oracle on the full "
              f"24^3x64 lattice on {cores} cores, per iteration the difference, median over steps, scaled to its "
              f"{full} iterations per solve")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "solves/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(s / max(args.steps, 1) * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "dims": list(DIMS), "c_sw": C_SW, "m": MASS, "mu": MU},
            "cpu_baseline": {"value": round(value, 6), "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "sample": sample, "one_core": one},
            "e2e": {"value": round(value, 6), "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--prec", type=int, default=2, help="sloppy precision: 1 = FP32, 2 = FP16 storage")
    ap.add_argument("--recon", type=int, default=12, choices=[8, 12, 18],
                    help="link compression of the sloppy operator (thin / long links)")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--bicgstab-steps", type=int, default=3,
                    help="also time the mixed-precision BiCGStab solve of the same system")
    ap.add_argument("--gcr-steps", type=int, default=3,
                    help="also time the mixed-precision restarted GCR solve of the same system")
    ap.add_argument("--gcr-restart", type=int, default=0, help="GCR directions before a restart (0 = 12)")
    ap.add_argument("--with-configs", type=int, default=1,
                    help="1: also run the 36-RHS 32^3x96 and the 48^3x144 HISQ workloads and a short serving trace into the line")
    ap.add_argument("--persistent-steps", type=int, default=3,
                    help="also time the solve with the persistent CG kernel and with 1 / 4 iterations per graph")
    ap.add_argument("--ref-iters", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--eig-dims", type=int, nargs=4, default=[8, 8, 8, 16], help="eigen: lattice extents x y z t")
    ap.add_argument("--nev", type=int, default=2, help="eigen: low modes wanted")
    ap.add_argument("--nkv", type=int, default=24, help="eigen: Krylov basis size")
    ap.add_argument("--degree", type=int, default=96, help="eigen: Chebyshev filter degree")
    ap.add_argument("--lambda-cut", type=float, default=0.6, help="eigen: filter edge")
    ap.add_argument("--eig-tol", type=float, default=1e-8, help="eigen: residual bound")
    ap.add_argument("--max-restarts", type=int, default=30, help="eigen: restart limit")
    ap.add_argument("--workload", default="tmc", choices=["tmc", "multirhs", "hisq", "serving", "dslash", "hisq3col", "overlap", "tmms", "eigen", "delta"],
                    help="tmc: 24^3x64 twisted-mass clover (default, the headline); multirhs: 32^3x96, "
                         "36 right-hand sides; hisq: 48^3x144 multi-shift; serving: Poisson request stream; "
                         "dslash: the operator kernels alone; hisq3col: HISQ 3-column propagator 24^3x64; "
                         "overlap: g5 D_w and the sign function; tmms: twisted multi-mass solve")
    ap.add_argument("--requests", type=int, default=400, help="serving: number of requests")
    ap.add_argument("--serving-requests", type=int, default=60,
                    help="requests of the short serving trace inside the default line (0: skip)")
    ap.add_argument("--fifo-requests", type=int, default=40,
                    help="serving: requests of the trace at the FIFO FP64 server's sustainable rate (0: skip)")
    ap.add_argument("--graph-iters", type=int, default=0,
                    help="CG iterations per CUDA graph (0: library default, -1: no graphs)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        reference_arm(args)
    elif args.workload == "multirhs":
        print(json.dumps(run_multirhs(args)), flush=True)
    elif args.workload == "hisq":
        print(json.dumps(run_hisq(args)), flush=True)
    elif args.workload == "dslash":
        run_dslash(args)
    elif args.workload == "hisq3col":
        run_hisq_propagator(args)
    elif args.workload == "overlap":
        run_overlap(args)
    elif args.workload == "tmms":
        run_twisted_multimass(args)
    elif args.workload == "serving":
        print(json.dumps(run_serving(args)), flush=True)
    elif args.workload == "eigen":
        run_eigen(args)
    elif args.workload == "delta":
        run_delta(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
