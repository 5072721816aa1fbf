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
  * clocks sampled with nvidia-smi during the timed region.
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
#   FP16 spinor = 24 x 2 B + 4 B norm = 52 B; FP16 R12 link = 24 B; FP32 spinor 96 B, R12 link 48 B.
#   AINV epilogue reads A^{-1} (144 reals + norm); XPAY reads the clover (72 reals + norm) and y.
BYTES_PER_SITE = {
    "wilson_dslash_f16_ainv": 52 + 8 * 24 + (144 * 2 + 4) + 52,
    "wilson_dslash_f16_xpay": 52 + 8 * 24 + (72 * 2 + 4) + 52 + 52,
    "wilson_dslash_f32_ainv": 96 + 8 * 48 + 144 * 4 + 96,
    "wilson_dslash_f32_xpay": 96 + 8 * 48 + 72 * 4 + 96 + 96,
    "wilson_dslash_f64_ainv": 192 + 8 * 144 + 144 * 8 + 192,
    "wilson_dslash_f64_xpay": 192 + 8 * 144 + 72 * 8 + 192 + 192,
}
FLOPS_PER_SITE = {"hop": 1320, "ainv": 1320 + 2 * 6 * 6 * 8, "xpay": 1320 + 2 * 36 * 8 + 48}
# dram__bytes_read.sum + dram__bytes_write.sum per launch from one ncu capture of the
# benchmark configuration (profiles/); None until captured for the current kernel.
NCU_TRAFFIC = {}

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
    sp = lib.solve_params(solver=lib.MIXED_CGNR, tol=TOL, delta=0.1, prec_sloppy=args.prec, recon_sloppy=lib.R12)
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
    lib.profile_reset()
    lib.profile_enable(True)
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
    lib.profile_enable(False)
    clocks = sampler.stop() if rank == 0 else None
    ms = ev0.elapsed_time(ev1)
    t = torch.tensor([ms], device=dev, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = world * args.steps / (ms_max * 1e-3)

    # dominant kernel and its roofline, from the events recorded in the timed region
    kernels = {}
    for name in BYTES_PER_SITE:
        n, tot = lib.profile_query(name)
        if n:
            kernels[name] = (n, tot)
    all_n, all_t = lib.profile_query("")
    dom = max(kernels, key=lambda k: kernels[k][1])
    n, tot = kernels[dom]
    vh = int(np.prod(DIMS)) // 2
    avg_s = tot / n * 1e-3
    byts = BYTES_PER_SITE[dom] * vh
    peak, peak_kind = measured_peaks()
    achieved = byts / avg_s / 1e9
    epi = dom.rsplit("_", 1)[1]
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_source": peak_kind, "frac_of_nominal_8tbs": round(achieved / 8000.0, 4),
                "algorithmic_bytes_per_launch": byts, "avg_launch_us": round(avg_s * 1e6, 2),
                "gflops": round(FLOPS_PER_SITE[epi] * vh / avg_s / 1e9, 1),
                "share_of_kernel_time": round(tot / all_t, 4), "traffic": NCU_TRAFFIC.get(dom)}
    per_kernel = {k: {"launches": v[0], "ms": round(v[1], 3),
                      "gbs": round(BYTES_PER_SITE[k] * vh / (v[1] / v[0] * 1e-3) / 1e9, 1)} for k, v in kernels.items()}

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

    # end to end through the C ABI with pinned host buffers
    bh = b.cpu().pin_memory()
    xh = torch.empty_like(bh).pin_memory()
    lat.solve(op, sp, [bh], out=[xh])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        lat.solve(op, sp, [bh], out=[xh])
    e2e_s = time.perf_counter() - t0
    tt = torch.tensor([e2e_s], device=dev, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    e2e = {"value": round(world * args.steps / float(tt.item()), 3), "unit": "solves/s",
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
                       "tol": TOL, "sloppy_precision": args.prec, "recon": 12, "delta": 0.1,
                       "parallelism": f"replicas{world}",
                       "l2": "inputs larger than L2 (clover inverse, clover and links ~0.3 GB per step)"},
            "iters": int(np.median(iters)), "reliable_updates": infos[-1]["reliable_updates"],
            "true_rel_residual_max": res,
            "latency_ms": {"p50": round(float(np.percentile(lat_ms, 50)), 3),
                           "p99": round(float(np.percentile(lat_ms, 99)), 3)},
            "roofline": roofline, "kernels": per_kernel, "fp64": fp64, "e2e": e2e,
            "gpu_launches": int(launches), "clocks": clocks,
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.cpu_iters)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


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


def cpu_baseline(niter):
    """The oracle's FP64 CGNR on the full lattice: niter iterations timed, scaled by
    the oracle's own iteration count for a complete solve."""
    W, b = oracle_setup()
    t0 = time.perf_counter()
    W.cgnr_fixed(b, niter)
    s = time.perf_counter() - t0
    full = oracle_iterations()
    per_solve = s / niter * full
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count()))
    return {"value": round(1.0 / per_solve, 6), "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": f"{niter} FP64 CGNR iterations of the oracle on the full 24^3x64 lattice ({s:.1f} s), "
                      f"scaled to its {full} iterations per solve"}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    W, b = oracle_setup()
    full = oracle_iterations()
    for _ in range(args.warmup):
        W.cgnr_fixed(b, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        W.cgnr_fixed(b, args.ref_iters)
    s = time.perf_counter() - t0
    per_solve = s / (args.steps * args.ref_iters) * full
    value = 1.0 / per_solve
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count()))
    sample = (f"each step: {args.ref_iters} FP64 CGNR iterations of the oracle on the full 24^3x64 lattice, "
              f"scaled to its {full} iterations per solve")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "solves/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(s / args.steps * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "dims": list(DIMS), "c_sw": C_SW, "m": MASS, "mu": MU},
            "cpu_baseline": {"value": round(value, 6), "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 6), "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--prec", type=int, default=2, help="sloppy precision: 1 = FP32, 2 = FP16 storage")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--cpu-iters", type=int, default=8)
    ap.add_argument("--ref-iters", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
