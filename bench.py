#!/usr/bin/env python3
"""Benchmark of the GB300 FLD solver.

Workload (one step = the whole hot path on one synthetic volume):
  128^3 fBm sphere cloud (seed 0, 5 octaves, base frequency 4,
  sigma_t = 200 max(0, fbm - 0.35)^1.5, vacuum outside r = 0.45), albedo
  0.95, unit directional light along -z baked by the transmittance march
  (step h/2), Levermore-Pomraning limiter, solved with red-black SOR to a
  relative residual of 1e-6 (single-precision sweeps, float-float correction
  sweeps once single precision stalls).  Per step: set_medium from
  device-resident arrays, bake, solve.

Metric: voxel-updates/s (one update = one phi_p update; one red-black
iteration = nx*ny*nz updates) over the timed solves, plus time to the
residual.  `--gpus N` under torchrun runs N independent replicas (one GPU
per rank, per-rank seed); the value is the sum of all ranks' updates over
the slowest rank's time.

`--impl reference` times the FP64 CPU oracle on the same workload (bounded
samples of its iterations) on the host cores.

Besides the headline line's roofline of the dominant sweep kernel, the cloud
workload reports the other sweep families, the same sweeps at 256^3 (HBM-
resident), the Jacobi iteration, the solve from a 2x coarser start (nested),
the solve with Anderson mixing of its blocks of sweeps (anderson; --anderson M
puts it in the timed solves instead), the end-to-end number through the API
with host buffers, and the oracle's
rate on the host cores.  Other workloads (--workload): c3 (the 256^3 three-
limiter runs with the bfloat16 medium and oracle checks), batch (many solves
of uneven size, one after another and batched), serve (a Poisson request
stream with continuous batching), pipeline (the paper's end-to-end render
workload: bake, 1/4-resolution solve, 1024^2 ray march).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "FLD voxel-updates/s & time to rel. residual 1e-6 (% HBM peak); p50/p99 solve latency"
UNIT = "voxel-updates/s"
# algorithmic bytes per voxel update of one sweep (D stored, as in Algorithm 1):
# reads phi, D, sigma', sigma_a' dl^2, j dl^2 and writes phi, D (4 bytes each).
# The method's bytes are the same for every precision family: the low word of
# phi that the hi/lo and float-float sweeps also move (8 more bytes) is a
# choice of this implementation's arithmetic, so it is not counted as useful
# traffic -- those passes are judged against the 28 bytes the method needs.
BYTES_PER_UPDATE = {"fp32": 28, "fh": 28, "ff": 28}
# with the bfloat16 medium the single-precision and hi/lo sweeps read sigma' and
# sigma_a' in 2 bytes each
BYTES_PER_UPDATE_BF16 = {"fp32": 24, "fh": 24, "ff": 28}
KERNEL_NAME = {"fp32": "k_pass2_f32 (single-precision red/black pass, two unknowns per thread)",
               "fh": "k_pass2_fh (hi/lo phi, FP32-summed red/black pass, two unknowns per thread)",
               "ff": "k_pass_ff (float-float correction pass)"}


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--omega", type=float, default=0.0, help="SOR factor (0 = library default)")
    ap.add_argument("--check-every", type=int, default=256)
    ap.add_argument("--max-iters", type=int, default=600000)
    ap.add_argument("--fp32-switch", type=float, default=0.0,
                    help="residual at which the float-float sweeps take over (0 = library default)")
    ap.add_argument("--nested", type=int, default=0,
                    help="start each solve from the solution of this many 2x coarser problems (0: cold start)")
    ap.add_argument("--anderson", type=int, default=0,
                    help="Anderson mixing over this many blocks of sweeps in the timed solves (0: plain SOR)")
    ap.add_argument("--anderson-m", type=int, default=8, help="extra 'anderson': history length")
    ap.add_argument("--anderson-check", type=int, default=64, help="extra 'anderson': sweeps per block")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="CPU-baseline sample length")
    ap.add_argument("--accuracy-n", type=int, default=64,
                    help="edge of the same-recipe cloud whose GPU solution is compared with the oracle's fixed point")
    ap.add_argument("--no-extras", action="store_true", help="skip cpu baseline / 256^3 roofline / e2e")
    ap.add_argument("--c3-n", type=int, default=256, help="c3 workload: edge of the timed solves")
    ap.add_argument("--c3-set", choices=["one", "diag", "full"], default="diag",
                    help="c3 workload: (seed, albedo) pairs -- one: (1, 0.95); diag: (1, 0.8), (2, 0.95), "
                         "(3, 0.99); full: all 9 -- each with the three limiters")
    ap.add_argument("--c3-limiters", default="lp,kershaw,larsen", help="c3 workload: limiters (comma list)")
    ap.add_argument("--c3-oracle-n", type=int, default=32,
                    help="c3 workload: edge of the same-recipe solves compared with the FP64 oracle's fixed point")
    ap.add_argument("--scenes", default="nebulae,manix,explosion", help="pipeline workload: scenes")
    ap.add_argument("--factor", type=int, default=4, help="pipeline workload: coarsening of the phi grid")
    ap.add_argument("--iters", type=int, default=64, help="sweeps workload: iterations timed per configuration")
    ap.add_argument("--sweep-n", default="128,256", help="sweeps workload: grid edges (the C2 medium tiled)")
    ap.add_argument("--workload", choices=["cloud", "batch", "serve", "c3", "pipeline", "sweeps"], default="cloud",
                    help="cloud: the 128^3 solve (default); batch: independent solves of uneven size, "
                         "batched in shared launches vs one after another")
    ap.add_argument("--count", type=int, default=16, help="batch workload: number of solves")
    ap.add_argument("--sizes", default="32,48,64,96", help="batch workload: edge lengths drawn from")
    ap.add_argument("--batch-modes", default="sequential,batched,batched_multi,sequential_anderson,batched_anderson",
                    help="batch workload: arms to run (sequential, batched, batched_multi, sequential_anderson, "
                         "batched_anderson, batched_anderson_multi; 'multi': batch_launch = 1)")
    ap.add_argument("--rate", type=float, default=0.0, help="serve workload: Poisson arrival rate (req/s; 0: profile)")
    ap.add_argument("--requests", type=int, default=0, help="serve workload: number of requests (0: profile)")
    ap.add_argument("--serve-profile", choices=["stated", "scaled"], default="stated",
                    help="serve workload: the stream as stated (200 req/s, 2000 requests, U{48..256}, 512^3 every "
                         "100th) or scaled to one GPU")
    ap.add_argument("--serve-seconds", type=float, default=120.0, help="serve workload: length of each arm (stated)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# ranks
# ---------------------------------------------------------------------------

class Ranks:
    def __init__(self, use_cuda: bool):
        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.dist = None
        self.device = None
        if self.world > 1:
            import torch
            import torch.distributed as dist
            backend = "nccl" if use_cuda else "gloo"
            if use_cuda:
                torch.cuda.set_device(self.local)
                self.device = torch.device("cuda", self.local)
            dist.init_process_group(backend=backend)
            self.dist = dist

    def barrier(self):
        if self.dist:
            self.dist.barrier()

    def reduce(self, value: float, op: str) -> float:
        if not self.dist:
            return value
        import torch
        t = torch.tensor([value], dtype=torch.float64, device=self.device or "cpu")
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX if op == "max" else self.dist.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.dist:
            self.dist.destroy_process_group()


class _OneRank:
    rank, world, local = 0, 1, 0


def reduce_ranks(values, world_max_time):
    """Whole-job throughput: all ranks' updates over the slowest rank's time."""
    return sum(values) / world_max_time if world_max_time > 0 else 0.0


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, local_index: int):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        ids = [x.strip() for x in vis.split(",")] if vis else []
        self.gpu = ids[local_index] if local_index < len(ids) else str(local_index)
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="fld_clocks_", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
            os.unlink(self.path)
        except OSError:
            return None
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


def traffic_record(kernel_key: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, valid only while
    the kernel source is unchanged since the capture (source hash recorded)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    src = os.path.join(ROOT, "paper_1403_8105_gb300", "csrc", "fld_kernels.cu")
    try:
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        for line in open(path):
            f = dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
            if f.get("kernel") == kernel_key and f.get("workload") == workload and f.get("src") == digest:
                return float(f["bytes_per_launch"])
    except (OSError, ValueError, KeyError):
        pass
    return None


# ---------------------------------------------------------------------------
# inputs
# ---------------------------------------------------------------------------

def workload_inputs(n: int, seed: int):
    import fld_inputs
    sig, alb = fld_inputs.cloud_medium(n, seed=seed, albedo=0.95)
    return sig, alb


def workload_config(args, ranks):
    return {
        "workload": f"C2 heterogeneous fBm sphere cloud {args.n}^3 (unit cube, h=1/{args.n}), albedo 0.95, "
                    f"unit directional light along -z (march step h/2), Levermore-Pomraning, "
                    f"rel. residual {args.tol:g}",
        "grid": [args.n, args.n, args.n],
        "seed": "0 + rank",
        "precision": "mixed: fp32 sweeps, float-float correction sweeps after the fp32 stall",
        "start": (f"nested: from the solution of {args.nested} successively 2x coarser box-averaged problems"
                  if args.nested else "cold: the paper's initial state, omega = 1 warm-up"),
        "scheme": "red-black SOR (Algorithm 1), self-consistent point update (local_iters=2)"
                  + (f", Anderson mixing over the last {args.anderson} blocks of sweeps" if args.anderson else ""),
        "limiter": "levermore-pomraning",
        "tol": args.tol,
        "l2": "flushed (256 MB write) before every timed step; the 128^3 working set (~70 MB) is L2-resident "
              "within a solve",
        "parallelism": f"replicas x{ranks.world}" if ranks.world > 1 else "1 GPU",
    }


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_gpu(args):
    import numpy as np
    import torch

    import paper_1403_8105_gb300 as fld

    ranks = Ranks(use_cuda=True)
    torch.cuda.set_device(ranks.local)
    dev = torch.device("cuda", ranks.local)
    fld.load(build_if_missing=True)
    n = args.n
    h = 1.0 / n
    nvox = n ** 3
    sig_np, alb_np = workload_inputs(n, seed=ranks.rank)
    sig = torch.from_numpy(sig_np).to(dev)
    alb = torch.from_numpy(alb_np).to(dev)
    torch.cuda.synchronize()          # inputs resident before the grid's stream reads them
    stream = torch.cuda.Stream(device=dev)
    g = fld.Grid(n, n, n, h, stream=stream.cuda_stream)
    p = fld.params(limiter="lp", precision="mixed", tol=args.tol, omega=args.omega, local_iters=2,
                   check_every=args.check_every, max_iters=args.max_iters, fp32_switch=args.fp32_switch,
                   nested=args.nested, anderson=args.anderson)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2

    def step():
        g.set_medium(sig, alb)
        g.bake_directional((0.0, 0.0, -1.0), 1.0)
        return g.solve(p)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        stream.synchronize()

        sampler = ClockSampler(ranks.local)
        ranks.barrier()
        torch.cuda.synchronize()
        sampler.start()
        results, step_ms = [], []
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        for _ in range(args.steps):
            flush.fill_(1.0)
            stream.synchronize()
            e0.record(stream)
            results.append(step())
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        ranks.barrier()
        clocks = sampler.stop()

    total_ms = sum(step_ms)
    updates = sum(r.iterations * nvox + r.updates_coarse for r in results)
    max_ms = ranks.reduce(total_ms, "max")
    all_updates = ranks.reduce(float(updates), "sum")
    value = all_updates / (max_ms / 1e3)
    launches = sum(int(r.kernels) + 3 for r in results)   # + set_medium validation (2) + bake (1)

    # sweep kernel timing inside the timed solves (graph blocks hold only passes)
    fam_ms = {"fp32": sum(r.ms_sweep_fp32 for r in results), "fh": sum(r.ms_sweep_mid for r in results),
              "ff": sum(r.ms_sweep_corr for r in results)}
    fam_it = {"fp32": sum(r.iterations_fp32 for r in results), "fh": sum(r.iterations_mid for r in results),
              "ff": sum(r.iterations_corr for r in results)}
    dom = max(fam_ms, key=lambda k: fam_ms[k])
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    peak_src = "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback 6.8 TB/s"

    def roof(fam, ms_total, iters, nv, workload, l2_resident):
        if iters == 0 or ms_total <= 0:
            return None
        launch_s = ms_total / 1e3 / (2 * iters)
        alg = BYTES_PER_UPDATE[fam] * nv / 2           # one launch updates one colour
        ach = alg / launch_s / 1e9
        return {"bound": "hbm", "kernel": KERNEL_NAME[fam], "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                "frac": round(ach / peak, 4), "traffic": traffic_record(fam, workload),
                "algorithmic_bytes_per_launch": alg, "launch_us": round(launch_s * 1e6, 3),
                "launches_measured": 2 * iters, "peak_source": peak_src, "l2_resident": l2_resident}

    roof_l2 = {f: roof(f, fam_ms[f], fam_it[f], nvox, f"cloud{n}", True) for f in fam_ms}
    roofline = roof_l2[dom]
    extras = {}
    if ranks.rank == 0:
        # The headline roofline is the dominant sweep family timed on a 256^3
        # volume, whose working set streams from HBM; at 128^3 the fields stay
        # in the 126 MB L2 between passes and the figure is not an HBM one.
        hbm = roofline_256(fld, torch, dev, sig_np, alb_np, roof, only=None if not args.no_extras else dom)
        if hbm.get(dom):
            roofline = dict(hbm[dom], dominant_in_solve=f"{dom}: {fam_ms[dom] / max(1e-9, sum(fam_ms.values())):.2f} "
                                                             f"of the sweep time of the {n}^3 solves")
        extras["roofline_hbm_resident"] = hbm
    extras["roofline_l2_resident_cloud"] = roof_l2
    if ranks.rank == 0 and not args.no_extras:
        extras["roofline_jacobi"] = roofline_jacobi(fld, torch, dev, sig_np, alb_np, peak, peak_src)
        extras["nested_start"] = nested_measure(fld, torch, g, stream, flush, sig, alb, p, n)
        extras["anderson"] = anderson_measure(fld, torch, g, stream, flush, sig, alb, p, n, args)
        extras["e2e"] = e2e_measure(fld, g, sig_np, alb_np, p, n, args)
        acc_n = args.accuracy_n
        acc_phi, acc_res = gpu_solve_at(fld, torch, dev, acc_n, p)
        base, acc = cpu_baseline(sig_np, alb_np, n, args.cpu_seconds, acc_n, acc_phi)
        extras["cpu_baseline"] = base
        acc.update({"gpu_rel_residual_fp64": acc_res.rel_residual,
                    "gpu_rel_residual_single_d": acc_res.rel_residual_single,
                    "gpu_iterations": acc_res.iterations, "gpu_fp64_sweeps": acc_res.iterations_fp64})
        extras["accuracy_vs_oracle"] = acc
        for k in ("rel_l2_vs_oracle", "rel_max_vs_oracle"):
            extras[k] = acc[k]
    g.close()

    times_s = [ms / 1e3 for ms in step_ms]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ranks.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (float-float correction sweeps; FP64 stop test and final sweeps)",
        "data": "synthetic",
        "config": workload_config(args, ranks),
        "time_to_residual_s": {"p50": statistics.median(times_s), "max": max(times_s)},
        "iterations_per_solve": [r.iterations for r in results],
        "coarse_iterations_per_solve": [r.iterations_coarse for r in results],
        "iterations_fp32_per_solve": [r.iterations_fp32 for r in results],
        "iterations_fp64_per_solve": [r.iterations_fp64 for r in results],
        "rel_residual": [r.rel_residual for r in results],
        "rel_residual_single_d": [r.rel_residual_single for r in results],
        "status": [fld.fld_status_string(r.status) for r in results],
        "roofline": roofline,
        "iterations_by_family_per_solve": {f: fam_it[f] // max(1, len(results)) for f in fam_it},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    line.update(extras)
    if "e2e" not in line:
        line["e2e"] = None
    ranks.barrier()
    if ranks.rank == 0:
        print(json.dumps(line), flush=True)
    ranks.close()


def roofline_256(fld, torch, dev, sig_np, alb_np, roof, only=None):
    """The same sweeps on a 256^3 volume (the 128^3 medium tiled 2x2x2), whose
    ~0.5 GB working set cannot stay in L2: the pass then streams from HBM.
    only: measure just that family."""
    import numpy as np
    n = 2 * sig_np.shape[0]
    sig = torch.from_numpy(np.tile(sig_np, (2, 2, 2))).to(dev)
    alb = torch.from_numpy(np.tile(alb_np, (2, 2, 2))).to(dev)
    torch.cuda.synchronize()
    stream = torch.cuda.Stream(device=dev)
    out = {}
    g = fld.Grid(n, n, n, 1.0 / n, stream=stream.cuda_stream)
    try:
        g.set_medium(sig, alb)
        g.bake_directional((0.0, 0.0, -1.0), 1.0)
        for fam, prec in (("fp32", "fp32"), ("fh", "pair"), ("ff", "mixed")):
            if only and fam != only:
                continue
            p = fld.params(limiter="lp", precision=prec, tol=0.0, local_iters=2, check_every=64, max_iters=64,
                           fp32_switch=1e30)
            g.solve(p, check=False)            # warm-up (and graph capture); MIXED switches after one block
            p.warm_start = 1                   # ... and its warm start continues with float-float sweeps
            r = g.solve(p, check=False)
            ms = {"fp32": r.ms_sweep_fp32, "fh": r.ms_sweep_mid, "ff": r.ms_sweep_corr}[fam]
            it = {"fp32": r.iterations_fp32, "fh": r.iterations_mid, "ff": r.iterations_corr}[fam]
            out[fam] = roof(fam, ms, it, n ** 3, f"cloud{n}", False)
    finally:
        g.close()
    return out


def nested_measure(fld, torch, g, stream, flush, sig, alb, p, n):
    """The same solve started from a 2x coarser box-averaged problem
    (fld_solve_params.nested = 1): one warm-up, then the median of 3."""
    import ctypes
    q = type(p)()
    ctypes.memmove(ctypes.byref(q), ctypes.byref(p), ctypes.sizeof(p))
    q.nested = 1
    times, res = [], []
    with torch.cuda.stream(stream):
        for k in range(4):
            flush.fill_(1.0)
            stream.synchronize()
            g.set_medium(sig, alb)
            g.bake_directional((0.0, 0.0, -1.0), 1.0)
            r = g.solve(q)
            if k:
                times.append(r.ms / 1e3)
                res.append(r)
    r = res[0]
    return {"time_to_residual_s_p50": statistics.median(times), "iterations": r.iterations,
            "coarse_iterations": r.iterations_coarse, "coarse_grid": [(n + 1) // 2] * 3,
            "voxel_updates_per_s": (r.iterations * n ** 3 + r.updates_coarse) / (r.ms / 1e3),
            "rel_residual": r.rel_residual, "status": fld.fld_status_string(r.status)}


def anderson_measure(fld, torch, g, stream, flush, sig, alb, p, n, args):
    """The same cold solve with Anderson mixing over the last --anderson-m
    blocks of --anderson-check sweeps (fld_solve_params.anderson): one
    warm-up, then the median of 3."""
    import ctypes
    q = type(p)()
    ctypes.memmove(ctypes.byref(q), ctypes.byref(p), ctypes.sizeof(p))
    q.anderson = args.anderson_m
    q.check_every = args.anderson_check
    q.nested = 0
    times, res = [], []
    with torch.cuda.stream(stream):
        for k in range(4):
            flush.fill_(1.0)
            stream.synchronize()
            g.set_medium(sig, alb)
            g.bake_directional((0.0, 0.0, -1.0), 1.0)
            r = g.solve(q, check=False)
            if k:
                times.append(r.ms / 1e3)
                res.append(r)
    r = res[0]
    return {"m": args.anderson_m, "sweeps_per_block": args.anderson_check,
            "time_to_residual_s_p50": statistics.median(times), "iterations": r.iterations,
            "iterations_by_family": {"fp32": r.iterations_fp32, "fh": r.iterations_mid, "ff": r.iterations_corr},
            "mixing_steps": r.anderson_steps, "history_restarts": r.anderson_resets,
            "voxel_updates_per_s": r.iterations * n ** 3 / (r.ms / 1e3),
            "rel_residual": r.rel_residual, "status": fld.fld_status_string(r.status)}


def roofline_jacobi(fld, torch, dev, sig_np, alb_np, peak, peak_src):
    """Throughput of the Jacobi variant (FP32): per iteration one fresh-D pass
    (reads phi, sigma'; writes D: 12 B per voxel) and one update pass (reads
    phi, D, sigma_a' dl^2, j dl^2; writes phi': 20 B per voxel) over every
    unknown, at 128^3 and at 256^3 (the medium tiled 2x2x2)."""
    import numpy as np
    out = {}
    stream = torch.cuda.Stream(device=dev)
    for rep in (1, 2):
        n = rep * sig_np.shape[0]
        sig = torch.from_numpy(np.tile(sig_np, (rep,) * 3)).to(dev)
        alb = torch.from_numpy(np.tile(alb_np, (rep,) * 3)).to(dev)
        torch.cuda.synchronize()
        g = fld.Grid(n, n, n, 1.0 / n, stream=stream.cuda_stream)
        try:
            g.set_medium(sig, alb)
            g.bake_directional((0.0, 0.0, -1.0), 1.0)
            p = fld.params(limiter="lp", precision="fp32", scheme="jacobi", tol=0.0, check_every=64, max_iters=64)
            g.solve(p, check=False)
            p.warm_start = 1
            r = g.solve(p, check=False)
            it_s = r.ms_sweep_fp32 / 1e3 / r.iterations_fp32
            alg = 32 * n ** 3
            ach = alg / it_s / 1e9
            out[f"cloud{n}"] = {"bound": "hbm", "kernel": "k_fresh_D_f + k_jacobi<float> (one Jacobi iteration)",
                                "achieved": round(ach, 1), "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 4),
                                "traffic": None, "algorithmic_bytes_per_iteration": alg,
                                "iteration_us": round(it_s * 1e6, 3), "iterations_measured": r.iterations_fp32,
                                "voxel_updates_per_s": n ** 3 / it_s, "peak_source": peak_src,
                                "l2_resident": n <= 128}
        finally:
            g.close()
    return out


def e2e_measure(fld, g, sig_np, alb_np, p, n, args):
    """The same steps through the public API with host buffers: the medium is
    copied host->device inside the step and phi is read back to the host."""
    import numpy as np
    import torch
    phi = np.empty((n + 2, n + 2, n + 2), np.float64)
    times, updates, checks = [], 0, 0
    for _ in range(max(1, args.e2e_steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.set_medium(sig_np, alb_np)
        g.bake_directional((0.0, 0.0, -1.0), 1.0)
        r = g.solve(p)
        fld.fld_get_state(g.handle, phi, None)
        times.append(time.perf_counter() - t0)
        updates += r.iterations * n ** 3 + r.updates_coarse
        checks += r.checks
    steps = max(1, args.e2e_steps)
    return {"value": updates / sum(times), "unit": UNIT, "steps": steps,
            "h2d_bytes_per_step": int(sig_np.nbytes + alb_np.nbytes),
            "d2h_bytes_per_step": int(phi.nbytes + 16 * checks / steps)}


def gpu_solve_at(fld, torch, dev, n, p):
    """The bench's solve (same parameters) on the same-recipe cloud of edge n;
    returns phi (padded, FP64, host) and the result."""
    import numpy as np
    sig_np, alb_np = workload_inputs(n, seed=0)
    stream = torch.cuda.Stream(device=dev)
    g = fld.Grid(n, n, n, 1.0 / n, stream=stream.cuda_stream)
    try:
        g.set_medium(sig_np, alb_np)
        g.bake_directional((0.0, 0.0, -1.0), 1.0)
        r = g.solve(p)
        phi = np.empty((n + 2, n + 2, n + 2), np.float64)
        fld.fld_get_state(g.handle, phi, None)
    finally:
        g.close()
    return phi, r


def cpu_baseline(sig_np, alb_np, n, seconds, acc_n=0, acc_phi=None):
    """The FP64 oracle as it stands, on the host cores.

    1. Baseline: iterations of Algorithm 1 on the same 128^3 cloud, for about
       `seconds`.
    2. Accuracy of the GPU result: the oracle's fixed point of the same recipe
       at edge acc_n (its own bake of the light, Anderson-mixed blocks of its
       sweeps until its fresh-D residual is <= 1e-10), against the GPU's
       phi of that cloud solved with the bench's parameters.  Returns
       (baseline, accuracy)."""
    import numpy as np
    import oracle
    q = oracle.bake_directional(sig_np, alb_np, 1.0 / n, (0, 0, -1), 1.0)
    prob = oracle.make_problem(sig_np, alb_np, q, 1.0 / n, limiter="lp", local_iters=2,
                               omega=oracle.omega_default(n, n, n))
    oracle.init_state(prob)
    it, t0 = 0, time.perf_counter()
    chunk = 2
    while True:
        oracle.rb_iteration(prob, chunk)
        it += chunk
        el = time.perf_counter() - t0
        if el >= seconds or it >= 100000:
            break
    base = {"value": it * n ** 3 / el, "unit": UNIT, "cores": prob.nthreads, "kind": "oracle",
            "sample": f"{it} iterations of Algorithm 1 (FP64, local_iters=2) on the {n}^3 cloud from the paper's "
                      f"initial state, {el:.1f} s; the oracle's full solve to 1e-6 at omega 1.93 takes 158,976 iterations"}
    # the same iterations on one host thread (a quarter of the time)
    cores = prob.nthreads
    prob.nthreads = 1
    it1, t0 = 0, time.perf_counter()
    while True:
        oracle.rb_iteration(prob, 1)
        it1 += 1
        el1 = time.perf_counter() - t0
        if el1 >= 0.25 * seconds or it1 >= 100000:
            break
    prob.nthreads = cores
    base["single_thread"] = {"value": it1 * n ** 3 / el1, "unit": UNIT, "cores": 1,
                             "sample": f"{it1} further iterations on one thread, {el1:.1f} s"}
    if not acc_n or acc_phi is None:
        return base, {}
    s2, a2 = workload_inputs(acc_n, seed=0)
    h = 1.0 / acc_n
    q2 = oracle.bake_directional(s2, a2, h, (0, 0, -1), 1.0)
    ref = oracle.make_problem(s2, a2, q2, h, limiter="lp", local_iters=2, omega=1.6)
    oracle.init_state(ref)
    t0 = time.perf_counter()
    sweeps, rel = oracle.solve_anderson(ref, 1e-10, sweeps_per_block=32, m=8)
    t_ref = time.perf_counter() - t0
    inner = (slice(1, -1),) * 3
    a, b = acc_phi[inner], ref.phi[inner]
    floor = 1e-3 * np.abs(b).max()
    acc = {"grid": [acc_n] * 3, "recipe": "the bench's cloud recipe (seed 0, albedo 0.95, light along -z) at this edge",
           "rel_l2_vs_oracle": float(np.linalg.norm(a - b) / np.linalg.norm(b)),
           "rel_max_vs_oracle": float(np.abs(a - b).max() / np.abs(b).max()),
           "rel_max_per_element_vs_oracle": float((np.abs(a - b) / np.maximum(np.abs(b), floor)).max()),
           "per_element_floor": "1e-3 of max |phi*|",
           "oracle_fixed_point": f"Anderson-mixed blocks of Algorithm 1 (FP64, 32 sweeps, m=8, omega 1.6): {sweeps} "
                                 f"sweeps to rel. residual {rel:.2e}, {t_ref:.1f} s on {ref.nthreads} cores"}
    return base, acc


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    n = args.n
    sig_np, alb_np = workload_inputs(n, seed=0)
    q = oracle.bake_directional(sig_np, alb_np, 1.0 / n, (0, 0, -1), 1.0)
    prob = oracle.make_problem(sig_np, alb_np, q, 1.0 / n, limiter="lp", local_iters=2,
                               omega=oracle.omega_default(n, n, n))
    oracle.init_state(prob)
    per_step = 8     # iterations per step: a bounded sample of the solve
    for _ in range(args.warmup):
        oracle.rb_iteration(prob, per_step)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.rb_iteration(prob, per_step)
    el = time.perf_counter() - t0
    value = args.steps * per_step * n ** 3 / el
    cfg = workload_config(args, _OneRank())
    cfg["parallelism"] = "host cores"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": prob.nthreads, "kind": "oracle",
                         "sample": f"each step = {per_step} iterations of Algorithm 1 (FP64) on the {n}^3 cloud"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_batch(args):
    """Independent solves of uneven size (edges drawn from --sizes, per-solve
    fBm seed, albedo U[0.8, 0.99], point or oblique directional light), solved
    to the residual one after another with fld_solve and together with
    fld_solve_batch; both timed with CUDA events on one stream."""
    import numpy as np
    import torch

    import fld_inputs
    import paper_1403_8105_gb300 as fld

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    sizes = tuple(int(x) for x in args.sizes.split(","))
    specs = fld_inputs.batch_cases(args.count, seed=1234, sizes=sizes)
    stream = torch.cuda.Stream(device=dev)
    media = []
    for sp in specs:
        sig, alb = fld_inputs.cloud_medium(sp["n"], seed=sp["seed"] % 100000, albedo=sp["albedo"])
        media.append((torch.from_numpy(sig).to(dev), torch.from_numpy(alb).to(dev), sp))
    torch.cuda.synchronize()
    p = fld.params(limiter="lp", precision="mixed", tol=args.tol, check_every=args.check_every,
                   max_iters=args.max_iters)
    pa = fld.params(limiter="lp", precision="mixed", tol=args.tol, check_every=args.anderson_check,
                    max_iters=args.max_iters, anderson=args.anderson_m)

    def setup():
        grids = []
        for sig, alb, sp in media:
            n = sp["n"]
            g = fld.Grid(n, n, n, 1.0 / n, stream=stream.cuda_stream)
            g.set_medium(sig, alb)
            lt = sp["light"]
            if lt.kind == "point":
                g.bake_point(lt.pos, lt.power)
            else:
                g.bake_directional(lt.dir, lt.radiance)
            grids.append(g)
        stream.synchronize()
        return grids

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    modes = tuple(m for m in args.batch_modes.split(",") if m)
    known = ("sequential", "batched", "batched_multi", "sequential_anderson", "batched_anderson",
             "batched_anderson_multi")
    if not modes or any(m not in known for m in modes):
        raise SystemExit(f"--batch-modes: choose from {', '.join(known)}")
    for mode in modes:
        grids = setup()
        pm = pa if "anderson" in mode else p
        if mode.endswith("multi"):
            # one multi-grid launch per colour pass for the grids of a table
            pm = fld.params(**{**{k: getattr(pm, k) for k, _ in pm._fields_}, "batch_launch": 1})
        with torch.cuda.stream(stream):
            e0.record(stream)
            if mode.startswith("sequential"):
                rs, done_ms = [], []
                t0 = time.perf_counter()
                for g in grids:
                    rs.append(g.solve(pm))
                    done_ms.append(1e3 * (time.perf_counter() - t0))
            else:
                st, rs = fld.fld_solve_batch(grids, pm)
            e1.record(stream)
            e1.synchronize()
        ms = e0.elapsed_time(e1)
        upd = sum(r.iterations * g.shape[0] * g.shape[1] * g.shape[2] for r, g in zip(rs, grids))
        # latency: time from the start of the run to each solve's finish
        lat = sorted(r.ms for r in rs) if mode.startswith("batched") else sorted(done_ms)
        out[mode] = {"ms": ms, "updates": upd, "value": upd / (ms / 1e3),
                     "converged": sum(r.status == fld.FLD_OK for r in rs),
                     "per_solve_fields": ["edge", "status", "iterations", "rel_residual", "fp64_iterations",
                                          "anderson_resets", "omega_backoffs"],
                     "per_solve": [[g.shape[0], fld.fld_status_string(r.status), r.iterations,
                                    float("%.3g" % r.rel_residual), r.iterations_fp64, r.anderson_resets,
                                    r.omega_backoffs] for r, g in zip(rs, grids)]}
        if lat:
            out[mode]["latency_ms_p50"] = float(np.percentile(lat, 50))
            out[mode]["latency_ms_p99"] = float(np.percentile(lat, 99))
        for g in grids:
            g.close()
    head = out.get("batched") or next(iter(out.values()))
    line = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 0,
        "ms_per_step": head["ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (float-float correction sweeps)", "data": "synthetic",
        "config": {"workload": f"batch of {args.count} independent solves, edges from {sizes}, per-solve fBm "
                               f"seed, albedo U[0.8,0.99], point or oblique light, LP, rel. residual {args.tol:g}",
                   "sizes": [sp["n"] for sp in specs]},
        **out,
        "anderson": {"m": args.anderson_m, "sweeps_per_block": args.anderson_check},
    }
    for a, b in (("sequential", "batched"), ("sequential", "batched_anderson"),
                 ("sequential_anderson", "batched_anderson"), ("batched", "batched_multi"),
                 ("batched_anderson", "batched_anderson_multi")):
        if a in out and b in out:
            line[f"speedup_{b}_vs_{a}"] = out[a]["ms"] / out[b]["ms"]
    print(json.dumps(line), flush=True)


def run_serve(args):
    """A Poisson stream of independent solves served with continuous batching.

    --serve-profile stated (default): the configuration as stated -- rate
    --rate (200 req/s), --requests (2000) requests, edges U{48..256}, a 512^3
    request every 100th, per-request medium (one of four seeded 256^3 fBm
    clouds, resampled trilinearly to the request's edge and flipped/permuted by
    the request's seed), albedo U[0.8, 0.99], point or oblique light, LP, rel.
    residual --tol, Anderson mixing (m = --anderson-m, --anderson-check sweeps
    per block).  One GPU cannot keep up with this stream, so every arm runs
    for --serve-seconds and reports offered against achieved load, what was
    left unfinished, and the latency of what finished.  Arms: continuous
    batching; one request at a time (FIFO) with the same parameters; one at a
    time without Anderson mixing; one at a time in plain FP64 sweeps.
    --serve-profile scaled: the earlier stream scaled to one GPU (30 req/s,
    120 requests, edges U{24..64}, a 96^3 request every 50th), run to
    completion."""
    import numpy as np
    import torch
    import torch.nn.functional as F

    import fld_inputs
    import paper_1403_8105_gb300 as fld
    from paper_1403_8105_gb300 import serve

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stated = args.serve_profile == "stated"
    rate = args.rate if args.rate > 0 else (200.0 if stated else 30.0)
    count = args.requests if args.requests > 0 else (2000 if stated else 120)
    nmin, nmax = (48, 256) if stated else (24, 64)
    heavy_every, heavy_n = (100, 512) if stated else (50, 96)
    deadline = args.serve_seconds if stated else None
    arr = serve.poisson_arrivals(count, rate, 77)
    base_n = 256 if stated else 64
    bases = []
    for b in range(4):
        sig, _ = fld_inputs.cloud_medium(base_n, seed=b, albedo=0.9)
        bases.append(torch.from_numpy(sig).to(dev)[None, None])
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]

    def medium(n, seed, albedo):
        rg = np.random.default_rng(seed)
        v = F.interpolate(bases[seed % 4], size=(n, n, n), mode="trilinear", align_corners=False)[0, 0]
        v = v.permute(*perms[int(rg.integers(0, 6))])
        flips = [a for a in range(3) if rg.integers(0, 2)]
        if flips:
            v = torch.flip(v, flips)
        return v.contiguous(), torch.full((n, n, n), albedo, dtype=torch.float32, device=dev)

    am = args.anderson_m

    def make_requests(limit=None):
        reqs = []
        r2 = np.random.default_rng(78)
        for i in range(count if limit is None else limit):
            n = heavy_n if (i + 1) % heavy_every == 0 else int(r2.integers(nmin, nmax + 1))
            seed = int(r2.integers(0, 1 << 30))
            albedo = float(r2.uniform(0.8, 0.99))
            if r2.integers(0, 2):
                light = fld_inputs.Light(kind="point", pos=(float(r2.uniform(0.1, 0.9)), float(r2.uniform(0.1, 0.9)),
                                                             float(r2.uniform(1.05, 1.5))), power=2.0)
            else:
                light = fld_inputs.Light(kind="directional", dir=(float(r2.uniform(-0.3, 0.3)),
                                                                  float(r2.uniform(-0.3, 0.3)), -1.0))
            reqs.append(serve.Request(rid=i, arrival=float(arr[i]), n=n, medium=(seed, albedo), light=light,
                                      footprint=serve.footprint_bytes(n, anderson=am)))
        return reqs

    class Backend(serve.GpuBackend):
        def admit(self, req):
            seed, albedo = req.medium
            req.medium = medium(req.n, seed, albedo)
            g = super().admit(req)
            req.medium = (seed, albedo)
            return g

    common = dict(limiter="lp", precision="mixed", tol=args.tol, max_iters=args.max_iters, temporal_depth=-1)
    p = fld.params(check_every=args.anderson_check, anderson=am, **common)
    p_plain = fld.params(check_every=64, **common)
    stream = torch.cuda.Stream(device=dev)
    # warm-up: two small requests
    w = [serve.Request(rid=r.rid, arrival=0.0, n=min(r.n, 64), medium=r.medium, light=r.light, footprint=r.footprint)
         for r in make_requests(2)]
    be = Backend(p, stream=stream.cuda_stream)
    serve.serve(w, be)
    be.close()

    reqs = make_requests()
    torch.cuda.synchronize()
    be = Backend(p, stream=stream.cuda_stream)
    try:
        reqs, st = serve.serve(reqs, be, max_active=64, deadline=deadline)
    finally:
        be.close()
    fin = [r for r in reqs if r.finished >= 0]
    upd = sum(r.result.iterations * r.n ** 3 for r in fin)
    cont = dict(st, voxel_updates_per_s=(st["voxel_updates"] or upd) / st["run_s"],
                voxel_updates_per_s_finished=upd / st["run_s"],
                converged=sum(r.result.status == fld.FLD_OK for r in fin))

    def one_at_a_time(params, limit_s, max_requests=None, chunk=None):
        """Requests in arrival order, one solve at a time, until `limit_s`.
        With `chunk`, a solve runs in chunks of that many iterations (later
        chunks continue from the state with warm_start), so the arm stops
        within one chunk of its deadline (the plain FP64 arm, whose single
        solves can take many minutes); a request still unsolved then is not
        counted, its partial work is."""
        import ctypes
        rs = make_requests()
        t0 = time.perf_counter()
        lat, upd, n_done, work, failed = [], 0, 0, 0, 0
        for r in rs:
            now = time.perf_counter() - t0
            if (limit_s is not None and now >= limit_s) or (max_requests and n_done >= max_requests):
                break
            if now < r.arrival:
                time.sleep(r.arrival - now)
            g = fld.Grid(r.n, r.n, r.n, 1.0 / r.n, stream=stream.cuda_stream)
            g.set_medium(*medium(r.n, *r.medium))
            if r.light.kind == "point":
                g.bake_point(r.light.pos, r.light.power)
            else:
                g.bake_directional(r.light.dir, r.light.radiance)
            q = type(params)()
            ctypes.memmove(ctypes.byref(q), ctypes.byref(params), ctypes.sizeof(params))
            its, ok, late = 0, False, False
            while its < params.max_iters:
                q.max_iters = min(chunk or params.max_iters, params.max_iters - its)
                res = g.solve(q, check=False)
                its += res.iterations
                work += res.iterations * r.n ** 3
                if res.status != fld.FLD_ERR_NOT_CONVERGED or res.iterations < q.max_iters:
                    ok = res.status == fld.FLD_OK
                    break
                q.warm_start, q.warmup_iters = 1, 0
                if limit_s is not None and time.perf_counter() - t0 >= limit_s:
                    late = True
                    break
            g.close()
            if late:
                break
            if ok:
                lat.append(time.perf_counter() - t0 - r.arrival)
                upd += its * r.n ** 3
                n_done += 1
            else:
                failed += 1
        span = time.perf_counter() - t0
        return {"requests": n_done, "not_converged": failed, "run_s": span,
                "latency_s_p50": float(np.percentile(lat, 50)) if lat else None,
                "latency_s_p99": float(np.percentile(lat, 99)) if lat else None,
                "throughput_req_s": n_done / span, "voxel_updates_per_s": work / span,
                "voxel_updates_per_s_finished": upd / span}

    print(f"serve: continuous batching done ({cont['requests']} requests)", file=sys.stderr, flush=True)
    seq = one_at_a_time(p, deadline)
    print(f"serve: one at a time done ({seq['requests']} requests)", file=sys.stderr, flush=True)
    seq_plain = one_at_a_time(p_plain, deadline)
    print(f"serve: one at a time, no Anderson, done ({seq_plain['requests']} requests)", file=sys.stderr, flush=True)
    p64 = fld.params(limiter="lp", precision="fp64", tol=args.tol, check_every=64, max_iters=args.max_iters)
    seq64 = one_at_a_time(p64, deadline, max_requests=None if stated else 12, chunk=4096)
    mean_vox = float(np.mean([r.n ** 3 for r in make_requests()]))
    line = {
        "metric": METRIC, "value": cont["voxel_updates_per_s"], "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 1,
        "ms_per_step": cont["run_s"] * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (float-float correction sweeps; FP64 stop test)", "data": "synthetic",
        "config": {"workload": f"Poisson stream of {count} FLD solves at {rate:g} req/s, edges U{{{nmin}..{nmax}}}, "
                               f"every {heavy_every}th {heavy_n}^3, per-request medium/albedo/light, LP, "
                               f"rel. residual {args.tol:g}, Anderson m={am}",
                   "profile": args.serve_profile,
                   "deadline_s": deadline,
                   "admission": "free device memory >= footprint / 0.9 and < 64 solves in flight"},
        "offered": {"req_s": rate, "voxels_per_s": rate * mean_vox, "mean_voxels_per_request": mean_vox},
        "continuous_batching": cont, "one_at_a_time": seq, "one_at_a_time_no_anderson": seq_plain,
        "one_at_a_time_fp64": seq64,
        "throughput_gain_vs_one_at_a_time": cont["throughput_req_s"] / seq["throughput_req_s"]
        if seq["throughput_req_s"] else None,
        "throughput_gain_vs_fp64": cont["throughput_req_s"] / seq64["throughput_req_s"]
        if seq64["throughput_req_s"] else None,
    }
    print(json.dumps(line), flush=True)


C3_SEEDS = (1, 2, 3)
C3_ALBEDOS = (0.8, 0.95, 0.99)
C3_LIMITERS = ("lp", "kershaw", "larsen")


def c3_cases(which, limiters=C3_LIMITERS):
    if which == "one":
        pairs = [(1, 0.95)]
    elif which == "diag":
        pairs = list(zip(C3_SEEDS, C3_ALBEDOS))
    else:
        pairs = [(s, a) for s in C3_SEEDS for a in C3_ALBEDOS]
    return [(s, a, lim) for s, a in pairs for lim in limiters]


def run_c3(args):
    """The 256^3 three-limiter runs: fBm clouds with seeds 1-3 and albedo in
    {0.8, 0.95, 0.99}, Levermore-Pomraning / Kershaw / Larsen (n = 2), unit
    directional light along -z, sigma' and sigma_a' stored in bfloat16,
    single-precision sweeps with hi/lo and float-float correction sweeps, to a
    relative residual of 1e-6.  Per solve: device time of fld_solve (after the
    bake, grid resident, L2 flushed before), iterations, the library's
    residual, and the FP64 oracle's own residual of the returned phi on the
    same rounded medium.  The same recipe at --c3-oracle-n, where the oracle
    reaches its fixed point (1e-10) in seconds, gives the error of the
    mixed-precision phi against the oracle per limiter, and the shift of the
    oracle's phi* caused by rounding the medium to bfloat16."""
    import numpy as np
    import torch

    import fld_inputs
    import oracle
    import paper_1403_8105_gb300 as fld

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    fld.load(build_if_missing=True)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    cases = c3_cases(args.c3_set, tuple(x for x in args.c3_limiters.split(",") if x))

    def params(lim, n):
        return fld.params(limiter=lim, larsen_n=2.0, precision="mixed", tol=args.tol, local_iters=2,
                          check_every=args.check_every if n >= 128 else 32, max_iters=max(args.max_iters, 4000000),
                          medium_bf16=1)

    def baked_grid(n, seed, albedo):
        # the oracle bakes the light and both sides solve with that source,
        # so the oracle's checks below read no GPU-made input
        sig, alb = fld_inputs.cloud_medium(n, seed=seed, albedo=albedo)
        q = oracle.bake_directional(sig, alb, 1.0 / n, (0.0, 0.0, -1.0), 1.0).astype(np.float32)
        g = fld.Grid(n, n, n, 1.0 / n, stream=stream.cuda_stream)
        g.set_medium(torch.from_numpy(sig).to(dev), torch.from_numpy(alb).to(dev))
        g.set_source(torch.from_numpy(q).to(dev))
        g.q = q.astype(np.float64)
        return g, sig, alb

    with torch.cuda.stream(stream):
        for lim in C3_LIMITERS:                    # warm-up: module load, per-limiter kernels
            g, _, _ = baked_grid(32, 0, 0.9)
            g.solve(params(lim, 32))
            g.close()
        stream.synchronize()

        sampler = ClockSampler(0)
        sampler.start()
        rows, total_ms, total_updates, launches = [], 0.0, 0, 0
        for seed, albedo, lim in cases:
            n = args.c3_n
            g, sig, alb = baked_grid(n, seed, albedo)
            flush.fill_(1.0)
            stream.synchronize()
            r = g.solve(params(lim, n))
            stream.synchronize()
            phi, D = g.get_state()
            j = g.q
            g.close()
            prob = oracle.make_problem(sig, alb, j, 1.0 / n, limiter=lim, larsen_n=2.0, medium_bf16=True)
            prob.phi, prob.D = phi, D
            rel_oracle = oracle.residual(prob)[0]
            total_ms += r.ms
            total_updates += r.iterations * n ** 3
            launches += int(r.kernels) + 3
            rows.append({"seed": seed, "albedo": albedo, "limiter": lim, "status": fld.fld_status_string(r.status),
                         "time_to_residual_s": r.ms / 1e3, "iterations": r.iterations,
                         "iterations_by_family": {"fp32": r.iterations_fp32, "fh": r.iterations_mid,
                                                  "ff": r.iterations_corr},
                         "rel_residual": r.rel_residual, "rel_residual_oracle_fp64": rel_oracle,
                         "voxel_updates_per_s": r.iterations * n ** 3 / (r.ms / 1e3),
                         "min_phi": float(phi[1:-1, 1:-1, 1:-1].min())})
            print(json.dumps({"c3_case": rows[-1]}), flush=True)
        clocks = sampler.stop()

        # error against the oracle's fixed point on the same recipe at a size it can solve
        small = []
        m = args.c3_oracle_n
        for seed, albedo, lim in cases:
            g, sig, alb = baked_grid(m, seed, albedo)
            r = g.solve(params(lim, m))
            phi, _ = g.get_state()
            j = g.q
            g.close()
            ref, ref_rel = {}, {}
            for bf in (True, False):
                # the fixed point does not depend on omega: a conservative one
                # keeps the FP64 reference solve from cycling
                prob = oracle.make_problem(sig, alb, j, 1.0 / m, limiter=lim, larsen_n=2.0, local_iters=2,
                                           omega=1.5, medium_bf16=bf)
                oracle.init_state(prob)
                _, ref_rel[bf], _ = oracle.solve(prob, tol=1e-10, max_iters=100000, check_every=50)
                ref[bf] = prob.phi[1:-1, 1:-1, 1:-1]
            inner = phi[1:-1, 1:-1, 1:-1]
            l2 = float(np.linalg.norm(inner - ref[True]) / np.linalg.norm(ref[True]))
            mx = float(np.abs(inner - ref[True]).max() / np.abs(ref[True]).max())
            quant = float(np.linalg.norm(ref[True] - ref[False]) / np.linalg.norm(ref[False]))
            small.append({"seed": seed, "albedo": albedo, "limiter": lim, "n": m,
                          "status": fld.fld_status_string(r.status), "iterations": r.iterations,
                          "rel_l2_vs_oracle": l2, "rel_max_vs_oracle": mx, "oracle_rel_residual": ref_rel[True],
                          "bf16_medium_shift_of_phi_star": quant})
            print(json.dumps({"c3_oracle_case": small[-1]}), flush=True)

    times = [row["time_to_residual_s"] for row in rows]
    peaks = measured_peaks()
    line = {
        "metric": METRIC, "value": total_updates / (total_ms / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": len(rows), "warmup": len(C3_LIMITERS), "ms_per_step": total_ms / max(1, len(rows)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 sweeps, bf16 medium (float-float correction sweeps)", "data": "synthetic",
        "config": {"workload": f"C3 fBm sphere clouds {args.c3_n}^3, seeds/albedos {args.c3_set}, limiters LP / "
                               f"Kershaw / Larsen-2, bf16 sigma'/sigma_a', rel. residual {args.tol:g}",
                   "grid": [args.c3_n] * 3, "l2": "flushed (256 MB write) before every solve",
                   "parallelism": "1 GPU"},
        "time_to_residual_s": {"p50": statistics.median(times), "max": max(times)},
        "cases": rows, "oracle_error_same_recipe": small,
        "peak_hbm_gbs": peaks["hbm_gbs"] if peaks else None,
        "gpu_launches": launches, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


# The paper's end-to-end render times (GTX TITAN, single precision, solve to
# Rbar/jbar = 1e-4 on a grid of a quarter of the data's resolution, light bake
# and 1024^2 primary ray march included; Sec. 6.2, Figs. 1, 8, 9): context only.
PAPER_RENDER_S = {"nebulae": 0.6, "manix": 1.8, "explosion": 0.7}


def run_pipeline(args):
    """The paper's timed workload, end to end, on synthetic stand-ins of its
    three scenes (fld_inputs.paper_scene): per colour channel the light bake
    (plus emission) at full resolution, the box-averaged medium and source on
    a grid of 1/factor the resolution, the FLD solve there (to the paper's
    1e-4 and to 1e-6; three channels solved as one batch), and the 1024^2
    primary ray march at full resolution with phi upsampled.  Stages timed
    with CUDA events on one stream, inputs resident on the device; the median
    of --steps runs after --warmup."""
    import numpy as np
    import torch

    import fld_inputs
    import paper_1403_8105_gb300 as fld

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    fld.load(build_if_missing=True)
    stream = torch.cuda.Stream(device=dev)
    f = args.factor
    rows = []
    for name in [x for x in args.scenes.split(",") if x]:
        sc = fld_inputs.paper_scene(name)
        nz, ny, nx = sc.sigma_t.shape
        cx, cy, cz = (nx + f - 1) // f, (ny + f - 1) // f, (nz + f - 1) // f
        sig = torch.from_numpy(sc.sigma_t).to(dev)
        albs = [torch.from_numpy(a).to(dev) for a in sc.albedos]
        emis = torch.from_numpy(sc.emission).to(dev) if sc.emission is not None else None
        torch.cuda.synchronize()
        fine = [fld.Grid(nx, ny, nz, sc.h, stream=stream.cuda_stream) for _ in albs]
        coarse = [fld.Grid(cx, cy, cz, f * sc.h, stream=stream.cuda_stream) for _ in albs]
        box = (nx * sc.h, ny * sc.h, nz * sc.h)
        ctr = tuple(0.5 * b for b in box)
        cam = fld.camera(eye=(ctr[0] + 0.35 * box[1], ctr[1] + 0.45 * box[1], ctr[2] - 2.1 * box[1]), target=ctr,
                         fov_deg=40.0, width=1024, height=1024, background=0.05)
        images = [torch.empty((1024, 1024), dtype=torch.float32, device=dev) for _ in albs]
        for tol in (1e-4, 1e-6):
            p = fld.params(limiter="lp", precision="mixed", tol=tol, check_every=64, max_iters=args.max_iters)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
            runs = []
            for it in range(args.warmup + args.steps):
                with torch.cuda.stream(stream):
                    stream.synchronize()
                    ev[0].record(stream)
                    for g, a in zip(fine, albs):
                        g.set_medium(sig, a)
                        if emis is not None:
                            g.set_source(emis)
                        g.bake_directional(sc.light_dir, sc.light_radiance, accumulate=1 if emis is not None else 0)
                    ev[1].record(stream)
                    for g, c in zip(fine, coarse):
                        g.downsample_to(c, f)
                    ev[2].record(stream)
                    if len(coarse) == 1:
                        rs = [coarse[0].solve(p)]
                    else:
                        st, rs = fld.fld_solve_batch(coarse, p)
                    ev[3].record(stream)
                    for g, c, img in zip(fine, coarse, images):
                        fld.fld_render(g.handle, c.handle, cam, img, None, 1.0, 2.2)
                    ev[4].record(stream)
                    ev[4].synchronize()
                if it >= args.warmup:
                    ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(4)]
                    runs.append({"bake_ms": ms[0], "downsample_ms": ms[1], "solve_ms": ms[2], "render_ms": ms[3],
                                 "total_ms": sum(ms), "iterations": [r.iterations for r in rs],
                                 "rel_residual": [r.rel_residual for r in rs],
                                 "status": [fld.fld_status_string(r.status) for r in rs]})
            med = sorted(runs, key=lambda r: r["total_ms"])[len(runs) // 2]
            rows.append({"scene": name, "grid": [nx, ny, nz], "phi_grid": [cx, cy, cz], "channels": len(albs),
                         "tol": tol, **med, "paper_s_gtx_titan_tol_1e-4": PAPER_RENDER_S.get(name),
                         "image_mean_radiance": [float(img.mean()) for img in images]})
            print(json.dumps({"pipeline_case": rows[-1]}), flush=True)
        for g in fine + coarse:
            g.close()
    line = {"metric": "end-to-end render time (light bake + FLD solve at 1/%d resolution + 1024^2 ray march)" % f,
            "unit": "ms", "higher_is_better": False, "n_gpus": 1, "data": "synthetic stand-ins of the paper's scenes",
            "steps": args.steps, "warmup": args.warmup, "cases": rows}
    print(json.dumps(line), flush=True)


def run_sweeps(args):
    """Every sweep family (single precision, hi/lo, float-float) in every
    launch shape the library offers (launched colour passes; blocked launches
    of T = 1, 2, 4 iterations) on the C2 cloud medium tiled to each edge of
    --sweep-n: CUDA-event time per iteration over --iters iterations after a
    warm-up, voxel-updates/s, and the algorithmic bytes (28 per update) over
    that time against the measured HBM peak."""
    import numpy as np
    import torch

    import paper_1403_8105_gb300 as fld

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    base_sig, base_alb = workload_inputs(128, seed=0)
    out = {}
    for n in (int(x) for x in args.sweep_n.split(",")):
        rep = max(1, n // 128)
        sig = np.tile(base_sig, (rep,) * 3)[:n, :n, :n].copy()
        alb = np.tile(base_alb, (rep,) * 3)[:n, :n, :n].copy()
        stream = torch.cuda.Stream(device=dev)
        g = fld.Grid(n, n, n, 1.0 / n, stream=stream.cuda_stream)
        try:
            g.set_medium(sig, alb)
            g.bake_directional((0.0, 0.0, -1.0), 1.0)
            with torch.cuda.stream(stream):
                # a state 512 sweeps into the solve
                g.solve(fld.params(precision="fp32", tol=0.0, max_iters=512, check_every=256, temporal_depth=-1),
                        check=False)
                for fam, prec in (("fp32", "fp32"), ("fh", "pair"), ("ff", "mixed")):
                    shapes = [(-1, 2)] + ([(-1, 4), (1, 0), (2, 0), (4, 0)] if fam != "ff" else [])
                    for depth, cells in shapes:
                        p = fld.params(precision=prec, warm_start=1, temporal_depth=depth, omega=1.9,
                                       cells_per_thread=cells if depth < 0 else 0)
                        g.iterate(p, args.iters)
                        stream.synchronize()
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        g.iterate(p, args.iters)
                        e1.record(stream)
                        e1.synchronize()
                        us = 1e3 * e0.elapsed_time(e1) / args.iters
                        ach = 28.0 * n ** 3 / (us * 1e-6) / 1e9
                        if depth >= 0:
                            name = f"blocked T={depth}"
                        elif fam == "ff":
                            name = "launched, 1 unknown per thread"
                        else:
                            name = f"launched, {cells} unknowns per thread"
                        out[f"{n} {fam} {name}"] = {
                            "us_per_iteration": round(us, 3), "voxel_updates_per_s": n ** 3 / (us * 1e-6),
                            "algorithmic_GBps": round(ach, 1), "frac_of_measured_peak": round(ach / peak, 4)}
        finally:
            g.close()
    print(json.dumps({"workload": "sweeps", "peak_gbs": peak, "bytes_per_update": 28, "results": out}), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "c3":
        run_c3(args)
    elif args.workload == "pipeline":
        run_pipeline(args)
    elif args.workload == "sweeps":
        run_sweeps(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
