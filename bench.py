"""Benchmark: DoF/s of the CutFEM multigrid solve to a 1e-8 relative residual.

One step = one CG solve (V-cycle preconditioner, x_0 = 0, rtol 1e-8) of the
3D Q2 ball problem on a 224^3 background mesh (16,851,851 active DoFs, 6
levels: the "~17M DoF" sphere), FP64 plain form, inputs resident in HBM.  The
mixed form (FP32 V-cycle inside FP64 CG) is timed on the same problem to the
same residual and reported under "mixed", with its distance to the FP64
solution.  The 128^3 and 64^3 sizes follow under "sizes" (the 64^3 one also
against the stored oracle solution).  Each rank solves its own copy of the
problem (weak scaling, no collective on the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--extra NAME ...] [--no-batch] [--no-serve]

--impl reference times the CPU oracle (test infrastructure, plain numpy /
scipy) on a bounded sample of the same workload: the same ball on a 32^3
mesh (4 levels), PCG only (its setup is untimed).
"""

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "DoF/s solved to 1e-8 rel. residual, mixed vs FP64 form; p50/p99 latency"
WORKLOAD = "ball3d_q2_n224"
EXTRA = ("ball3d_q2_n128", "ball3d_q2_n64")
SAMPLE = "ball3d_q2_n32"
RTOL = 1e-8


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def _workload_desc(name):
    from paper_2508_11608_gb300.workloads import CONFIGS
    c = CONFIGS[name]
    return (f"{name}: 3D Poisson -Laplace u = f, u = prod sin(pi x_k), on the ball r={c['radius']} "
            f"at {tuple(c['center'])} cut from [-1,1]^3, {c['n_cells']}^3 cells, Q{c['degree']}, "
            f"{c['n_levels']} levels, Nitsche 20p^2/h, ghost penalty 0.1, n_c=2, CG + V-cycle "
            f"(1 pre/1 post MVS step), rtol {RTOL:g}")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except OSError:
        return {}


# FP64 and FP32 FMA throughput of this GB300 pool, measured by an FMA probe
# (2 flops per FMA; method and output in profiles/alu_peaks_gb300.md).
FP64_PEAK_TFLOPS = 1.26
FP32_PEAK_TFLOPS = 78.5


# DRAM traffic of a kernel relative to its algorithmic bytes, from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum over a few launches of
# one kernel on a small case; profiles/ holds the summary and the command).
# The bench scales it by the algorithmic bytes of a launch of the timed
# workload.  Valid only for the kernel sources it was taken on (sha256 over
# kernels.cuh and cutpipe.cuh).
TRAFFIC = {
    # ncu, one finest-level launch of the 128^3 mixed solve (colour 2 of the
    # first cut sweep): DRAM 117.74 + 3.99 MB against 89.32 MB algorithmic
    # (profiles/k_cut_warp_ball3d_q2_n128_mixed.md)
    ("k_cut_warp", "fp32"): {"dram_over_algorithmic": 121.73 / 89.32,
                             "kernels_sha256": "bdf2fa516d56fd94f76f6dabdb35aee623d8d9638b9252c4d75d029b7e533075"},
    # the same launch of the FP64 solve: DRAM 223.33 + 4.98 MB against
    # 171.20 MB algorithmic (profiles/k_cut_warp_ball3d_q2_n128_mixed.md)
    ("k_cut_warp", "fp64"): {"dram_over_algorithmic": 228.31 / 171.20,
                             "kernels_sha256": "bdf2fa516d56fd94f76f6dabdb35aee623d8d9638b9252c4d75d029b7e533075"},
}


def _kernels_sha256():
    import hashlib
    h = hashlib.sha256()
    for name in ("kernels.cuh", "cutpipe.cuh"):
        with open(os.path.join(ROOT, "paper_2508_11608_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def cpu_baseline(steps=1, threads=1):
    """Oracle PCG on the bounded sample in a subprocess, with the BLAS and
    OpenMP thread limits set to `threads`."""
    code = r"""
import json, os, sys, time
sys.path.insert(0, %r)
from oracle import Hierarchy, Sphere
from paper_2508_11608_gb300.workloads import CONFIGS
c = CONFIGS[%r]
H = Hierarchy(Sphere(c["center"], c["radius"]), c["dim"], c["n_cells"], c["degree"], c["n_levels"])
b = H.rhs()
n = b.size
out = []
for s in range(%d):
    t = time.perf_counter()
    x, it, hist = H.pcg(b, rtol=%r)
    out.append((time.perf_counter() - t, it))
print(json.dumps({"n": int(n), "runs": out}))
""" % (ROOT, SAMPLE, steps, RTOL)
    t = str(threads)
    env = dict(os.environ, OMP_NUM_THREADS=t, OPENBLAS_NUM_THREADS=t, MKL_NUM_THREADS=t)
    p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if p.returncode != 0:
        return {"error": p.stderr.strip().splitlines()[-1] if p.stderr.strip() else "failed"}
    r = json.loads(p.stdout.strip().splitlines()[-1])
    secs = [t for t, _ in r["runs"]]
    return {"n": r["n"], "secs": secs, "iterations": r["runs"][-1][1]}


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return 0
    res = cpu_baseline(steps=args.warmup + args.steps)
    if "error" in res:
        print(json.dumps({"impl": "reference", "unavailable": res["error"]}))
        return 0
    secs = res["secs"][args.warmup:]
    tot = sum(secs)
    value = res["n"] * len(secs) / tot
    sample = (f"oracle PCG (numpy/scipy, 1 thread) on {SAMPLE} ({res['n']} active DoFs), same ball "
              f"and method at 32^3 cells instead of 224^3, {res['iterations']} CG iterations; setup untimed")
    line = {
        "metric": METRIC, "value": value, "unit": "DoF/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(secs), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": _workload_desc(WORKLOAD), "sample": SAMPLE},
        "impl": "reference",
        "cpu_baseline": {"value": value, "unit": "DoF/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "DoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def agg_max(v, dist=None, device=None):
    """Max of a per-rank float over all ranks (the rank-local value without a
    process group).  gloo reduces CPU tensors, nccl device tensors."""
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def whole_job_rate(units_per_rank, world, ms_local, dist=None, device=None):
    """Weak scaling: every rank processes units_per_rank in its own timed
    region; the job's rate is all units over the slowest rank's time."""
    ms = agg_max(ms_local, dist, device)
    return world * units_per_rank / (ms * 1e-3), ms


def _timed_solves(pb, b, x, prec, steps, warmup, stream, flush, dist=None, profile_kernel=None, level=-1):
    """CUDA-event time of `steps` solves after `warmup` untimed ones, L2
    flushed before each timed solve.  Returns (ms list, infos, launches,
    profile); with profile_kernel, that family's launches (on `level`, or
    all levels) are event-timed one by one."""
    import torch
    pb.set_precision(prec)
    for _ in range(warmup):
        pb.solve(b, x, rtol=RTOL)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if profile_kernel:
        pb.profile_start(profile_kernel, level)
    l0 = pb.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    infos = []
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        infos.append(pb.solve(b, x, rtol=RTOL))
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = pb.launch_count() - l0
    prof = pb.profile_read() if profile_kernel else None
    return [e0.elapsed_time(e1) for e0, e1 in ev], infos, launches, prof


# the kernel of each profiled family in the 3D Q2 workloads (FP32 V-cycle
# of the mixed form / FP64 form)
KERNEL_NAMES = {1: ("k_cut_warp", "k_cut_warp"), 2: ("k_smooth_tc", "k_smooth_cart"),
                3: ("k_apply_bulk (V-cycle) + k_apply_sf (outer CG)", "k_apply_sf"),
                4: ("k_apply_bnd", "k_apply_bnd"), 5: ("k_face_moments_to + k_face_moments", "k_face_moments_to + k_face_moments")}


def _family_profile(cm, pb, b, x, prec, stream, flush):
    """Event-timed passes (graphs off for the timed family) of each kernel
    family: summed launch time, launches, algorithmic flops and bytes."""
    out = {}
    for kern in (cm._lib.CF_K_CUT_SOLVE, cm._lib.CF_K_INTERIOR, cm._lib.CF_K_APPLY_BULK,
                 cm._lib.CF_K_APPLY_BND, cm._lib.CF_K_FACE_MOMENTS):
        msk, _, _, pr = _timed_solves(pb, b, x, prec, 2, 1, stream, flush, profile_kernel=kern)
        pr["share"] = pr["ms"] / sum(msk)
        out[kern] = pr
    return out


def _roofline(cm, prof, prec, hbm):
    top = max(prof, key=lambda k: prof[k]["share"])
    pr = prof[top]
    per_launch_ms = pr["ms"] / max(pr["launches"], 1)
    fl_rate = pr["flops"] / (pr["ms"] * 1e-3) / 1e12 if pr["ms"] > 0 else 0.0
    by_rate = pr["bytes"] / (pr["ms"] * 1e-3) / 1e9 if pr["ms"] > 0 else 0.0
    alu = FP64_PEAK_TFLOPS if prec == cm.CF_FP64 else FP32_PEAK_TFLOPS
    t_alu = pr["flops"] / (alu * 1e12)
    t_hbm = pr["bytes"] / (hbm * 1e9)
    if t_alu >= t_hbm:
        roof = {"bound": "alu", "achieved": fl_rate, "peak": alu, "unit": "TFLOP/s", "frac": fl_rate / alu,
                "peak_source": ("FP64" if prec == cm.CF_FP64 else "FP32") +
                " FMA throughput measured on this pool (method in profiles/alu_peaks_gb300.md), of measured"}
    else:
        roof = {"bound": "hbm", "achieved": by_rate, "peak": hbm, "unit": "GB/s", "frac": by_rate / hbm,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs, of measured"}
    bytes_per_launch = pr["bytes"] / max(pr["launches"], 1)
    idx = 1 if prec == cm.CF_FP64 else 0
    tr = TRAFFIC.get((KERNEL_NAMES[top][idx], "fp64" if prec == cm.CF_FP64 else "fp32"))
    traffic = None
    if tr and tr["kernels_sha256"] == _kernels_sha256():
        traffic = tr["dram_over_algorithmic"] * bytes_per_launch
    roof.update({"kernel": KERNEL_NAMES[top][idx], "family": top, "traffic": traffic, "per_launch_ms": per_launch_ms,
                 "launches_timed": pr["launches"], "share_of_step": pr["share"],
                 "shares": {KERNEL_NAMES[k][idx]: round(prof[k]["share"], 4) for k in prof},
                 "flops_per_launch": pr["flops"] / max(pr["launches"], 1), "bytes_per_launch": bytes_per_launch,
                 "timing": "CUDA events on the launching stream around every launch of the family, "
                           "summed over 2 timed solves"})
    return roof


def _rel(a, b):
    import torch
    return (torch.linalg.norm(a - b) / torch.linalg.norm(b)).item()


def _size_line(cm, torch, name, dev, stream, flush, steps):
    """FP64 and mixed DoF/s of one more configuration (smaller sizes)."""
    from paper_2508_11608_gb300.workloads import problem_kwargs
    t0 = time.perf_counter()
    pb = cm.Problem(**problem_kwargs(name))
    setup_s = time.perf_counter() - t0
    n = pb.n_dofs()
    b = torch.zeros(n, dtype=torch.float64, device=dev)
    pb.rhs(b)
    xs, out = {}, {"workload": name, "active_dofs": n, "host_setup_s": setup_s}
    for prec, key in ((cm.CF_FP64, "fp64"), (cm.CF_MIXED, "mixed")):
        x = torch.zeros_like(b)
        ms, infos, _, _ = _timed_solves(pb, b, x, prec, steps, 3, stream, flush)
        xs[key] = x
        out[key] = {"value": n * len(ms) / (sum(ms) * 1e-3), "unit": "DoF/s", "ms_per_solve": sum(ms) / len(ms),
                    "iterations": infos[-1]["iterations"], "true_rel_residual": infos[-1]["true_rel_residual"]}
    out["mixed"]["rel_l2_vs_fp64"] = _rel(xs["mixed"], xs["fp64"])
    gold = os.path.join(ROOT, "tests", "golden", name + "_pcg.npz")
    if os.path.exists(gold):
        import numpy as np
        xo = torch.tensor(np.load(gold)["x"], device=dev)
        out["fp64"]["rel_l2_vs_oracle"] = _rel(xs["fp64"], xo)
        out["mixed"]["rel_l2_vs_oracle"] = _rel(xs["mixed"], xo)
    pb.close()
    return out


def run_ours(args):
    import numpy as np
    import torch

    import paper_2508_11608_gb300 as cm
    from paper_2508_11608_gb300.workloads import problem_kwargs

    rank, world, local = _env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    workload = args.workload

    t0 = time.perf_counter()
    pb = cm.Problem(**problem_kwargs(workload))
    setup_s = time.perf_counter() - t0
    n = pb.n_dofs()
    b = torch.zeros(n, dtype=torch.float64, device=dev)
    x = torch.zeros_like(b)
    pb.rhs(b)
    # L2 is 129 MB: a 512 MB write between timed solves evicts it
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float64, device=dev)

    # FP64 plain form: the headline (CUDA graphs on, nothing else timed)
    sampler = ClockSampler(local)
    sampler.start()
    ms64, inf64, launches, _ = _timed_solves(pb, b, x, cm.CF_FP64, args.steps, args.warmup, stream, flush, dist)
    clocks = sampler.stop()
    x64 = x.clone()
    # mixed form, same final residual
    ms32, inf32, launches32, _ = _timed_solves(pb, b, x, cm.CF_MIXED, args.steps, args.warmup, stream, flush, dist)
    mixed_err = _rel(x, x64)

    # kernel families, event-timed in separate passes of the same workload
    hbm = _peaks().get("hbm_gbs", 6800.0)
    prof32 = _family_profile(cm, pb, b, x, cm.CF_MIXED, stream, flush)
    prof64 = _family_profile(cm, pb, b, x, cm.CF_FP64, stream, flush)
    roof = _roofline(cm, prof32, cm.CF_MIXED, hbm)
    roof64 = _roofline(cm, prof64, cm.CF_FP64, hbm)
    # the dominant family's finest-level launches alone (the average above
    # includes the coarse levels' latency-bound launches)
    for rf, prec in ((roof, cm.CF_MIXED), (roof64, cm.CF_FP64)):
        fam = rf["family"]
        _, _, _, pf = _timed_solves(pb, b, x, prec, 2, 1, stream, flush, profile_kernel=fam,
                                    level=pb.n_levels - 1)
        if pf["launches"] > 0 and pf["ms"] > 0:
            sec = pf["ms"] * 1e-3
            fin = {"level": pb.n_levels - 1, "launches_timed": pf["launches"],
                   "per_launch_ms": pf["ms"] / pf["launches"]}
            if rf["unit"] == "GB/s":
                fin["achieved"] = pf["bytes"] / sec / 1e9
            else:
                fin["achieved"] = pf["flops"] / sec / 1e12
            fin["frac"] = fin["achieved"] / rf["peak"]
            rf["finest_level"] = fin

    # e2e through the C ABI with host buffers: H2D of b, solve, D2H of x
    pb.set_precision(cm.CF_FP64)
    hb = torch.empty(n, dtype=torch.float64, pin_memory=True)
    hb.copy_(b.cpu())
    hx = torch.empty(n, dtype=torch.float64, pin_memory=True)
    db = torch.empty_like(b)
    e2e_ms = []
    for k in range(args.steps + 1):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        db.copy_(hb, non_blocking=True)
        pb.solve(db, x, rtol=RTOL)
        hx.copy_(x, non_blocking=True)
        torch.cuda.synchronize()
        if k > 0:
            e2e_ms.append(1e3 * (time.perf_counter() - t))
    pb.close()
    del x, x64, db, b

    extra = {}
    if world == 1:
        for name in args.extra:
            extra[name] = _size_line(cm, torch, name, dev, stream, flush, max(3, args.steps // 2))
    batched = None
    if not args.no_batch:
        batched = run_batched(cm, torch, dev, stream, args)
    served = None
    if not args.no_serve and world == 1:
        served = run_serving(cm, torch, args)

    value, tot64 = whole_job_rate(n * args.steps, world, sum(ms64), dist, dev)
    mixed_value, tot32 = whole_job_rate(n * args.steps, world, sum(ms32), dist, dev)
    e2e_value, _ = whole_job_rate(n * len(e2e_ms), world, sum(e2e_ms), dist, dev)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    cpu_line = None
    if world == 1:
        cpu1 = cpu_baseline(steps=2, threads=1)
        cpun = cpu_baseline(steps=2, threads=os.cpu_count() or 1)
        if "error" not in cpu1:
            cpu_line = {"value": cpu1["n"] / min(cpu1["secs"]), "unit": "DoF/s", "cores": 1, "kind": "oracle",
                        "sample": f"oracle PCG on {SAMPLE} ({cpu1['n']} DoFs, {cpu1['iterations']} iterations; the "
                                  f"same ball at 32^3 cells), best of {len(cpu1['secs'])}; setup untimed",
                        "host_cores": os.cpu_count()}
            if "error" not in cpun:
                cpu_line["all_threads"] = {
                    "value": cpun["n"] / min(cpun["secs"]), "threads": os.cpu_count(),
                    "note": "BLAS/OpenMP thread limits set to the host's core count; scipy's sparse products "
                            "run on one thread whatever the limit"}

    line = {
        "metric": METRIC, "value": value, "unit": "DoF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot64 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": _workload_desc(workload), "active_dofs": n,
                   "form": "FP64 plain (CG, V-cycle, smoother, transfer all FP64), CUDA graphs",
                   "l2": "512 MB buffer written between timed solves (flush); the vectors exceed L2 too",
                   "iterations": inf64[-1]["iterations"],
                   "true_rel_residual": inf64[-1]["true_rel_residual"], "host_setup_s": setup_s},
        "latency_ms": {"p50": float(np.percentile(ms64, 50)), "p99": float(np.percentile(ms64, 99))},
        "mixed": {"value": mixed_value, "unit": "DoF/s", "ms_per_step": tot32 / args.steps,
                  "iterations": inf32[-1]["iterations"],
                  "true_rel_residual": inf32[-1]["true_rel_residual"],
                  "rel_l2_vs_fp64": mixed_err,
                  "speedup_vs_fp64": mixed_value / value,
                  "latency_ms": {"p50": float(np.percentile(ms32, 50)), "p99": float(np.percentile(ms32, 99))},
                  "gpu_launches": launches32,
                  "form": "FP32 V-cycle (smoother, transfer, cut-patch inverses) inside FP64 CG"},
        "e2e": {"value": e2e_value, "unit": "DoF/s", "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n},
        "gpu_launches": launches,
        "roofline": roof,
        "roofline_fp64": roof64,
        "cpu_baseline": cpu_line,
        "clocks": clocks,
        "sizes": extra,
        "batched": batched,
        "served": served,
    }
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


def run_batched(cm, torch, dev, stream, args):
    """256 seeded 2D flower instances (N in {32..256}, Q2/Q3 mixed), solved
    together through cf_batch_* in the mixed form; DoF/s over all instances."""
    from paper_2508_11608_gb300.workloads import flower_batch
    specs = flower_batch(count=args.batch_count)
    t0 = time.perf_counter()
    pbs = [cm.Problem(**k) for k in specs]
    setup_s = time.perf_counter() - t0
    bt = cm.Batch(pbs)
    bs, xs = [], []
    for pb in pbs:
        b = torch.zeros(pb.n_dofs(), dtype=torch.float64, device=dev)
        pb.rhs(b)
        bs.append(b)
        xs.append(torch.zeros_like(b))
    ndof = sum(pb.n_dofs() for pb in pbs)
    bt.solve(bs, xs, precision=cm.CF_MIXED)
    torch.cuda.synchronize()
    steps = max(2, args.steps // 3)
    l0 = bt.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        ev[k][0].record(stream)
        infos = bt.solve(bs, xs, precision=cm.CF_MIXED)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    its = [i["iterations"] for i in infos]
    launches = (bt.launch_count() - l0) / steps
    return {"value": ndof * steps / (sum(ms) * 1e-3), "unit": "DoF/s", "instances": len(pbs),
            "active_dofs": ndof, "ms_per_batch_solve": sum(ms) / steps, "precision": "mixed",
            "iterations_min_max": [min(its), max(its)],
            "worst_true_rel_residual": max(i["true_rel_residual"] for i in infos),
            "launches_per_batch_solve": launches, "host_setup_s": setup_s,
            "launch_mode": "each CG iteration's two halves (q = A p .. (r, r) and z = B r .. p) replayed as "
                           "CUDA graphs captured per version of the work lists",
            "workload": "2D flowers r = 0.6 + 0.1 cos(m (theta - theta0)), m in 3..7, offset <= 0.05, "
                        "N in {32, 64, 128, 256}, Q2/Q3, coarsest 8^2, seed 20260101"}


def run_serving(cm, torch, args):
    """Served form: a seeded stream of 3D Q2 requests (spheres, ellipsoids,
    tori; 32^3..96^3) with Poisson arrivals, served by cf_server_* with
    continuous batching in the mixed form.  Latency = arrival to result; the
    host builds each hierarchy after its arrival, so it includes setup."""
    import numpy as np
    from paper_2508_11608_gb300.workloads import serving_requests
    reqs = serving_requests(count=args.serve_count)
    rng = np.random.default_rng(20260103)
    gaps = rng.exponential(1.0 / args.serve_rate, len(reqs))
    arrivals = np.cumsum(gaps) - gaps[0]
    srv = cm.Server(hbm_budget_bytes=64 << 30, max_active=32, precision=cm.CF_MIXED)
    ids = [srv.submit(arrival_s=float(a), **k) for k, a in zip(reqs, arrivals)]
    srv.run()
    res = [srv.result(i) for i in ids]
    st = srv.stats()
    lat = np.array([r["latency_s"] for r in res]) * 1e3
    dev = np.array([r["done"] - r["admitted"] for r in res]) * 1e3
    ndof = sum(r["ndof"] for r in res)
    span = max(r["done"] for r in res) - min(r["arrival"] for r in res)
    srv.close()
    return {"value": ndof / span, "unit": "DoF/s", "requests": len(res), "active_dofs": ndof,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "device_latency_ms": {"p50": float(np.percentile(dev, 50)), "p99": float(np.percentile(dev, 99))},
            "worst_true_rel_residual": max(r["true_rel_residual"] for r in res),
            "peak_active": st["peak_active"], "peak_device_gb": st["peak_device_bytes"] / 1e9,
            "arrival_rate_per_s": args.serve_rate, "precision": "mixed",
            "workload": "3D Q2 spheres r in [0.4,0.8] / ellipsoids semi-axes in [0.4,0.8] / tori R=0.6 r=0.2, "
                        "offset <= 0.05, N in {32,48,64,96}, seed 20260102, Poisson arrivals seed 20260103; "
                        "latency includes the host setup after arrival, device_latency is admission to result"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, help="headline configuration (workloads.CONFIGS)")
    ap.add_argument("--extra", nargs="*", default=list(EXTRA), help="further sizes timed after the headline")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-form measurement")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--no-serve", action="store_true", help="skip the served-form measurement")
    ap.add_argument("--serve-count", type=int, default=16)
    ap.add_argument("--serve-rate", type=float, default=0.5, help="Poisson arrivals per second")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
