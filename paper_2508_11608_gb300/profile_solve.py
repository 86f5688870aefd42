"""Run and time solves of one workload (also the driver for profiler runs,
for example: ncu --metrics gpu__time_duration.sum --clock-control none --csv
python -m paper_2508_11608_gb300.profile_solve ball3d_q2_n64 fp64 1).

    python -m paper_2508_11608_gb300.profile_solve WORKLOAD [fp64|mixed|both] [SOLVES]
        [--interior V] [--cut V] [--families [--levels]]

WORKLOAD names paper_2508_11608_gb300.workloads.CONFIGS.  Prints the host
setup time, the solve info and, over the solves after the first, the
CUDA-event time per solve and DoF/s (inputs resident on the device).
--interior / --cut force a launch variant (cf_set_kernel_variant); with
--families every kernel family is event-timed in one more pass of solves:
summed launch time, launches, and the achieved rate of its algorithmic
flops and bytes."""

import argparse
import sys
import time

import torch

import paper_2508_11608_gb300 as cm
from paper_2508_11608_gb300 import _lib
from paper_2508_11608_gb300.workloads import problem_kwargs

FAMILIES = {_lib.CF_K_CUT_SOLVE: "cut-patch step", _lib.CF_K_INTERIOR: "interior-patch step",
            _lib.CF_K_APPLY_BULK: "operator, bulk", _lib.CF_K_APPLY_BND: "operator, boundary",
            _lib.CF_K_FACE_MOMENTS: "ghost-face moments"}


def main(argv):
    ap = argparse.ArgumentParser()
    ap.add_argument("workload", nargs="?", default="ball3d_q2_n64")
    ap.add_argument("precision", nargs="?", default="fp64", choices=["fp64", "mixed", "both"])
    ap.add_argument("solves", nargs="?", type=int, default=2)
    ap.add_argument("--interior", type=int, default=0)
    ap.add_argument("--cut", type=int, default=0)
    ap.add_argument("--families", action="store_true")
    ap.add_argument("--levels", action="store_true", help="with --families: one line per level")
    a = ap.parse_args(argv[1:])
    precs = {"fp64": [cm.CF_FP64], "mixed": [cm.CF_MIXED], "both": [cm.CF_FP64, cm.CF_MIXED]}[a.precision]
    t0 = time.perf_counter()
    pb = cm.Problem(**problem_kwargs(a.workload))
    setup_s = time.perf_counter() - t0
    pb.set_kernel_variant(_lib.CF_VAR_INTERIOR, a.interior)
    pb.set_kernel_variant(_lib.CF_VAR_CUT, a.cut)
    n = pb.n_dofs()
    b = torch.zeros(n, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    pb.rhs(b)
    stream = torch.cuda.current_stream()
    for prec in precs:
        pb.set_precision(prec)
        label = "mixed" if prec == cm.CF_MIXED else "fp64"
        ms = []
        for k in range(a.solves):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = pb.solve(b, x, rtol=1e-8)
            e1.record(stream)
            torch.cuda.synchronize()
            if k > 0:
                ms.append(e0.elapsed_time(e1))
        print(a.workload, "precision", label, "dofs", n, "setup_s", round(setup_s, 2), info, flush=True)
        if ms:
            avg = sum(ms) / len(ms)
            print(f"  ms_per_solve {avg:.3f} dof_per_s {n / (avg * 1e-3):.4e} over {len(ms)} solves", flush=True)
        if a.families:
            for fam, name in FAMILIES.items():
                for lev in (range(pb.n_levels) if a.levels else [-1]):
                    pb.profile_start(fam, lev)
                    pb.solve(b, x, rtol=1e-8)
                    pr = pb.profile_read()
                    if pr["launches"] == 0:
                        continue
                    per = pr["ms"] / pr["launches"]
                    where = f"L{lev}" if lev >= 0 else "all"
                    print(f"  {label} {name:22s} {where:3s} {pr['ms']:9.3f} ms  {pr['launches']:5d} launches  "
                          f"{per * 1e3:8.2f} us/launch  {pr['bytes'] / (pr['ms'] * 1e-3) / 1e9:8.1f} GB/s  "
                          f"{pr['flops'] / (pr['ms'] * 1e-3) / 1e12:7.3f} TFLOP/s  "
                          f"{pr['bytes'] / pr['launches'] / 1e6:8.2f} MB/launch (algorithmic)", flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv))
