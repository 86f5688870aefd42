"""Run and time solves of one workload (also the driver for profiler runs,
for example: ncu --metrics gpu__time_duration.sum --clock-control none --csv
python -m paper_2508_11608_gb300.profile_solve ball3d_q2_n64 fp64 1).

Arguments: workload name (paper_2508_11608_gb300.workloads.CONFIGS),
precision (fp64 | mixed | both), number of solves.  Prints the host setup
time, the solve info and, over the solves after the first, the CUDA-event
time per solve and DoF/s (inputs resident on the device)."""

import sys
import time

import torch

import paper_2508_11608_gb300 as cm
from paper_2508_11608_gb300.workloads import problem_kwargs


def main(argv):
    name = argv[1] if len(argv) > 1 else "ball3d_q2_n64"
    which = argv[2] if len(argv) > 2 else "fp64"
    precs = {"fp64": [cm.CF_FP64], "mixed": [cm.CF_MIXED], "both": [cm.CF_FP64, cm.CF_MIXED]}[which]
    solves = int(argv[3]) if len(argv) > 3 else 2
    t0 = time.perf_counter()
    pb = cm.Problem(**problem_kwargs(name))
    setup_s = time.perf_counter() - t0
    n = pb.n_dofs()
    b = torch.zeros(n, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    pb.rhs(b)
    stream = torch.cuda.current_stream()
    for prec in precs:
        pb.set_precision(prec)
        ms = []
        for k in range(solves):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = pb.solve(b, x, rtol=1e-8)
            e1.record(stream)
            torch.cuda.synchronize()
            if k > 0:
                ms.append(e0.elapsed_time(e1))
        label = "mixed" if prec == cm.CF_MIXED else "fp64"
        print(name, "precision", label, "dofs", n, "setup_s", round(setup_s, 2), info, flush=True)
        if ms:
            avg = sum(ms) / len(ms)
            print(f"  ms_per_solve {avg:.3f} dof_per_s {n / (avg * 1e-3):.4e} over {len(ms)} solves", flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv))
