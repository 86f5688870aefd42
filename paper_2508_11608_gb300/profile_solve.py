"""Run a few solves of one workload, for profiling the library under a
profiler (for example: ncu --metrics gpu__time_duration.sum --clock-control
none --csv python -m paper_2508_11608_gb300.profile_solve ball3d_q2_n64 fp64 2).

Arguments: workload name (paper_2508_11608_gb300.workloads.CONFIGS),
precision (fp64 | mixed), number of solves."""

import sys

import torch

import paper_2508_11608_gb300 as cm
from paper_2508_11608_gb300.workloads import problem_kwargs


def main(argv):
    name = argv[1] if len(argv) > 1 else "ball3d_q2_n64"
    prec = cm.CF_MIXED if (len(argv) > 2 and argv[2] == "mixed") else cm.CF_FP64
    solves = int(argv[3]) if len(argv) > 3 else 2
    pb = cm.Problem(**problem_kwargs(name))
    n = pb.n_dofs()
    b = torch.zeros(n, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    pb.rhs(b)
    pb.set_precision(prec)
    for _ in range(solves):
        info = pb.solve(b, x, rtol=1e-8)
    torch.cuda.synchronize()
    print(name, "precision", prec, "dofs", n, info)
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv))
