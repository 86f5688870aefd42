"""Writes tests/golden/ball3d_q2_n64_pcg.npz: the oracle's PCG solution of the
3D Q2 ball problem on the 64^3 background mesh (5 levels, rtol 1e-8), the
full-vector parity target of the GPU solve at that size.

Calls only the oracle (assembled operator, explicit patch matrices, the same
V-cycle inside CG; Sec. 2.2 and Sec. 2.3).  The problem definition is written
out here rather than imported, so the stored values depend on nothing but
oracle/.

    python tests/golden/make_ball64_solution.py

Stores: x (FP64, DoF order = increasing lattice index), the right-hand side's
norm, the CG iteration count, the recursive and the true relative residual.
"""

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import Hierarchy, Sphere  # noqa: E402

# ball r = 0.7 at (0.05, 0.03, 0.02) cut from [-1, 1]^3, 64^3 cells, Q2, 5 levels
CENTER, RADIUS, DIM, N, DEGREE, LEVELS, RTOL = [0.05, 0.03, 0.02], 0.7, 3, 64, 2, 5, 1e-8
OUT = os.path.join(HERE, "ball3d_q2_n64_pcg.npz")


def main():
    t0 = time.time()
    H = Hierarchy(Sphere(CENTER, RADIUS), DIM, N, DEGREE, LEVELS)
    t1 = time.time()
    b = H.rhs()
    x, it, hist = H.pcg(b, rtol=RTOL)
    t2 = time.time()
    A = H.levels[-1].A
    bn = float(np.linalg.norm(b))
    true_rel = float(np.linalg.norm(b - A @ x) / bn)
    np.savez_compressed(OUT, x=x, b_norm=bn, iterations=it, rel_residual=hist[-1] / bn,
                        true_rel_residual=true_rel)
    print(f"{x.size} DoFs, {it} iterations, true rel residual {true_rel:.3e}; "
          f"setup {t1 - t0:.1f} s, solve {t2 - t1:.1f} s -> {OUT}")


if __name__ == "__main__":
    main()
