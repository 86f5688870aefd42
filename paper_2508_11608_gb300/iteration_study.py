"""Iteration counts of the V-cycle (Sec. 2.2) used three ways, on the 2D
setting of the paper's experiments (Sec. 4): the circle of radius 1 on
[-1.21, 1.21]^2, Q1/Q2/Q3, coarsest mesh 4 x 4, residual reduction 1e-9.
Each result line (JSON) carries the iterations and the fractional count
n_frac = n_it * (-8) / log10(||r_n|| / ||r_0||) the paper uses for
fine-grained comparisons.

  python -m paper_2508_11608_gb300.iteration_study refine [max_cells] [fp64|mixed]
      CG, GMRES(30) and the V-cycle iteration under mesh refinement (n_c = 2)
  python -m paper_2508_11608_gb300.iteration_study nc [cells]
      GMRES and the V-cycle iteration for n_c = 1..4 cut sweeps
  python -m paper_2508_11608_gb300.iteration_study ghost [cells]
      GMRES for ghost-penalty factors: gamma_1 over [0.05, 0.15] for Q1;
      Q2 / Q3 vary gamma_2 / gamma_3 with the lower factors at the best
      value found for the lower degree
  python -m paper_2508_11608_gb300.iteration_study smoother [max_cells]
      GMRES with the vertex-patch smoother against the degree-5 Chebyshev
      smoother under refinement"""

import json
import math
import sys

import torch

import paper_2508_11608_gb300 as cm


def _problem(p, n, n_c=2, gammas=(0.1, 0.1, 0.1, 0.0), prec=cm.CF_FP64, smoother=cm.CF_SMOOTHER_MVS):
    levels = int(math.log2(n // 4)) + 1
    pb = cm.Problem(2, n, levels, p, center=[0.0, 0.0], radius=1.0, lo=-1.21, hi=1.21, n_c=n_c,
                    gamma_ghost=tuple(gammas), smoother=smoother)
    pb.set_precision(prec)
    b = torch.zeros(pb.n_dofs(), dtype=torch.float64, device="cuda")
    pb.rhs(b)
    return pb, b, levels


def _run(solver, b, rtol=1e-9):
    x = torch.zeros_like(b)
    info = solver(b, x, rtol=rtol, maxit=500, allow_noconv=True)
    it, rel = info["iterations"], info["rel_residual"]
    nfrac = it * -8.0 / math.log10(rel) if 0.0 < rel < 1.0 else float("nan")
    return it, round(nfrac, 2)


def refine(nmax, prec):
    for p in (1, 2, 3):
        n = 8
        while n <= nmax:
            pb, b, levels = _problem(p, n, prec=prec)
            out = {"mode": "refine", "degree": p, "cells": n, "levels": levels, "dofs": pb.n_dofs()}
            for name, solver in (("cg", pb.solve), ("gmres", pb.solve_gmres), ("vcycle", pb.solve_vcycle)):
                out[name], out[name + "_nfrac"] = _run(solver, b)
            print(json.dumps(out), flush=True)
            pb.close()
            n *= 2


def n_c_sweep(n):
    for p in (1, 2, 3):
        for n_c in (1, 2, 3, 4):
            pb, b, _ = _problem(p, n, n_c=n_c)
            out = {"mode": "nc", "degree": p, "cells": n, "n_c": n_c}
            out["gmres"], out["gmres_nfrac"] = _run(pb.solve_gmres, b)
            out["vcycle"], out["vcycle_nfrac"] = _run(pb.solve_vcycle, b)
            print(json.dumps(out), flush=True)
            pb.close()


def ghost_sweep(n):
    best = [0.1, 0.1, 0.1]
    for p in (1, 2, 3):
        results = []
        for g in (0.05, 0.075, 0.1, 0.125, 0.15):
            gam = list(best) + [0.0]
            gam[p - 1] = g
            pb, b, _ = _problem(p, n, gammas=gam)
            it, nfrac = _run(pb.solve_gmres, b)
            results.append((nfrac, g))
            print(json.dumps({"mode": "ghost", "degree": p, "cells": n, "gammas": gam[:p], "gmres": it,
                              "gmres_nfrac": nfrac}), flush=True)
            pb.close()
        best[p - 1] = min(results)[1]
    print(json.dumps({"mode": "ghost", "best_gammas": best}), flush=True)


def smoother_sweep(nmax):
    for p in (1, 2, 3):
        n = 8
        while n <= nmax:
            out = {"mode": "smoother", "degree": p, "cells": n}
            for name, sm in (("mvs", cm.CF_SMOOTHER_MVS), ("chebyshev", cm.CF_SMOOTHER_CHEBYSHEV)):
                pb, b, _ = _problem(p, n, smoother=sm)
                out[name], out[name + "_nfrac"] = _run(pb.solve_gmres, b)
                pb.close()
            print(json.dumps(out), flush=True)
            n *= 2


def main(argv):
    mode = argv[1] if len(argv) > 1 else "refine"
    if mode == "refine":
        nmax = int(argv[2]) if len(argv) > 2 else 256
        prec = cm.CF_MIXED if (len(argv) > 3 and argv[3] == "mixed") else cm.CF_FP64
        refine(nmax, prec)
    elif mode == "nc":
        n_c_sweep(int(argv[2]) if len(argv) > 2 else 128)
    elif mode == "ghost":
        ghost_sweep(int(argv[2]) if len(argv) > 2 else 128)
    elif mode == "smoother":
        smoother_sweep(int(argv[2]) if len(argv) > 2 else 256)
    else:
        raise SystemExit("mode: refine | nc | ghost | smoother")
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv))
