"""Served-form study: a seeded stream of 3D Q2 solve requests (spheres,
ellipsoids, tori on 32^3 .. 96^3 meshes) served with continuous batching
(cf_server_*), at Poisson arrival rates of 0.5, 0.8 and 1.0 times the
measured capacity, in the mixed and the FP64 form, to the same 1e-8 residual.

    python -m paper_2508_11608_gb300.serve_study [--requests 500] [--burst 48]
        [--rates 0.5 0.8 1.0] [--out FILE]

Capacity: requests per second completed when `--burst` requests of the same
stream all arrive at once (mixed form; the host setup after arrival, the
admission by HBM footprint and the device solves all count).  Each run then
submits `--requests` requests with exponential inter-arrival gaps (seed
20260103) at rate x capacity.  Latency = arrival to result (host setup
included); device latency = admission to result.  Prints one JSON object per
run and writes them all to --out."""

import argparse
import json
import sys
import time

import numpy as np

import paper_2508_11608_gb300 as cm
from paper_2508_11608_gb300.workloads import serving_requests


def serve(reqs, arrivals, precision, budget=96 << 30, max_active=32):
    srv = cm.Server(hbm_budget_bytes=budget, max_active=max_active, precision=precision)
    ids = [srv.submit(arrival_s=float(a), **k) for k, a in zip(reqs, arrivals)]
    t0 = time.perf_counter()
    srv.run()
    wall = time.perf_counter() - t0
    res = [srv.result(i) for i in ids]
    st = srv.stats()
    srv.close()
    lat = np.array([r["latency_s"] for r in res]) * 1e3
    dev = np.array([r["done"] - r["admitted"] for r in res]) * 1e3
    ndof = sum(r["ndof"] for r in res)
    span = max(r["done"] for r in res) - min(r["arrival"] for r in res)
    return {"requests": len(res), "active_dofs": int(ndof), "dof_per_s": ndof / span,
            "requests_per_s": len(res) / span, "span_s": span, "wall_s": wall,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "device_latency_ms": {"p50": float(np.percentile(dev, 50)), "p99": float(np.percentile(dev, 99))},
            "iterations_max": int(max(r["iterations"] for r in res)),
            "worst_true_rel_residual": float(max(r["true_rel_residual"] for r in res)),
            "peak_active": st["peak_active"], "peak_device_gb": st["peak_device_bytes"] / 1e9}


def main(argv):
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=500)
    ap.add_argument("--burst", type=int, default=48)
    ap.add_argument("--rates", type=float, nargs="*", default=[0.5, 0.8, 1.0])
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv[1:])
    reqs = serving_requests(count=a.requests)
    out = []
    burst = serve(reqs[:a.burst], np.zeros(a.burst), cm.CF_MIXED)
    capacity = burst["requests_per_s"]
    out.append({"run": "capacity (burst, mixed)", **burst})
    print(json.dumps(out[-1]), flush=True)
    for rate in a.rates:
        lam = rate * capacity
        rng = np.random.default_rng(20260103)
        gaps = rng.exponential(1.0 / lam, len(reqs))
        arrivals = np.cumsum(gaps) - gaps[0]
        for prec, name in ((cm.CF_MIXED, "mixed"), (cm.CF_FP64, "fp64")):
            r = serve(reqs, arrivals, prec)
            out.append({"run": f"{name}, lambda = {rate} x capacity", "precision": name,
                        "arrival_rate_per_s": lam, **r})
            print(json.dumps(out[-1]), flush=True)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(out, f, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv))
