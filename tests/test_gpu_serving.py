"""Served form: requests arriving over time are admitted by HBM footprint
and solved with continuous batching; each result equals the same problem
solved alone (same iterations, same iterate), and admission respects the
budget."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2508_11608_gb300 as cm  # noqa: E402
from paper_2508_11608_gb300.workloads import rotation  # noqa: E402

DEV = "cuda:0"

REQS = [
    dict(dim=3, n_cells=16, n_levels=3, degree=2,
         levelset={"kind": "sphere", "center": [0.02, 0.01, -0.03], "radius": 0.6}),
    dict(dim=3, n_cells=16, n_levels=2, degree=2,
         levelset={"kind": "ellipsoid", "center": [0.01, 0.0, 0.02], "axes": [0.7, 0.5, 0.6],
                   "rot": rotation(0.3, 0.2, 0.1)}),
    dict(dim=3, n_cells=16, n_levels=2, degree=2,
         levelset={"kind": "torus", "center": [0.0, 0.02, 0.01], "rot": rotation(0.5, 0.9, 0.0),
                   "major": 0.6, "minor": 0.2}),
    dict(dim=3, n_cells=24, n_levels=3, degree=2,
         levelset={"kind": "sphere", "center": [-0.02, 0.03, 0.0], "radius": 0.75}),
    dict(dim=3, n_cells=8, n_levels=2, degree=2,
         levelset={"kind": "sphere", "center": [0.0, 0.0, 0.01], "radius": 0.45}),
]


def _alone(k, prec):
    pb = cm.Problem(**k)
    n = pb.n_dofs()
    b = torch.zeros(n, dtype=torch.float64, device=DEV)
    x = torch.zeros_like(b)
    pb.rhs(b)
    pb.set_precision(prec)
    info = pb.solve(b, x, rtol=1e-8)
    torch.cuda.synchronize()
    return x.cpu().numpy(), info


@pytest.mark.parametrize("prec", [cm.CF_FP64, cm.CF_MIXED])
def test_each_result_same_alone_and_in_the_mix(prec):
    srv = cm.Server(hbm_budget_bytes=40 << 30, max_active=16, precision=prec, keep_solutions=True)
    ids = [srv.submit(k["dim"], k["n_cells"], k["n_levels"], k["degree"], k["levelset"], arrival_s=0.02 * i)
           for i, k in enumerate(REQS)]
    srv.run()
    st = srv.stats()
    assert st["peak_active"] >= 2  # requests overlapped on the device
    for rid, k in zip(ids, REQS):
        r = srv.result(rid)
        xa, ia = _alone(k, prec)
        assert r["iterations"] == ia["iterations"]
        assert np.abs(r["x"] - xa).max() <= 1e-13 * np.abs(xa).max()
        assert r["true_rel_residual"] <= 1.01e-8
        assert r["done"] >= r["admitted"] >= r["arrival"]


def test_admission_respects_budget():
    # a budget that holds one of these problems at a time
    one = cm.Problem(**REQS[0])
    del one
    srv = cm.Server(hbm_budget_bytes=300 << 20, max_active=16, precision=cm.CF_FP64)
    ids = [srv.submit(k["dim"], k["n_cells"], k["n_levels"], k["degree"], k["levelset"], arrival_s=0.0)
           for k in REQS[:3]]
    srv.run()
    st = srv.stats()
    assert st["peak_device_bytes"] <= 300 << 20
    for rid in ids:
        assert srv.result(rid)["true_rel_residual"] <= 1.01e-8


def test_request_larger_than_budget_fails_cleanly():
    srv = cm.Server(hbm_budget_bytes=1 << 20, max_active=4, precision=cm.CF_FP64)
    rid = srv.submit(**{k: v for k, v in REQS[0].items()}, arrival_s=0.0)
    srv.run()
    with pytest.raises(cm.CutmgError) as e:
        srv.result(rid)
    assert "budget" in str(e.value)


def test_footprint_estimate_covers_the_device_allocation():
    k = dict(dim=3, n_cells=32, n_levels=4, degree=2, center=[0.05, 0.03, 0.02], radius=0.7)
    est = cm.Problem(**k, host_only=True).footprint()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    pb = cm.Problem(**k)
    b = torch.zeros(pb.n_dofs(), dtype=torch.float64, device=DEV)
    x = torch.zeros_like(b)
    pb.rhs(b)
    pb.solve(b, x, rtol=1e-8)  # graphs and CG scratch allocated
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    used = free0 - free1 - 2 * b.numel() * 8
    assert 0.5 * est <= used <= 1.25 * est + (64 << 20)
