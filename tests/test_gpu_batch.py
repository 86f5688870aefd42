"""Batched form: problems solved together through cf_batch_* give the same
iterates as each solved alone through cf_solve (same floating-point
operations), for mixed degrees, sizes and shapes, in both precisions."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2508_11608_gb300 as cm  # noqa: E402
from paper_2508_11608_gb300.workloads import flower_batch, problem_kwargs  # noqa: E402

DEV = "cuda:0"


def _solve_alone(pb, prec):
    n = pb.n_dofs()
    b = torch.zeros(n, dtype=torch.float64, device=DEV)
    x = torch.zeros_like(b)
    pb.rhs(b)
    pb.set_precision(prec)
    info = pb.solve(b, x, rtol=1e-8)
    pb.set_precision(cm.CF_FP64)
    torch.cuda.synchronize()
    return x.cpu().numpy(), info


@pytest.mark.parametrize("prec", [cm.CF_FP64, cm.CF_MIXED])
def test_batch_matches_single_solves_2d(prec):
    specs = flower_batch(count=6, seed=7, sizes=(16, 32), degrees=(2, 3), coarsest=8)
    pbs = [cm.Problem(**k) for k in specs]
    alone = [_solve_alone(pb, prec) for pb in pbs]
    bt = cm.Batch(pbs)
    bs, xs = [], []
    for pb in pbs:
        b = torch.zeros(pb.n_dofs(), dtype=torch.float64, device=DEV)
        pb.rhs(b)
        bs.append(b)
        xs.append(torch.zeros_like(b))
    infos = bt.solve(bs, xs, rtol=1e-8, precision=prec)
    torch.cuda.synchronize()
    for (xa, ia), x, ib in zip(alone, xs, infos):
        assert ib["iterations"] == ia["iterations"]
        xb = x.cpu().numpy()
        assert np.abs(xb - xa).max() <= 1e-13 * np.abs(xa).max()
        assert ib["true_rel_residual"] <= 1.01e-8


def test_batch_3d_mixed_shapes():
    specs = [problem_kwargs("ball3d_q2_n16"),
             dict(dim=3, n_cells=16, n_levels=2, degree=2,
                  levelset={"kind": "torus", "center": [0.01, 0.02, 0.0], "rot": np.eye(3).tolist(),
                            "major": 0.6, "minor": 0.2}),
             dict(dim=3, n_cells=8, n_levels=2, degree=1,
                  levelset={"kind": "ellipsoid", "center": [0.0, 0.01, 0.02], "axes": [0.7, 0.5, 0.6],
                            "rot": np.eye(3).tolist()})]
    pbs = [cm.Problem(**k) for k in specs]
    alone = [_solve_alone(pb, cm.CF_FP64) for pb in pbs]
    bt = cm.Batch(pbs)
    bs, xs = [], []
    for pb in pbs:
        b = torch.zeros(pb.n_dofs(), dtype=torch.float64, device=DEV)
        pb.rhs(b)
        bs.append(b)
        xs.append(torch.zeros_like(b))
    infos = bt.solve(bs, xs, rtol=1e-8)
    torch.cuda.synchronize()
    for (xa, ia), x, ib in zip(alone, xs, infos):
        assert ib["iterations"] == ia["iterations"]
        assert np.abs(x.cpu().numpy() - xa).max() <= 1e-13 * np.abs(xa).max()


def test_batch_launches_do_not_grow_with_count():
    specs = flower_batch(count=12, seed=9, sizes=(16,), degrees=(2,), coarsest=8)
    pbs = [cm.Problem(**k) for k in specs]
    counts = []
    for k in (2, 12):
        bt = cm.Batch(pbs[:k])
        bs, xs = [], []
        for pb in pbs[:k]:
            b = torch.zeros(pb.n_dofs(), dtype=torch.float64, device=DEV)
            pb.rhs(b)
            bs.append(b)
            xs.append(torch.zeros_like(b))
        l0 = bt.launch_count()
        infos = bt.solve(bs, xs)
        its = max(i["iterations"] for i in infos)
        counts.append((bt.launch_count() - l0) / max(its, 1))
    assert counts[1] <= 1.3 * counts[0]
