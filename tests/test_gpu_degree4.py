"""Degree 4 in 2D (beyond the Q3 the paper runs) on the GPU against the
oracle, through the C ABI: disk r = 0.7 on 32², 3 levels.  The closure of a
Q4 patch has 81 > 64 nodes, so the cut patches run the record kernel
(k_cut_warp / k_cut_team) as in 3D Q2.

Tolerances come from the conditioning: the Q4 cut-patch matrices on these
meshes reach cond(A_j) = 3e7, so the library's explicit inverse and the
oracle's LAPACK solve, both backward stable, differ by up to u cond(A_j)
= 7e-9 of the update; FP64 colour steps, smoothing steps and V-cycles are
held to 1e-8, the operator and the transfer to the usual 1e-12 / 1e-13.
In the mixed form FP32 rounding (6e-8) times cond(A_j) leaves the worst
patches' updates with no correct digit, so only its convergence to the FP64
form's residual is checked."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2508_11608_gb300 as cm  # noqa: E402
from paper_2508_11608_gb300 import _lib  # noqa: E402
from paper_2508_11608_gb300.workloads import CONFIGS, problem_kwargs, random_vector  # noqa: E402
from oracle import Hierarchy, Sphere  # noqa: E402

NAME = "disk2d_q4_n32"
DEV = "cuda:0"


def _t(a):
    return torch.tensor(a, dtype=torch.float64, device=DEV)


def _n(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.fixture(scope="module")
def pair():
    c = CONFIGS[NAME]
    pb = cm.Problem(**problem_kwargs(NAME))
    H = Hierarchy(Sphere(c["center"], c["radius"]), c["dim"], c["n_cells"], c["degree"], c["n_levels"])
    yield pb, H
    pb.set_kernel_variant(_lib.CF_VAR_CUT, 0)
    pb.set_kernel_variant(_lib.CF_VAR_INTERIOR, 0)


def test_apply(pair):
    pb, H = pair
    for l in range(pb.n_levels):
        x = random_vector(pb.n_dofs(l), 100 + l)
        y = torch.zeros(pb.n_dofs(l), dtype=torch.float64, device=DEV)
        pb.level_apply(l, _t(x), y)
        assert rel(_n(y), H.levels[l].A @ x) < 1e-12


def _steps(pb, H, cut):
    outs = []
    for l in range(1, pb.n_levels):
        n = pb.n_dofs(l)
        for col in range(1 << pb.dim):
            x0 = random_vector(n, 7 + col)
            b = random_vector(n, 300 + col)
            xg = _t(x0)
            pb.colour_step(l, cut, col, xg, _t(b))
            xo = H.colour_step(l, x0, b, cut, col)
            g = _n(xg)
            assert np.abs(g - xo).max() <= 1e-8 * np.abs(xo - x0).max() + 1e-15 * np.abs(x0).max(), (l, cut, col)
            outs.append(g)
    return outs


def test_interior_colour_steps(pair):
    pb, H = pair
    ref = None
    for v in (1, 2):  # half-warp / block per patch: the same arithmetic
        pb.set_kernel_variant(_lib.CF_VAR_INTERIOR, v)
        outs = _steps(pb, H, False)
        if ref is None:
            ref = outs
        else:
            for a, b in zip(ref, outs):
                assert np.array_equal(a, b)
    pb.set_kernel_variant(_lib.CF_VAR_INTERIOR, 0)


def test_cut_colour_steps_every_variant(pair):
    pb, H = pair
    ref = None
    for v in (0, 1, 2, 3, 4, 5, 6):
        pb.set_kernel_variant(_lib.CF_VAR_CUT, v)
        outs = _steps(pb, H, True)
        if ref is None:
            ref = outs
        else:
            for a, b in zip(ref, outs):
                assert np.array_equal(a, b), v
    pb.set_kernel_variant(_lib.CF_VAR_CUT, 0)


def test_smoothing_transfer_vcycle(pair):
    pb, H = pair
    for l in range(1, pb.n_levels):
        n = pb.n_dofs(l)
        b = random_vector(n, 11)
        for post in (False, True):
            xg = torch.zeros(n, dtype=torch.float64, device=DEV)
            pb.smooth(l, xg, _t(b), post=post)
            assert rel(_n(xg), H.smooth(l, np.zeros(n), b, post=post)) < 1e-8
        r = random_vector(n, 21)
        bc = torch.zeros(pb.n_dofs(l - 1), dtype=torch.float64, device=DEV)
        pb.restrict(l, _t(r), bc)
        assert rel(_n(bc), H.P[l].T @ r) < 1e-13
    r = random_vector(pb.n_dofs(), 41)
    z = torch.zeros(pb.n_dofs(), dtype=torch.float64, device=DEV)
    pb.vcycle(_t(r), z)
    assert rel(_n(z), H.vcycle(r)) < 1e-8


def test_solves(pair):
    pb, H = pair
    n = pb.n_dofs()
    b = torch.zeros(n, dtype=torch.float64, device=DEV)
    pb.rhs(b)
    bo = H.rhs()
    assert rel(_n(b), bo) < 1e-13
    xo, it, _ = H.pcg(bo, rtol=1e-8)
    x = torch.zeros(n, dtype=torch.float64, device=DEV)
    info = pb.solve(b, x, rtol=1e-8)
    assert abs(info["iterations"] - it) <= 1
    assert info["true_rel_residual"] <= 1.01e-8
    assert np.linalg.norm(_n(x) - xo) <= 1e-7 * np.linalg.norm(xo)
    pb.set_precision(cm.CF_MIXED)
    try:
        xm = torch.zeros(n, dtype=torch.float64, device=DEV)
        im = pb.solve(b, xm, rtol=1e-8)
    finally:
        pb.set_precision(cm.CF_FP64)
    assert im["true_rel_residual"] <= 1.01e-8
    print(f"Q4 32^2: FP64 {info['iterations']} iterations (oracle {it}), mixed {im['iterations']}")


def test_batched_q4_equals_solo():
    from paper_2508_11608_gb300.workloads import flower_batch
    specs = flower_batch(count=3, seed=11, sizes=(16, 32), degrees=(4,), coarsest=8)
    pbs = [cm.Problem(**k) for k in specs]
    bs, xs, alone = [], [], []
    for pb in pbs:
        b = torch.zeros(pb.n_dofs(), dtype=torch.float64, device=DEV)
        pb.rhs(b)
        x = torch.zeros_like(b)
        info = pb.solve(b, x, rtol=1e-8)
        alone.append((_n(x), info))
        bs.append(b)
        xs.append(torch.zeros_like(b))
    bt = cm.Batch(pbs)
    infos = bt.solve(bs, xs, rtol=1e-8, precision=cm.CF_FP64)
    for (xa, ia), x, ib in zip(alone, xs, infos):
        assert ib["iterations"] == ia["iterations"]
        assert np.abs(_n(x) - xa).max() <= 1e-13 * np.abs(xa).max()


def test_served_q4_requests_equal_solo():
    reqs = [dict(dim=2, n_cells=32, n_levels=3, degree=4,
                 levelset={"kind": "sphere", "center": [0.031, 0.017], "radius": 0.7}),
            dict(dim=2, n_cells=16, n_levels=2, degree=4,
                 levelset={"kind": "flower", "center": [0.01, -0.02], "lobes": 5, "phase": 0.3})]
    srv = cm.Server(hbm_budget_bytes=8 << 30, max_active=4, precision=cm.CF_FP64, keep_solutions=True)
    ids = [srv.submit(k["dim"], k["n_cells"], k["n_levels"], k["degree"], k["levelset"], arrival_s=0.0) for k in reqs]
    srv.run()
    for rid, k in zip(ids, reqs):
        r = srv.result(rid)
        pb = cm.Problem(**k)
        b = torch.zeros(pb.n_dofs(), dtype=torch.float64, device=DEV)
        pb.rhs(b)
        x = torch.zeros_like(b)
        info = pb.solve(b, x, rtol=1e-8)
        assert r["iterations"] == info["iterations"] > 0
        xa = _n(x)
        assert np.abs(r["x"] - xa).max() <= 1e-13 * np.abs(xa).max()
