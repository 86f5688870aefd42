"""The CUDA path against the oracle beyond the default parameters and shapes,
through the C ABI:
  * the number n_c of cut-patch sweeps per smoothing step (eq.
    "smoother-split"; Sec. 4 studies n_c = 1..4) and the ghost-penalty factor
    gamma_k (eq. "cutfem-ghost"; Sec. 4 sweeps it), on 2D Q3 and 3D Q2;
  * one instance of a batch of 2D flowers and one served 3D request (an
    ellipsoid and a torus) compared with the oracle directly, not only with
    the GPU's own single-problem solve.
Tolerances as in test_gpu_parity: smoothing steps and V-cycles 1e-10 (FP64),
solves CG iterations within one and relative L2 1e-10."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2508_11608_gb300 as cm  # noqa: E402
from paper_2508_11608_gb300.workloads import flower_batch, random_vector  # noqa: E402
from oracle import Hierarchy  # noqa: E402
from oracle.levelset import Ellipsoid, Flower, Sphere, Torus  # noqa: E402

DEV = "cuda:0"


def _t(a):
    return torch.tensor(a, dtype=torch.float64, device=DEV)


def _n(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _oracle_ls(spec):
    k = spec["kind"]
    if k == "sphere":
        return Sphere(spec["center"], spec["radius"])
    if k == "flower":
        return Flower(spec["center"], spec["lobes"], spec["phase"], spec.get("base", 0.6), spec.get("amplitude", 0.1))
    if k == "ellipsoid":
        return Ellipsoid(spec["center"], spec["axes"], np.asarray(spec["rot"]))
    if k == "torus":
        return Torus(spec["center"], np.asarray(spec["rot"]), spec["major"], spec["minor"])
    raise ValueError(k)


def _check_solve(pb, H):
    n = pb.n_dofs()
    b = torch.zeros(n, dtype=torch.float64, device=DEV)
    pb.rhs(b)
    bo = H.rhs()
    assert np.abs(_n(b) - bo).max() <= 1e-13 * np.abs(bo).max()
    r = random_vector(n, 41)
    z = torch.zeros(n, dtype=torch.float64, device=DEV)
    pb.vcycle(_t(r), z)
    zo = H.vcycle(r)
    assert np.abs(_n(z) - zo).max() <= 1e-10 * np.abs(zo).max()
    x = torch.zeros(n, dtype=torch.float64, device=DEV)
    info = pb.solve(b, x, rtol=1e-8)
    xo, it, _ = H.pcg(bo, rtol=1e-8)
    assert abs(info["iterations"] - it) <= 1, (info["iterations"], it)
    assert np.linalg.norm(_n(x) - xo) <= 1e-10 * np.linalg.norm(xo)
    return info["iterations"], it


CASES = [
    (2, 32, 3, 3, [0.031, 0.017]),
    (3, 16, 3, 2, [0.05, 0.03, 0.02]),
]


@pytest.mark.parametrize("dim,N,L,p,c", CASES)
@pytest.mark.parametrize("n_c", [1, 3])
def test_cut_sweeps_per_step_match_the_oracle(dim, N, L, p, c, n_c):
    pb = cm.Problem(dim, N, L, p, center=c, radius=0.7, n_c=n_c)
    H = Hierarchy(Sphere(c, 0.7), dim, N, p, L, n_c=n_c)
    l = pb.n_levels - 1
    bl = random_vector(pb.n_dofs(l), 11)
    for post in (False, True):
        xg = torch.zeros(pb.n_dofs(l), dtype=torch.float64, device=DEV)
        pb.smooth(l, xg, _t(bl), post=post)
        xo = H.smooth(l, np.zeros(pb.n_dofs(l)), bl, post=post)
        assert np.abs(_n(xg) - xo).max() <= 1e-11 * np.abs(xo).max()
    _check_solve(pb, H)


@pytest.mark.parametrize("dim,N,L,p,c", CASES)
def test_ghost_penalty_factor_matches_the_oracle(dim, N, L, p, c):
    g = [0.05] * p
    pb = cm.Problem(dim, N, L, p, center=c, radius=0.7, gamma_ghost=tuple(g) + (0.0,) * (4 - p))
    H = Hierarchy(Sphere(c, 0.7), dim, N, p, L, gammas=g)
    l = pb.n_levels - 1
    x = random_vector(pb.n_dofs(l), 5)
    y = torch.zeros(pb.n_dofs(l), dtype=torch.float64, device=DEV)
    pb.level_apply(l, _t(x), y)
    yo = H.levels[l].A @ x
    assert np.abs(_n(y) - yo).max() <= 1e-12 * np.abs(yo).max()
    _check_solve(pb, H)


def test_batched_flower_instance_matches_the_oracle():
    """One 2D flower of a mixed batch (Q2 and Q3, two sizes), batched solve
    against the oracle's PCG of that flower."""
    specs = flower_batch(count=4, seed=7, sizes=(16, 32), degrees=(2, 3), coarsest=8)
    pbs = [cm.Problem(**k) for k in specs]
    bt = cm.Batch(pbs)
    bs, xs = [], []
    for pb in pbs:
        b = torch.zeros(pb.n_dofs(), dtype=torch.float64, device=DEV)
        pb.rhs(b)
        bs.append(b)
        xs.append(torch.zeros_like(b))
    infos = bt.solve(bs, xs, rtol=1e-8, precision=cm.CF_FP64)
    torch.cuda.synchronize()
    for i in (0, 3):
        k = specs[i]
        H = Hierarchy(_oracle_ls(k["levelset"]), 2, k["n_cells"], k["degree"], k["n_levels"])
        xo, it, _ = H.pcg(H.rhs(), rtol=1e-8)
        assert abs(infos[i]["iterations"] - it) <= 1
        assert np.linalg.norm(_n(xs[i]) - xo) <= 1e-10 * np.linalg.norm(xo)


@pytest.mark.parametrize("spec", [
    {"kind": "ellipsoid", "center": [0.02, -0.01, 0.03], "axes": [0.7, 0.5, 0.6],
     "rot": [[0.8, 0.6, 0.0], [-0.6, 0.8, 0.0], [0.0, 0.0, 1.0]]},
    {"kind": "torus", "center": [0.01, 0.02, 0.0], "rot": [[1, 0, 0], [0, 0.6, 0.8], [0, -0.8, 0.6]],
     "major": 0.6, "minor": 0.2},
])
def test_served_request_matches_the_oracle(spec):
    """A 3D Q2 request through the served form (continuous batching,
    FP64), its solution against the oracle's PCG of the same problem."""
    N, L = 16, 2
    srv = cm.Server(hbm_budget_bytes=8 << 30, max_active=4, precision=cm.CF_FP64, keep_solutions=True)
    rid = srv.submit(dim=3, n_cells=N, n_levels=L, degree=2, levelset=spec, arrival_s=0.0)
    srv.run()
    res = srv.result(rid)
    srv.close()
    H = Hierarchy(_oracle_ls(spec), 3, N, 2, L)
    xo, it, _ = H.pcg(H.rhs(), rtol=1e-8)
    assert abs(res["iterations"] - it) <= 1
    assert np.linalg.norm(res["x"] - xo) <= 1e-10 * np.linalg.norm(xo)
