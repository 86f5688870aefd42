"""CUDA path against the oracle, element by element, through the C ABI.

Tolerances: FP64 kernels 1e-12 relative per step (rounding of sums of a few
hundred terms); the solve 1e-10 relative L2 and CG iterations within one;
FP32 kernels (mixed form) 2e-5 relative per step (single rounding ~6e-8
amplified by the conditioning of the local solves), except the interior-patch
step of the mixed form, whose dense map runs on the tensor cores with TF32
operands (unit roundoff 2^-11 = 4.9e-4; 2e-2 of the update, as the variant
tests)."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2508_11608_gb300 as cm  # noqa: E402
from paper_2508_11608_gb300.workloads import CONFIGS, problem_kwargs, random_vector  # noqa: E402
from oracle import Hierarchy, Sphere  # noqa: E402

NAMES = ["disk2d_q2_n32", "ball3d_q2_n16", "disk2d_q3_n32", "ball3d_q1_n16"]
DEV = "cuda:0"


def _t(a):
    return torch.tensor(a, dtype=torch.float64, device=DEV)


def _n(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.fixture(scope="module", params=NAMES)
def pair(request):
    c = CONFIGS[request.param]
    pb = cm.Problem(**problem_kwargs(request.param))
    H = Hierarchy(Sphere(c["center"], c["radius"]), c["dim"], c["n_cells"], c["degree"], c["n_levels"])
    return pb, H, request.param


@pytest.mark.parametrize("prec,tol", [(cm.CF_FP64, 1e-12), (cm.CF_MIXED, 2e-5)])
def test_apply(pair, prec, tol):
    pb, H, _ = pair
    for l in range(pb.n_levels):
        x = random_vector(pb.n_dofs(l), 100 + l)
        y = torch.zeros(pb.n_dofs(l), dtype=torch.float64, device=DEV)
        pb.level_apply(l, _t(x), y, precision=prec)
        assert rel(_n(y), H.levels[l].A @ x) < tol


@pytest.mark.parametrize("prec,tol", [(cm.CF_FP64, 1e-11), (cm.CF_MIXED, 2e-4)])
def test_colour_steps(pair, prec, tol):
    pb, H, _ = pair
    for l in range(1, pb.n_levels):
        n = pb.n_dofs(l)
        for cut in (False, True):
            tstep = 2e-2 if (prec == cm.CF_MIXED and not cut) else tol
            for col in range(1 << pb.dim):
                x0 = random_vector(n, 7 + col)
                b = random_vector(n, 300 + col)
                xg = _t(x0)
                pb.colour_step(l, cut, col, xg, _t(b), precision=prec)
                xo = H.colour_step(l, x0, b, cut, col)
                # the FP32 path also rounds the untouched entries of x to FP32
                floor = np.abs(x0).max() * (1e-6 if prec == cm.CF_MIXED else 1e-15)
                err = np.abs(_n(xg) - xo).max()
                assert err <= tstep * np.abs(xo - x0).max() + floor, (l, cut, col)


def test_smoothing_step(pair):
    pb, H, _ = pair
    for l in range(1, pb.n_levels):
        n = pb.n_dofs(l)
        b = random_vector(n, 11)
        for post in (False, True):
            xg = torch.zeros(n, dtype=torch.float64, device=DEV)
            pb.smooth(l, xg, _t(b), post=post)
            xo = H.smooth(l, np.zeros(n), b, post=post)
            assert rel(_n(xg), xo) < 1e-11


def test_transfer(pair):
    pb, H, _ = pair
    for l in range(1, pb.n_levels):
        r = random_vector(pb.n_dofs(l), 21)
        bc = torch.zeros(pb.n_dofs(l - 1), dtype=torch.float64, device=DEV)
        pb.restrict(l, _t(r), bc)
        assert rel(_n(bc), H.P[l].T @ r) < 1e-13
        xc = random_vector(pb.n_dofs(l - 1), 22)
        xf0 = random_vector(pb.n_dofs(l), 23)
        xf = _t(xf0)
        pb.prolongate(l, _t(xc), xf)
        assert rel(_n(xf), xf0 + H.P[l] @ xc) < 1e-13


def test_coarse_solve(pair):
    pb, H, _ = pair
    import scipy.linalg as sla
    b0 = random_vector(pb.n_dofs(0), 31)
    x0 = torch.zeros(pb.n_dofs(0), dtype=torch.float64, device=DEV)
    pb.coarse_solve(_t(b0), x0)
    assert rel(_n(x0), sla.cho_solve(H.coarse_chol, b0)) < 1e-10


def test_vcycle(pair):
    pb, H, _ = pair
    r = random_vector(pb.n_dofs(), 41)
    z = torch.zeros(pb.n_dofs(), dtype=torch.float64, device=DEV)
    pb.vcycle(_t(r), z)
    assert rel(_n(z), H.vcycle(r)) < 1e-10


def test_rhs_and_solve_fp64(pair):
    pb, H, _ = pair
    n = pb.n_dofs()
    b = torch.zeros(n, dtype=torch.float64, device=DEV)
    pb.rhs(b)
    bo = H.rhs()
    assert rel(_n(b), bo) < 1e-13
    x = torch.zeros(n, dtype=torch.float64, device=DEV)
    info = pb.solve(b, x, rtol=1e-8)
    xo, it, hist = H.pcg(bo, rtol=1e-8)
    assert abs(info["iterations"] - it) <= 1
    assert np.linalg.norm(_n(x) - xo) <= 1e-10 * np.linalg.norm(xo)
    assert info["true_rel_residual"] <= 1.01e-8


def test_solve_mixed_reaches_fp64_accuracy(pair):
    pb, H, _ = pair
    n = pb.n_dofs()
    b = torch.zeros(n, dtype=torch.float64, device=DEV)
    pb.rhs(b)
    bo = H.rhs()
    pb.set_precision(cm.CF_MIXED)
    try:
        x = torch.zeros(n, dtype=torch.float64, device=DEV)
        info = pb.solve(b, x, rtol=1e-8)
    finally:
        pb.set_precision(cm.CF_FP64)
    xo, it, _ = H.pcg(bo, rtol=1e-8)
    assert info["true_rel_residual"] <= 1.01e-8
    # both are 1e-8 solutions of the same system: they agree to ~cond * 1e-8
    assert np.linalg.norm(_n(x) - xo) <= 1e-6 * np.linalg.norm(xo)
    assert info["iterations"] <= it + 2


def test_zero_rhs(pair):
    pb, H, _ = pair
    n = pb.n_dofs()
    b = torch.zeros(n, dtype=torch.float64, device=DEV)
    x = torch.ones(n, dtype=torch.float64, device=DEV)
    info = pb.solve(b, x)
    assert info["iterations"] == 0
    assert _n(x).max() == 0.0
