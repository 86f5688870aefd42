"""The paper's two other ways to use the V-cycle (Sec. 2.2): as the solver
itself (x += B (b - A x)) and as the right preconditioner of GMRES, through
cf_solve_vcycle / cf_solve_gmres, against the oracle's restatements.

Both follow fixed recurrences, so after the same number of iterations the
GPU and oracle iterates agree to rounding: compared element by element at
1e-10 relative (as the CG solve).  Converged runs: iterations within one and
the true residual below the tolerance."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2508_11608_gb300 as cm  # noqa: E402
from paper_2508_11608_gb300.workloads import CONFIGS, problem_kwargs  # noqa: E402
from oracle import Hierarchy, Sphere  # noqa: E402
from oracle.fem import assemble_rhs  # noqa: E402

NAMES = ["disk2d_q2_n32", "ball3d_q2_n16", "disk2d_q3_n32", "ball3d_q1_n16"]
DEV = "cuda:0"


@pytest.fixture(scope="module", params=NAMES)
def case(request):
    c = CONFIGS[request.param]
    pb = cm.Problem(**problem_kwargs(request.param))
    H = Hierarchy(Sphere(c["center"], c["radius"]), c["dim"], c["n_cells"], c["degree"], c["n_levels"])
    b = torch.zeros(pb.n_dofs(), dtype=torch.float64, device=DEV)
    pb.rhs(b)
    return pb, H, b, H.rhs()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_vcycle_iteration_matches_the_oracle_step_by_step(case):
    pb, H, b, bo = case
    pb.set_precision(cm.CF_FP64)
    x = torch.zeros_like(b)
    info = pb.solve_vcycle(b, x, rtol=1e-30, maxit=4, allow_noconv=True)
    torch.cuda.synchronize()
    xo, it, _ = H.vcycle_solve(bo, rtol=1e-30, maxit=4)
    assert info["iterations"] == it == 4
    assert _rel(x.cpu().numpy(), xo) <= 1e-10


@pytest.mark.parametrize("restart,steps", [(30, 5), (3, 7)])
def test_gmres_matches_the_oracle_step_by_step(case, restart, steps):
    pb, H, b, bo = case
    pb.set_precision(cm.CF_FP64)
    x = torch.zeros_like(b)
    info = pb.solve_gmres(b, x, rtol=1e-30, restart=restart, maxit=steps, allow_noconv=True)
    torch.cuda.synchronize()
    xo, it, _ = H.gmres(bo, rtol=1e-30, restart=restart, maxit=steps)
    assert info["iterations"] == it == steps
    assert _rel(x.cpu().numpy(), xo) <= 1e-10


def test_converged_solvers_match_the_oracle(case):
    pb, H, b, bo = case
    pb.set_precision(cm.CF_FP64)
    for solver, ref in ((pb.solve_vcycle, H.vcycle_solve), (pb.solve_gmres, H.gmres)):
        x = torch.zeros_like(b)
        info = solver(b, x, rtol=1e-9)
        torch.cuda.synchronize()
        xo, it, _ = ref(bo, rtol=1e-9)
        assert abs(info["iterations"] - it) <= 1, (solver.__name__, info, it)
        # the V-cycle iteration stops on the true residual, GMRES on its
        # recursive estimate, which differs from it by rounding
        assert info["true_rel_residual"] <= (1e-9 if solver == pb.solve_vcycle else 1.1e-9)
        if info["iterations"] == it:  # the same recurrence to the same step
            assert _rel(x.cpu().numpy(), xo) <= 1e-10


def test_mixed_gmres_reaches_fp64_accuracy(case):
    pb, _, b, _ = case
    pb.set_precision(cm.CF_MIXED)
    x = torch.zeros_like(b)
    info = pb.solve_gmres(b, x, rtol=1e-9)
    torch.cuda.synchronize()
    assert info["true_rel_residual"] <= 1.1e-9
    pb.set_precision(cm.CF_FP64)


def test_user_data_right_hand_side_solve_matches_the_oracle(case):
    """cf_rhs_user on the device equals the host assembly bit for bit, and
    the CG solve for u in Q_p (f = -Laplace u, g = u) matches the oracle's
    solve of the same data (iterations within one, iterates 1e-10 relative
    when the counts agree).  The discrete solution is u only up to the cut
    quadrature's error, so u's nodal values bound it loosely."""
    pb, H, _, _ = case
    p, d = pb.degree, pb.dim
    cz = 0.25 if d == 3 else 0.0

    def u(x):
        return 1.0 + x[0] - 0.5 * x[1] ** p + cz * x[d - 1] ** p

    def f(x):
        if p == 1:
            return 0.0
        return 0.5 * p * (p - 1) * x[1] ** (p - 2) - cz * p * (p - 1) * x[d - 1] ** (p - 2)

    pb.set_precision(cm.CF_FP64)
    b = torch.zeros(pb.n_dofs(), dtype=torch.float64, device=DEV)
    pb.rhs_user(f, u, b)
    torch.cuda.synchronize()
    bh = pb.rhs_user(f, u)
    assert np.array_equal(b.cpu().numpy(), bh)
    x = torch.zeros_like(b)
    info = pb.solve(b, x, rtol=1e-10)
    torch.cuda.synchronize()
    bo = assemble_rhs(H.fine.lev, H.gamma_D, H.q, u=lambda X: np.array([u(r) for r in X]),
                      f=lambda X: np.array([f(r) for r in X]))
    assert np.abs(bh - bo).max() <= 1e-13 * np.abs(bo).max()
    xo, it, _ = H.pcg(bo, rtol=1e-10)
    assert abs(info["iterations"] - it) <= 1, (info, it)
    if info["iterations"] == it:
        assert _rel(x.cpu().numpy(), xo) <= 1e-10
    ue = np.array([u(r) for r in pb.dof_coords()])
    assert np.abs(x.cpu().numpy() - ue).max() <= 1e-3 * np.abs(ue).max()
