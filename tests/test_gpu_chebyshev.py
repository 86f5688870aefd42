"""The Chebyshev smoother baseline (the paper's comparison in Sec. 4) through
the C ABI against the oracle: one V-cycle element by element (FP64, 1e-10
relative, as the vertex-patch V-cycle), the CG solve (iterations within one,
iterates 1e-10 when the counts agree), the mixed form, and the batched form
refusing it."""

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


@pytest.fixture(scope="module", params=NAMES)
def case(request):
    c = CONFIGS[request.param]
    pb = cm.Problem(**problem_kwargs(request.param), smoother=cm.CF_SMOOTHER_CHEBYSHEV)
    H = Hierarchy(Sphere(c["center"], c["radius"]), c["dim"], c["n_cells"], c["degree"], c["n_levels"],
                  smoother="chebyshev")
    return pb, H


def test_chebyshev_vcycle_matches_the_oracle(case):
    pb, H = case
    pb.set_precision(cm.CF_FP64)
    r = random_vector(pb.n_dofs(), 31)
    z = torch.zeros(pb.n_dofs(), dtype=torch.float64, device=DEV)
    pb.vcycle(torch.tensor(r, device=DEV), z)
    torch.cuda.synchronize()
    zo = H.vcycle(r)
    assert np.abs(z.cpu().numpy() - zo).max() <= 1e-10 * np.abs(zo).max()


def test_chebyshev_cg_matches_the_oracle(case):
    pb, H = case
    pb.set_precision(cm.CF_FP64)
    b = torch.zeros(pb.n_dofs(), dtype=torch.float64, device=DEV)
    pb.rhs(b)
    x = torch.zeros_like(b)
    info = pb.solve(b, x, rtol=1e-8)
    torch.cuda.synchronize()
    xo, it, _ = H.pcg(H.rhs(), rtol=1e-8)
    assert abs(info["iterations"] - it) <= 1, (info, it)
    assert info["true_rel_residual"] <= 1e-8
    if info["iterations"] == it:
        assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-10 * np.linalg.norm(xo)


def test_chebyshev_mixed_reaches_fp64_accuracy(case):
    pb, _ = case
    pb.set_precision(cm.CF_MIXED)
    b = torch.zeros(pb.n_dofs(), dtype=torch.float64, device=DEV)
    pb.rhs(b)
    x = torch.zeros_like(b)
    info = pb.solve(b, x, rtol=1e-8)
    torch.cuda.synchronize()
    assert info["true_rel_residual"] <= 1e-8
    pb.set_precision(cm.CF_FP64)


def test_batched_form_refuses_the_chebyshev_smoother(case):
    pb, _ = case
    with pytest.raises(cm.CutmgError):
        cm.Batch([pb])
