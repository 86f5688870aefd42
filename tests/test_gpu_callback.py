"""A domain given only through level-set callbacks (CF_LS_CALLBACK): setup on
the host from the sampled bounds, then the V-cycle and the CG solve through
the C ABI against the oracle's restatement of the same reading (one V-cycle
element by element at 1e-10 relative; CG iterations within one, iterates
1e-10 relative when the counts agree)."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2508_11608_gb300 as cm  # noqa: E402
from paper_2508_11608_gb300.workloads import random_vector  # noqa: E402
from oracle import Hierarchy  # noqa: E402
from oracle.levelset import make_levelset  # noqa: E402

from callback_shapes import superellipse  # noqa: E402

DEV = "cuda:0"
CASES = {
    "superellipse2d_q2_n32": (2, 32, 3, 2, superellipse([0.03, -0.02], [0.7, 0.55])),
    "superellipse2d_q3_n16": (2, 16, 2, 3, superellipse([0.03, -0.02], [0.7, 0.55])),
    "superellipse3d_q2_n8": (3, 8, 2, 2, superellipse([0.03, -0.02, 0.01], [0.7, 0.55, 0.6])),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    d, N, L, p, spec = CASES[request.param]
    pb = cm.Problem(d, N, L, p, levelset=spec)
    H = Hierarchy(make_levelset(spec), d, N, p, L)
    return pb, H


def test_callback_vcycle_matches_the_oracle(case):
    pb, H = case
    r = random_vector(pb.n_dofs(), 41)
    z = torch.zeros(pb.n_dofs(), dtype=torch.float64, device=DEV)
    pb.vcycle(torch.tensor(r, device=DEV), z)
    torch.cuda.synchronize()
    zo = H.vcycle(r)
    assert np.abs(z.cpu().numpy() - zo).max() <= 1e-10 * np.abs(zo).max()


def test_callback_solve_matches_the_oracle(case):
    pb, H = case
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
