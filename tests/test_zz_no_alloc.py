"""cf_coarse_solve_noalloc: the coarse solve for callers that cannot let a
library call allocate device memory (graph capture, caller-owned memory
arenas, allocation-free hot loops).  Its result must equal the allocating
cf_coarse_solve's on two calls in a row, it must refuse coarse levels larger
than its fixed staging array, leave the device's free memory unchanged and
run inside a CUDA graph capture.  Kept in its own file, collected last."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2508_11608_gb300 as cm  # noqa: E402
from paper_2508_11608_gb300.workloads import problem_kwargs, random_vector  # noqa: E402

DEV = "cuda:0"


@pytest.mark.parametrize("name", ["disk2d_q2_n32", "ball3d_q2_n16"])
def test_noalloc_coarse_solve_matches_allocating_one(name):
    pb = cm.Problem(**problem_kwargs(name))
    n0 = pb.n_dofs(0)
    for call in range(2):
        b0 = torch.tensor(random_vector(n0, 500 + call), dtype=torch.float64, device=DEV)
        ref = torch.zeros(n0, dtype=torch.float64, device=DEV)
        got = torch.full((n0,), np.nan, dtype=torch.float64, device=DEV)
        pb.coarse_solve(b0, ref, precision=cm.CF_FP64)
        pb.coarse_solve_noalloc(b0, got)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.abs(g - r).max() <= 1e-12 * np.abs(r).max(), call


def test_noalloc_rejects_large_coarse_level():
    # 2D, one level of 96^2 cells: the coarsest lattice has 193^2 = 37249 > 32768
    # nodes (a small disk keeps the dense coarse inverse tiny)
    pb = cm.Problem(2, 96, 1, 2, center=[0.01, 0.02], radius=0.05)
    n0 = pb.n_dofs(0)
    b0 = torch.zeros(n0, dtype=torch.float64, device=DEV)
    x0 = torch.zeros(n0, dtype=torch.float64, device=DEV)
    with pytest.raises(cm.CutmgError) as e:
        pb.coarse_solve_noalloc(b0, x0)
    assert e.value.status == cm._lib.CF_EINVAL
    assert "at most" in str(e.value)


def test_noalloc_call_leaves_free_device_memory_unchanged():
    # after one call (kernels loaded, the array's address looked up), further
    # calls take no device memory: the device's free bytes stay the same
    pb = cm.Problem(**problem_kwargs("ball3d_q2_n16"))
    n0 = pb.n_dofs(0)
    b0 = torch.tensor(random_vector(n0, 900), dtype=torch.float64, device=DEV)
    x0 = torch.zeros(n0, dtype=torch.float64, device=DEV)
    pb.coarse_solve_noalloc(b0, x0)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        pb.coarse_solve_noalloc(b0, x0)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_coarse_solve_runs_inside_cuda_graph_capture():
    # captured in the global capture mode, where any device allocation during
    # the capture (by this thread or another) fails it; the graph then
    # replays the solve on new contents of the same input buffer
    pb = cm.Problem(**problem_kwargs("ball3d_q2_n16"))
    n0 = pb.n_dofs(0)
    b0 = torch.tensor(random_vector(n0, 910), dtype=torch.float64, device=DEV)
    x0 = torch.zeros(n0, dtype=torch.float64, device=DEV)
    pb.coarse_solve_noalloc(b0, x0)  # first call outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="global"):
        pb.coarse_solve_noalloc(b0, x0)
    for seed in (911, 912):
        b0.copy_(torch.tensor(random_vector(n0, seed), dtype=torch.float64, device=DEV))
        x0.fill_(np.nan)
        g.replay()
        ref = torch.zeros(n0, dtype=torch.float64, device=DEV)
        pb.coarse_solve(b0, ref, precision=cm.CF_FP64)
        torch.cuda.synchronize()
        r, x = ref.cpu().numpy(), x0.cpu().numpy()
        assert np.abs(x - r).max() <= 1e-12 * np.abs(r).max(), seed
