"""Every launch variant of the colour-step kernels against the oracle, element
by element, and against each other, through the C ABI.

The automatic launch choice depends on how many patches a colour holds, so
the parity cases (a few hundred patches per colour) would otherwise never run
the variants the large benchmark sizes use.  cf_set_kernel_variant forces
each one on the same small problems:
  interior step, FP32 (mixed form): dense map with 1 or 2 patches per thread,
    the split form with several threads per patch, and the tensor-core form;
  interior step, FP64: two patches per warp (a half-warp each), one block per patch;
  cut-patch step (3D Q2): each patch's record (inverse and cut-cell rows)
    prefetched into L2 by a bulk prefetch when its loads are issued, one
    patch ahead, or not; and, where the automatic choice runs colours of few
    patches one patch per block with its warps working together, eight
    warps per block with one patch each, or one warp per block;
  operator rows of nodes with only uncut cells: element matrices or sum
    factorisation.
Tolerances as in test_gpu_parity (FP64 1e-11 of the update, FP32 2e-4); the
variants that share an arithmetic must agree bit for bit.  The tensor-core
form rounds its operands to TF32 (10-bit mantissa, unit roundoff 4.9e-4),
so it is held to 2e-2 of the update, and its solves to the FP64 residual."""

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

NAMES = ["disk2d_q2_n32", "ball3d_q2_n16", "disk2d_q3_n32", "ball3d_q1_n16"]
DEV = "cuda:0"


def _t(a):
    return torch.tensor(a, dtype=torch.float64, device=DEV)


def _n(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.fixture(scope="module", params=NAMES)
def pair(request):
    c = CONFIGS[request.param]
    pb = cm.Problem(**problem_kwargs(request.param))
    H = Hierarchy(Sphere(c["center"], c["radius"]), c["dim"], c["n_cells"], c["degree"], c["n_levels"])
    yield pb, H, request.param
    pb.set_kernel_variant(_lib.CF_VAR_INTERIOR, 0)
    pb.set_kernel_variant(_lib.CF_VAR_CUT, 0)
    pb.set_kernel_variant(_lib.CF_VAR_OPERATOR, 0)


def _steps(pb, H, cut, prec, tol):
    """Every colour step of one kind on every smoothing level; returns the
    GPU results and checks each against the oracle."""
    outs = []
    for l in range(1, pb.n_levels):
        n = pb.n_dofs(l)
        for col in range(1 << pb.dim):
            x0 = random_vector(n, 7 + col)
            b = random_vector(n, 300 + col)
            xg = _t(x0)
            pb.colour_step(l, cut, col, xg, _t(b), precision=prec)
            xo = H.colour_step(l, x0, b, cut, col)
            got = _n(xg)
            floor = np.abs(x0).max() * (1e-6 if prec == cm.CF_MIXED else 1e-15)
            assert np.abs(got - xo).max() <= tol * np.abs(xo - x0).max() + floor, (l, cut, col)
            outs.append(got)
    return outs


INTERIOR = [(cm.CF_FP64, [1, 2], 1e-11), (cm.CF_MIXED, [1, 2, 3], 2e-4)]


@pytest.mark.parametrize("prec,variants,tol", INTERIOR)
def test_interior_variants_match_oracle_and_each_other(pair, prec, variants, tol):
    pb, H, _ = pair
    ref = None
    for v in variants:
        pb.set_kernel_variant(_lib.CF_VAR_INTERIOR, v)
        outs = _steps(pb, H, False, prec, tol)
        if ref is None:
            ref = outs
        else:
            for a, b in zip(ref, outs):
                assert np.array_equal(a, b), v
    pb.set_kernel_variant(_lib.CF_VAR_INTERIOR, 0)


def test_interior_tensor_core_variant_matches_oracle(pair):
    pb, H, _ = pair
    pb.set_kernel_variant(_lib.CF_VAR_INTERIOR, 4)
    try:
        _steps(pb, H, False, cm.CF_MIXED, 2e-2)
    finally:
        pb.set_kernel_variant(_lib.CF_VAR_INTERIOR, 0)


@pytest.mark.parametrize("prec,tol", [(cm.CF_FP64, 1e-11), (cm.CF_MIXED, 2e-4)])
def test_cut_variants_match_oracle_and_each_other(pair, prec, tol):
    pb, H, name = pair
    if name != "ball3d_q2_n16":
        pytest.skip("one cut kernel form for (d, p) with at most 64 closure nodes")
    ref = None
    for v in (1, 2, 3, 4, 5, 6):
        pb.set_kernel_variant(_lib.CF_VAR_CUT, v)
        outs = _steps(pb, H, True, prec, tol)
        if ref is None:
            ref = outs
        else:
            for a, b in zip(ref, outs):
                assert np.array_equal(a, b), v
    pb.set_kernel_variant(_lib.CF_VAR_CUT, 0)


def test_solve_with_every_variant_takes_the_oracle_iterations(pair):
    pb, H, _ = pair
    n = pb.n_dofs()
    b = torch.zeros(n, dtype=torch.float64, device=DEV)
    pb.rhs(b)
    xo, it, _ = H.pcg(H.rhs(), rtol=1e-8)
    for prec, vs in ((cm.CF_FP64, (1, 2)), (cm.CF_MIXED, (1, 2, 3, 4))):
        pb.set_precision(prec)
        for v in vs:
            pb.set_kernel_variant(_lib.CF_VAR_INTERIOR, v)
            x = torch.zeros_like(b)
            info = pb.solve(b, x, rtol=1e-8)
            assert info["true_rel_residual"] <= 1.01e-8, (prec, v)
            if prec == cm.CF_FP64:
                assert abs(info["iterations"] - it) <= 1
                assert np.linalg.norm(_n(x) - xo) <= 1e-10 * np.linalg.norm(xo)
            else:
                assert info["iterations"] <= it + 2, (v, info["iterations"], it)
    pb.set_precision(cm.CF_FP64)
    pb.set_kernel_variant(_lib.CF_VAR_INTERIOR, 0)


def test_bad_variants_are_rejected(pair):
    pb, _, _ = pair
    for fam, v in ((0, 1), (4, 1), (_lib.CF_VAR_INTERIOR, 5), (_lib.CF_VAR_CUT, 7), (_lib.CF_VAR_CUT, -1),
                   (_lib.CF_VAR_OPERATOR, 3)):
        with pytest.raises(cm.CutmgError) as e:
            pb.set_kernel_variant(fam, v)
        assert e.value.status == _lib.CF_EINVAL


def test_wait_limit_runs_out_and_the_handle_recovers():
    """The tensor-core interior kernel's bounded wait on its product (mixed
    form): with a limit of zero polls every wait gives up at once (no hang:
    each block then waits for its own product within the default bound), the
    solve reports CF_ETIMEOUT, and with the default limit restored the same
    handle solves to the usual result."""
    pb = cm.Problem(**problem_kwargs("ball3d_q2_n16"))
    pb.set_precision(cm.CF_MIXED)
    n = pb.n_dofs()
    b = torch.zeros(n, dtype=torch.float64, device=DEV)
    pb.rhs(b)
    x = torch.zeros_like(b)
    ref = pb.solve(b, x, rtol=1e-8)
    xr = _n(x).copy()
    pb.set_wait_limit(0)
    with pytest.raises(cm.CutmgError) as e:
        pb.solve(b, torch.zeros_like(b), rtol=1e-8, maxit=3)
    assert e.value.status == _lib.CF_ETIMEOUT
    pb.set_wait_limit(1 << 22)
    x2 = torch.zeros_like(b)
    info = pb.solve(b, x2, rtol=1e-8)
    assert info["iterations"] == ref["iterations"]
    assert np.array_equal(_n(x2), xr)
    with pytest.raises(cm.CutmgError):
        pb.set_wait_limit(-1)


@pytest.mark.parametrize("prec,tol", [(cm.CF_FP64, 1e-12), (cm.CF_MIXED, 2e-5)])
def test_operator_variants_match_oracle(pair, prec, tol):
    """The rows of nodes whose cells are all uncut: element-matrix form
    (variant 1) and sum factorisation (variant 2), on every level, against
    the oracle's assembled operator."""
    pb, H, _ = pair
    for v in (1, 2):
        pb.set_kernel_variant(_lib.CF_VAR_OPERATOR, v)
        for l in range(pb.n_levels):
            x = random_vector(pb.n_dofs(l), 100 + l)
            y = torch.zeros(pb.n_dofs(l), dtype=torch.float64, device=DEV)
            pb.level_apply(l, _t(x), y, precision=prec)
            yo = H.levels[l].A @ x
            assert np.abs(_n(y) - yo).max() <= tol * np.abs(yo).max(), (v, l)
    pb.set_kernel_variant(_lib.CF_VAR_OPERATOR, 0)


def test_device_patch_inverses_match_the_host_inverses():
    """3D Q2: the cut-patch inverses of a device handle are formed on the GPU
    in FP64 (Cholesky, triangular inverse, W^T W); they agree with the host
    setup's inverses of the same patches (a host-only handle) and invert the
    oracle's patch matrix A[I_j, I_j]."""
    name = "ball3d_q2_n16"
    c = CONFIGS[name]
    dev = cm.Problem(**problem_kwargs(name))
    host = cm.Problem(**problem_kwargs(name), host_only=True)
    H = Hierarchy(Sphere(c["center"], c["radius"]), c["dim"], c["n_cells"], c["degree"], c["n_levels"])
    for l in range(1, dev.n_levels):
        pd = dev.host_patches(l)[1]
        ph = host.host_patches(l)[1]
        lev = H.levels[l]
        assert len(pd) == len(ph) > 0
        worst = 0.0
        for (va, na, ia), (vb, nb, ib) in zip(pd, ph):
            assert va == vb and np.array_equal(na, nb)
            worst = max(worst, np.abs(ia - ib).max() / np.abs(ib).max())
            idx = lev.lev.node_to_dof[na]
            Aj = lev.A[idx][:, idx].toarray()
            assert np.abs(ia @ Aj - np.eye(len(idx))).max() < 1e-9
        assert worst < 1e-10, (l, worst)
