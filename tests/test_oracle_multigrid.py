"""Pins of the oracle's transfer operators, patches, smoother, V-cycle and
PCG (Sec. 2.2, Sec. 2.3, Sec. 3)."""

import json
import math
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spl

from oracle.fem import Level
from oracle.levelset import Sphere
from oracle.multigrid import Hierarchy

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def h2d():
    return Hierarchy(Sphere([0.031, 0.017], 0.7), 2, 16, 2, 2)


@pytest.fixture(scope="module")
def h3d():
    return Hierarchy(Sphere([0.05, 0.03, 0.02], 0.7), 3, 8, 2, 2)


@pytest.mark.parametrize("which", ["h2d", "h3d"])
def test_prolongation_reproduces_coarse_qp(which, request):
    H = request.getfixturevalue(which)
    f, c = H.levels[1].lev, H.levels[0].lev
    Xf = f.node_coords(f.dof_nodes)
    Xc = c.node_coords(c.dof_nodes)
    d = f.d
    for deg in [(0,) * d, (1,) + (0,) * (d - 1), (2, 1, 2)[:d], (2,) * d]:
        u = lambda X: np.prod([X[:, k] ** deg[k] for k in range(d)], axis=0)
        assert np.abs(H.P[1] @ u(Xc) - u(Xf)).max() < 1e-13
    # one degree more is not reproduced (the check has teeth)
    u = lambda X: X[:, 0] ** 3
    assert np.abs(H.P[1] @ u(Xc) - u(Xf)).max() > 1e-4


@pytest.mark.parametrize("which", ["h2d", "h3d"])
def test_patches_cover_and_colours_are_disjoint(which, request):
    H = request.getfixturevalue(which)
    P = H.levels[1].patches
    n = H.levels[1].lev.ndof
    seen = np.zeros(n, dtype=int)
    for I in P.I:
        seen[I] += 1
    assert (seen > 0).all()
    for col in range(1 << P.d):
        mark = np.zeros(n, dtype=int)
        for j in np.nonzero(P.colour == col)[0]:
            mark[P.I[j]] += 1
        assert mark.max() <= 1
    p = H.p
    assert all(len(P.I[j]) == (2 * p - 1) ** P.d for j in np.nonzero(~P.cut)[0])


def test_cartesian_patch_matrix_is_kronecker_sum():
    """A_j of an interior patch equals K x M (x M) + ... built from the
    closed-form 1D Q2 matrices of a two-cell patch (Sec. 3, fast
    diagonalisation premise)."""
    H = Hierarchy(Sphere([0.05, 0.03, 0.02], 0.7), 3, 8, 2, 2)
    g = json.load(open(os.path.join(GOLD, "q2_reference_1d.json")))
    M1 = np.array(g["mass_times_30"]) / 30.0
    K1 = np.array(g["stiffness_times_3"]) / 3.0
    h = H.levels[1].lev.h
    Mp = np.zeros((5, 5))
    Kp = np.zeros((5, 5))
    for s in (0, 2):
        Mp[s:s + 3, s:s + 3] += M1 * h
        Kp[s:s + 3, s:s + 3] += K1 / h
    Mi, Ki = Mp[1:4, 1:4], Kp[1:4, 1:4]
    ref = (np.kron(np.kron(Mi, Mi), Ki) + np.kron(np.kron(Mi, Ki), Mi)
           + np.kron(np.kron(Ki, Mi), Mi))
    P = H.levels[1].patches
    js = np.nonzero(~P.cut)[0]
    assert js.size > 0
    for j in js[:5]:
        # the Kronecker sum is the same for any ordering of the directions
        assert np.allclose(P.Aj[j], ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("which", ["h2d", "h3d"])
def test_vcycle_symmetric_positive_definite_contracting(which, request):
    H = request.getfixturevalue(which)
    A = H.fine.A.toarray()
    n = A.shape[0]
    B = np.stack([H.vcycle(np.eye(n)[:, i]) for i in range(n)], axis=1)
    assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0
    rho = np.abs(np.linalg.eigvals(np.eye(n) - B @ A)).max()
    assert rho < 0.5


def test_pcg_matches_direct_solve(h2d):
    b = h2d.rhs()
    x, it, hist = h2d.pcg(b, rtol=1e-12)
    xd = spl.spsolve(h2d.fine.A.tocsc(), b)
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)
    assert hist[-1] <= 1e-12 * np.linalg.norm(b)


def test_literal_vertex_set_leaves_boundary_dofs_unsmoothed():
    """Documents why the covering reading is used: with patches only at
    vertices inside Omega and interior DoFs only, some DoFs of Omega_l lie in
    no patch."""
    lev = Level(Sphere([0.031, 0.017], 0.7), 2, 16, 2)
    p, N, d = 2, 16, 2
    covered = np.zeros(lev.ndof, dtype=bool)
    for i in range(1, N):
        for j in range(1, N):
            X = np.array([[-1 + lev.h * i, -1 + lev.h * j]])
            if lev.ls.phi(X)[0] < 0:
                for a in range(1, 2 * p):
                    for bb in range(1, 2 * p):
                        node = (p * (i - 1) + a) + lev.n * (p * (j - 1) + bb)
                        covered[lev.node_to_dof[node]] = True
    assert (~covered).sum() > 0


def test_iteration_counts_bounded_under_refinement():
    """Behavioural pin in the spirit of Table 1: iteration counts stay small
    and do not grow with refinement."""
    ls = Sphere([0.031, 0.017], 0.7)
    its = []
    for N, L in ((16, 2), (32, 3), (64, 4)):
        H = Hierarchy(ls, 2, N, 2, L)
        _, it, _ = H.pcg(H.rhs())
        its.append(it)
    assert max(its) <= 8
    assert its[-1] <= its[0] + 1


def _tiny_b_and_B(H):
    A = H.fine.A.toarray()
    n = A.shape[0]
    B = np.stack([H.vcycle(np.eye(n)[:, i]) for i in range(n)], axis=1)
    b = H.rhs()
    return A, B, b


def test_vcycle_solver_residuals_are_powers_of_the_iteration_matrix(h2d):
    """x_{k+1} = x_k + B (b - A x_k) from 0: r_k = (I - A B)^k b exactly."""
    H = h2d
    A, B, b = _tiny_b_and_B(H)
    _, it, hist = H.vcycle_solve(b, rtol=1e-30, maxit=5)
    r = b.copy()
    for k in range(1, 6):
        r = r - A @ (B @ r)
        assert hist[k] == pytest.approx(np.linalg.norm(r), rel=1e-9)


def test_gmres_is_the_minimal_residual_over_the_preconditioned_krylov_space(h2d):
    """After k steps from x_0 = 0, GMRES with right preconditioner B returns
    the x in B K_k(A B, b) of least ||b - A x||_2 (checked by least squares
    over an explicit orthonormal Krylov basis), for k = 1..4."""
    H = h2d
    A, B, b = _tiny_b_and_B(H)
    AB = A @ B
    K = [b / np.linalg.norm(b)]
    for k in range(1, 5):
        Q, _ = np.linalg.qr(np.stack(K, axis=1))
        Y = B @ Q                        # x = Y c
        c, *_ = np.linalg.lstsq(A @ Y, b, rcond=None)
        best = np.linalg.norm(b - A @ (Y @ c))
        x, it, hist = H.gmres(b, rtol=1e-30, restart=30, maxit=k)
        assert it == k
        assert np.linalg.norm(b - A @ x) == pytest.approx(best, rel=1e-8)
        assert hist[-1] == pytest.approx(best, rel=1e-8)
        K.append(AB @ K[-1])
        K[-1] = K[-1] / np.linalg.norm(K[-1])


def test_solvers_converge_to_the_direct_solution(h2d):
    H = h2d
    import scipy.sparse.linalg as spla
    b = H.rhs()
    xd = spla.spsolve(H.fine.A.tocsc(), b)
    for solve in (H.vcycle_solve, H.gmres):
        x, it, hist = solve(b, rtol=1e-12)
        assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)
        assert all(hist[i + 1] <= hist[i] * (1 + 1e-12) for i in range(len(hist) - 1))
    x3, _, _ = H.gmres(b, rtol=1e-12, restart=3)
    assert np.linalg.norm(x3 - xd) <= 1e-8 * np.linalg.norm(xd)


@pytest.fixture(scope="module")
def h2d_cheb():
    return Hierarchy(Sphere([0.031, 0.017], 0.7), 2, 16, 2, 2, smoother="chebyshev")


def test_chebyshev_smoother_is_the_scaled_chebyshev_polynomial(h2d_cheb):
    """With b = A x*, one smoothing maps the error e = x - x* to p(D^{-1} A) e,
    p(t) = T_k((theta - t) / delta) / T_k(theta / delta) on [lmin, lmax]: the
    recurrence against the closed form through the eigenvectors of the
    symmetric D^{-1/2} A D^{-1/2}."""
    H = h2d_cheb
    l = 1
    L = H.levels[l]
    A = L.A.toarray()
    dh = np.sqrt(L.dinv)
    lam, Q = np.linalg.eigh(dh[:, None] * A * dh[None, :])
    lmax = H.CHEB_SAFETY * L.lam_max
    lmin = lmax / H.CHEB_RANGE
    theta, delta = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
    k = H.cheb_degree
    Tk = np.polynomial.chebyshev.chebval
    coef = np.zeros(k + 1)
    coef[k] = 1.0
    p = Tk((theta - lam) / delta, coef) / Tk(theta / delta, coef)
    rng = np.random.default_rng(5)
    xs = rng.standard_normal(A.shape[0])
    x0 = rng.standard_normal(A.shape[0])
    x1 = H.chebyshev(l, x0, A @ xs)
    # e1 = D^{-1/2} Q diag(p) Q^T D^{1/2} e0
    e1 = (Q @ (p * (Q.T @ ((x0 - xs) / dh)))) * dh
    assert np.abs((x1 - xs) - e1).max() <= 1e-10 * np.abs(x0 - xs).max()
    # the estimate sits at the top of the spectrum of D^{-1} A
    assert L.lam_max == pytest.approx(lam.max(), rel=0.05)


def test_chebyshev_vcycle_is_symmetric_positive_definite(h2d_cheb):
    H = h2d_cheb
    A = H.fine.A.toarray()
    n = A.shape[0]
    B = np.stack([H.vcycle(np.eye(n)[:, i]) for i in range(n)], axis=1)
    assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0
    assert np.abs(np.linalg.eigvals(np.eye(n) - B @ A)).max() < 1.0
