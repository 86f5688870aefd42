"""The library's host setup (classification, DoF numbering, cut-cell and
uncut element matrices, right-hand side, patch sets, cut-patch inverses)
against the oracle, on CPU through cf_setup_host.  No device is touched."""

import numpy as np
import pytest

from oracle import Hierarchy
from oracle.fem import assemble_rhs

from callback_shapes import superellipse
from oracle.levelset import make_levelset

cm = pytest.importorskip("paper_2508_11608_gb300")


def _rot(a, b):
    import math
    ca, sa, cb, sb = math.cos(a), math.sin(a), math.cos(b), math.sin(b)
    Rz = np.array([[ca, -sa, 0], [sa, ca, 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, cb, -sb], [0, sb, cb]])
    return (Rz @ Rx).tolist()


SPH2 = {"kind": "sphere", "center": [0.031, 0.017], "radius": 0.7}
SPH3 = {"kind": "sphere", "center": [0.05, 0.03, 0.02], "radius": 0.7}
CASES = {
    "disk_q2": dict(dim=2, N=32, L=3, p=2, ls=SPH2),
    "disk_q3": dict(dim=2, N=16, L=2, p=3, ls=SPH2),
    "disk_q4": dict(dim=2, N=16, L=2, p=4, ls=SPH2),
    "ball_q2": dict(dim=3, N=8, L=2, p=2, ls=SPH3),
    "ball_q1": dict(dim=3, N=16, L=3, p=1, ls=SPH3),
    "flower_q2": dict(dim=2, N=32, L=3, p=2, ls={"kind": "flower", "center": [0.02, -0.03], "lobes": 5,
                                                 "phase": 0.4}),
    "ellipsoid_q2": dict(dim=3, N=8, L=2, p=2, ls={"kind": "ellipsoid", "center": [0.03, -0.02, 0.01],
                                                   "axes": [0.7, 0.5, 0.45], "rot": _rot(0.3, 0.5)}),
    "torus_q2": dict(dim=3, N=16, L=2, p=2, ls={"kind": "torus", "center": [0.02, 0.01, -0.03],
                                                "rot": _rot(0.4, 0.7), "major": 0.6, "minor": 0.2}),
    "disk_q1": dict(dim=2, N=32, L=3, p=1, ls=SPH2),
    # an oblique half-space: the cut runs to the edge of the box
    "plane3d_q2": dict(dim=3, N=8, L=2, p=2, ls={"kind": "plane", "normal": [0.36, 0.48, 0.8], "offset": 0.13}),
    "plane2d_q3": dict(dim=2, N=16, L=2, p=3, ls={"kind": "plane", "normal": [0.6, -0.8], "offset": -0.07}),
    # degenerate: a disk smaller than a cell, every patch cut, no interior one
    "tiny_q2": dict(dim=2, N=16, L=2, p=2, ls={"kind": "sphere", "center": [0.01, 0.02], "radius": 0.05}),
    # user level sets through point callbacks (sampled bounds on both sides)
    "callback_q2": dict(dim=2, N=32, L=3, p=2, ls=superellipse([0.03, -0.02], [0.7, 0.55])),
    "callback3d_q2": dict(dim=3, N=8, L=2, p=2, ls=superellipse([0.03, -0.02, 0.01], [0.7, 0.55, 0.6])),
}


@pytest.fixture(scope="module", params=list(CASES))
def pair(request):
    k = CASES[request.param]
    try:
        pb = cm.Problem(k["dim"], k["N"], k["L"], k["p"], levelset=k["ls"], host_only=True)
    except ImportError as e:
        pytest.skip(str(e))
    H = Hierarchy(make_levelset(k["ls"]), k["dim"], k["N"], k["p"], k["L"])
    return pb, H, k


def test_dof_numbering_matches(pair):
    pb, H, k = pair
    for l in range(k["L"]):
        assert np.array_equal(pb.dof_lattice(l), H.levels[l].lev.dof_nodes)
        X = pb.dof_coords(l)
        Xo = H.levels[l].lev.node_coords(H.levels[l].lev.dof_nodes)
        assert np.abs(X - Xo).max() < 1e-14


def test_cell_matrices_match(pair):
    pb, H, k = pair
    for l in range(k["L"]):
        parts = H.levels[l].parts
        lev = H.levels[l].lev
        for c, K in parts["cut"].items():
            Kp = pb.host_cell_matrix(l, c)
            assert np.abs(Kp - K).max() <= 1e-12 * np.abs(K).max()
        unc = np.nonzero(lev.active & ~lev.cut)[0]
        if unc.size:
            Kp = pb.host_cell_matrix(l, int(unc[0]))
            assert np.abs(Kp - parts["Kref"]).max() <= 1e-13 * np.abs(parts["Kref"]).max()


def test_rhs_matches(pair):
    pb, H, k = pair
    b, bo = pb.host_rhs(), H.rhs()
    assert np.abs(b - bo).max() <= 1e-13 * np.abs(bo).max()


def test_user_rhs_with_the_sine_data_is_the_manufactured_rhs(pair):
    pb, _, k = pair
    d = k["dim"]
    u = lambda x: float(np.prod(np.sin(np.pi * np.asarray(x))))
    b = pb.rhs_user(lambda x: d * np.pi ** 2 * u(x), u)
    bm = pb.host_rhs()
    assert np.abs(b - bm).max() <= 1e-14 * np.abs(bm).max()


def test_user_rhs_matches_the_oracle_for_polynomial_data(pair):
    """u = 1 + x + 2 y^2 (+ z^3 in 3D), f = -Laplace u: source and Dirichlet
    data both nonzero, neither tied to the built-in sine solution."""
    pb, H, k = pair
    d = k["dim"]

    def u_pt(x):
        return 1.0 + x[0] + 2.0 * x[1] ** 2 + (x[2] ** 3 if d == 3 else 0.0)

    def f_pt(x):
        return -4.0 - (6.0 * x[2] if d == 3 else 0.0)

    def u_arr(X):
        return 1.0 + X[:, 0] + 2.0 * X[:, 1] ** 2 + (X[:, 2] ** 3 if d == 3 else 0.0)

    def f_arr(X):
        return -4.0 - (6.0 * X[:, 2] if d == 3 else 0.0 * X[:, 0])

    fine = H.fine
    bo = assemble_rhs(fine.lev, H.gamma_D, H.q, u=u_arr, f=f_arr)
    b = pb.rhs_user(f_pt, u_pt)
    assert np.abs(b - bo).max() <= 1e-13 * np.abs(bo).max()
    # a missing function is zero: the two parts add up to the whole
    b_f, b_g = pb.rhs_user(f_pt, None), pb.rhs_user(None, u_pt)
    assert np.abs(b_f + b_g - b).max() <= 1e-14 * np.abs(b).max()
    assert np.abs(b_g - assemble_rhs(fine.lev, H.gamma_D, H.q, u=u_arr, f=lambda X: 0.0 * X[:, 0])).max() \
        <= 1e-13 * np.abs(bo).max()


def test_patches_and_inverses_match(pair):
    pb, H, k = pair
    d = k["dim"]
    for l in range(1, k["L"]):
        P = H.levels[l].patches
        lev = H.levels[l].lev
        N = lev.N
        pack = lambda v: int(sum(int(v[i]) * (N + 1) ** i for i in range(d)))
        inter, cut = pb.host_patches(l)
        o_inter = sorted(pack(v) for v, c in zip(P.verts, P.cut) if not c)
        assert sorted(inter) == o_inter
        o_cut = {pack(v): j for j, (v, c) in enumerate(zip(P.verts, P.cut)) if c}
        assert sorted(v for v, _, _ in cut) == sorted(o_cut)
        for v, nodes, inv in cut:
            j = o_cut[v]
            onodes = lev.dof_nodes[P.I[j]]
            assert sorted(nodes.tolist()) == sorted(onodes.tolist())
            order = np.argsort(onodes)
            Aj = P.Aj[j][np.ix_(order, order)]
            po = np.argsort(nodes)
            invs = inv[np.ix_(po, po)]
            I = invs @ Aj
            # a backward-stable inverse leaves about u cond(A_j); the Q4
            # patches on the 16² disk reach cond 3e7
            tol = max(1e-9, 1e-14 * np.linalg.cond(Aj))
            assert np.abs(I - np.eye(len(nodes))).max() < tol


def test_callback_level_set_needs_both_functions():
    spec = dict(superellipse([0.0, 0.0], [0.7, 0.6]))
    ls = cm._lib.make_levelset(spec)
    ls.grad = cm._lib.GRAD_FN()  # NULL
    lib = cm._lib.load()
    mesh = cm._lib.cf_mesh(2, 8, -1.0, 1.0, 1)
    import ctypes
    out = ctypes.c_void_p()
    st = lib.cf_setup_host(ctypes.byref(mesh), ctypes.byref(ls), 2, None, ctypes.byref(out))
    assert st == 1 and not out.value  # CF_EINVAL


def test_invalid_arguments_are_rejected():
    with pytest.raises(cm.CutmgError):
        cm.Problem(3, 16, 3, 3, center=[0, 0, 0], radius=0.5, host_only=True)  # 3D Q3 unsupported
    with pytest.raises(cm.CutmgError):
        cm.Problem(3, 16, 3, 4, center=[0, 0, 0], radius=0.5, host_only=True)  # 3D Q4 unsupported
    with pytest.raises(cm.CutmgError):
        cm.Problem(2, 16, 2, 5, center=[0, 0], radius=0.5, host_only=True)  # degree above 4
    with pytest.raises(cm.CutmgError):
        cm.Problem(2, 12, 4, 2, center=[0, 0], radius=0.5, host_only=True)  # 12 not divisible by 8
    with pytest.raises(cm.CutmgError):
        cm.Problem(2, 16, 2, 2, center=[0, 0], radius=-1.0, host_only=True)


def test_degenerate_domains_are_rejected():
    # no active cell: the domain misses the mesh
    with pytest.raises(cm.CutmgError, match="without active cells"):
        cm.Problem(2, 16, 2, 2, center=[5.0, 5.0], radius=0.5, host_only=True)
    # no cut cell: no Nitsche terms, the operator would be singular
    with pytest.raises(cm.CutmgError, match="no cut cell"):
        cm.Problem(2, 16, 2, 2, center=[0.0, 0.0], radius=10.0, host_only=True)
    # the coarsest level is solved densely: its size is bounded
    with pytest.raises(cm.CutmgError, match="coarsest level has 62351 DoFs"):
        cm.Problem(3, 32, 1, 2, center=[0.05, 0.03, 0.02], radius=0.7, host_only=True)


def test_footprint_estimate_grows_with_the_mesh():
    small = cm.Problem(3, 16, 3, 2, center=[0.05, 0.03, 0.02], radius=0.7, host_only=True)
    large = cm.Problem(3, 32, 4, 2, center=[0.05, 0.03, 0.02], radius=0.7, host_only=True)
    fs, fl = small.footprint(), large.footprint()
    # at least the FP64 + FP32 cut-patch inverses and the box vectors
    inv = small.stats()["inverse_entries"]
    assert fs >= 12 * inv
    assert fl > 4 * fs


@pytest.mark.parametrize("dim,N,L,p,spec", [
    (3, 16, 3, 2, {"kind": "sphere", "center": [0.05, 0.03, 0.02], "radius": 0.7}),
    (2, 64, 4, 3, {"kind": "flower", "center": [0.01, -0.02], "lobes": 5, "phase": 0.3}),
    (3, 16, 2, 1, {"kind": "torus", "center": [0.0, 0.0, 0.0], "major": 0.6, "minor": 0.2,
                   "rot": [[1, 0, 0], [0, 1, 0], [0, 0, 1]]}),
])
def test_pre_setup_footprint_equals_the_built_problems(dim, N, L, p, spec):
    """cf_footprint needs no built problem (sizes only, no quadrature, matrices
    or inverses) and gives the same bytes as the estimate from the full host
    setup."""
    pre = cm.footprint(dim, N, L, p, spec)
    built = cm.Problem(dim, N, L, p, levelset=spec, host_only=True).footprint()
    assert pre == built
    with pytest.raises(cm.CutmgError):
        cm.footprint(3, 16, 3, 3, spec)  # 3D Q3 is refused as by cf_setup


def test_interior_patch_update_is_the_exact_local_solve(pair):
    """x_I <- A_I^{-1} b_I - A_I^{-1} A_{I,B} x_B with A_I, A_{I,B} taken from
    the oracle's assembled matrix at interior patches (Sec. 2.3), and the
    rows of interior-patch DoFs reach no node outside the closure."""
    pb, H, k = pair
    d, p = k["dim"], k["p"]
    C, M = 2 * p + 1, 2 * p - 1
    for l in range(1, k["L"]):
        P = H.levels[l].patches
        lev = H.levels[l].lev
        A = H.levels[l].A.tocsr()
        W = pb.host_interior_update(l)
        inter = [j for j in range(len(P.verts)) if not P.cut[j]]
        for j in inter[:: max(1, len(inter) // 6)]:
            v = P.verts[j]
            cl = []
            for kc in range(C ** d):
                c, t = [], kc
                for _ in range(d):
                    c.append(t % C)
                    t //= C
                cl.append((sum((p * (int(v[q]) - 1) + c[q]) * lev.n ** q for q in range(d)),
                           all(1 <= c[q] <= C - 2 for q in range(d))))
            dofs = np.array([lev.node_to_dof[nd] for nd, _ in cl])
            inner = np.array([i for i, (_, a) in enumerate(cl) if a])
            outer = np.array([i for i, (_, a) in enumerate(cl) if not a])
            assert (dofs >= 0).all() and inner.size == M ** d
            AI = A[dofs[inner]][:, dofs[inner]].toarray()
            AIB = A[dofs[inner]][:, dofs[outer]].toarray()
            rows = A[dofs[inner]]
            assert set(rows.indices.tolist()) <= set(dofs.tolist())
            Wo = np.zeros_like(W)
            AIinv = np.linalg.inv(AI)
            Wo[:, inner] = AIinv
            Wo[:, outer] = -AIinv @ AIB
            assert np.abs(W - Wo).max() <= 1e-10 * np.abs(Wo).max()


def test_diagonal_matches_the_assembled_matrix(pair):
    _, H, k = pair
    # the diagonal is built for the Chebyshev smoother, which scales by it
    pb = cm.Problem(k["dim"], k["N"], k["L"], k["p"], levelset=k["ls"], host_only=True,
                    smoother=cm.CF_SMOOTHER_CHEBYSHEV)
    for l in range(1, k["L"]):
        d = pb.host_diagonal(l)
        do = H.levels[l].A.diagonal()
        assert np.abs(d - do).max() <= 1e-13 * np.abs(do).max()


def test_coarse_inverse_inverts_the_assembled_coarsest_matrix(pair):
    """The coarsest solve's explicit inverse (exact solve on the coarsest mesh,
    Sec. 2.2) against the oracle's assembled A_0: A_0 X = I and X equal to the
    LAPACK inverse, both within rounding amplified by the condition number,
    and X exactly symmetric (the library fills both triangles from one)."""
    pb, H, _ = pair
    X = pb.host_coarse_inverse()
    A0 = H.levels[0].A.toarray()
    ref = np.linalg.inv(A0)
    tol = 1e-14 * np.linalg.cond(A0)
    assert np.array_equal(X, X.T)
    assert np.abs(A0 @ X - np.eye(len(A0))).max() <= tol
    assert np.abs(X - ref).max() <= tol * np.abs(ref).max()


@pytest.mark.parametrize("name", ["ball_q2", "torus_q2", "disk_q3"])
def test_setup_is_the_same_on_any_number_of_threads(name):
    """The served form builds a request on however many host cores are free;
    every array of the setup must come out bit for bit the same."""
    k = CASES[name]
    a = cm.Problem(k["dim"], k["N"], k["L"], k["p"], levelset=k["ls"], host_only=True, setup_threads=1)
    for t in (3, 7):  # 7: the parallel loops' blocks split unevenly
        _same_setup(k, a, cm.Problem(k["dim"], k["N"], k["L"], k["p"], levelset=k["ls"], host_only=True,
                                     setup_threads=t))


def _same_setup(k, a, b):
    assert np.array_equal(a.host_rhs(), b.host_rhs())
    for l in range(k["L"]):
        assert a.n_dofs(l) == b.n_dofs(l)
        assert np.array_equal(a.dof_lattice(l), b.dof_lattice(l))
    assert np.array_equal(a.host_coarse_inverse(), b.host_coarse_inverse())
    for l in range(1, k["L"]):
        ia, ca = a.host_patches(l)
        ib, cb = b.host_patches(l)
        assert ia == ib and len(ca) == len(cb)
        for (va, na, Xa), (vb, nb, Xb) in zip(ca, cb):
            assert va == vb and np.array_equal(na, nb) and np.array_equal(Xa, Xb)
    L = k["L"] - 1
    for c in range(k["N"] ** k["dim"]):
        try:
            Ka = a.host_cell_matrix(L, c)
        except cm.CutmgError:  # inactive cell
            continue
        assert np.array_equal(Ka, b.host_cell_matrix(L, c))
