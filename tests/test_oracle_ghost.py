"""Pins of the oracle's ghost-face penalty (eq. "cutfem-ghost", Sec. 2.1)
against closed forms.

The penalty of one face F normal to e_k is
    g_F(u, u) = sum_{m=1..p} gamma_m h^(2m-1) / (m!)^2 int_F [d^m u / dx_k^m]^2 ds
(reading: weight h^(2m-1), the Burman-Hansbo scaling; the printed h^(2m+1)
makes the operator indefinite, pinned below).  For the kink functions
u_j = ((x_k - x_F)_+)^j, j <= p, the only nonzero jump across the face at
x_k = x_F is that of the j-th derivative, which is j!; on every other face the
function is polynomial (or independent of the face's normal coordinate), so
    g(u_j, u_j) = gamma_j h^(2j-1) |F| per face at x_F, |F| = h^(d-1).
Distinct gamma_m per order make a wrong order index, a wrong power of h, a
missing factorial or a missing face measure each change the value."""

import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.fem import Level, assemble_level, ghost_face_matrix
from oracle.levelset import Plane, Sphere

GAMMAS = [0.1, 0.23, 0.37, 0.51]


def _face_values(lev, k, xF, j):
    """Values of ((x_k - x_F)_+)^j at the local nodes [T1 | T2] of the face
    matrix, T1 = [x_F - h, x_F] and T2 = [x_F, x_F + h] along k."""
    nodes = lev.basis.nodes
    vals = []
    for side in (0, 1):
        for a in lev.local_mi:
            xk = xF + lev.h * (nodes[a[k]] - (1.0 if side == 0 else 0.0))
            vals.append(max(xk - xF, 0.0) ** j)
    return np.array(vals)


@pytest.mark.parametrize("d,p", [(2, 1), (2, 2), (2, 3), (2, 4), (3, 1), (3, 2)])
def test_face_matrix_on_kinks_is_gamma_h_power_face_measure(d, p):
    lev = Level(Sphere([0.0] * d, 0.55), d, 8, p)
    h = lev.h
    xF = 0.25  # any face position: the face matrix is translation invariant
    for k in range(d):
        G = ghost_face_matrix(lev, k, GAMMAS[:p])
        for j in range(1, p + 1):
            u = _face_values(lev, k, xF, j)
            expect = GAMMAS[j - 1] * h ** (2 * j - 1) * h ** (d - 1)
            # the Q4 face matrix (fourth derivatives) has entries up to 1e3
            # against values of 6e-3 for j = 1: the sum cancels about 1e5
            # and its rounding reaches a few 1e-12 relative
            assert u @ G @ u == pytest.approx(expect, rel=1e-13 if p < 4 else 1e-11, abs=0), (k, j)


@pytest.mark.parametrize("d,p", [(2, 1), (2, 2), (2, 3), (3, 2)])
def test_face_matrix_on_polynomials_across_the_face_is_zero(d, p):
    """u = (x_k - x_F)^j on both sides (no kink): every jump vanishes."""
    lev = Level(Sphere([0.0] * d, 0.55), d, 8, p)
    nodes = lev.basis.nodes
    for k in range(d):
        G = ghost_face_matrix(lev, k, GAMMAS[:p])
        for j in range(1, p + 1):
            u = np.array([(lev.h * (nodes[a[k]] - (1.0 if s == 0 else 0.0))) ** j
                          for s in (0, 1) for a in lev.local_mi])
            assert abs(u @ G @ u) < 1e-15


def _ghost_operator(lev, A, info):
    rows, cols, vals = [], [], []
    for (k, c1, c2) in info["ghost_faces"]:
        D = np.concatenate([lev.cell_dofs(c1), lev.cell_dofs(c2)])
        rows.append(np.repeat(D, D.size))
        cols.append(np.tile(D, D.size))
        vals.append(info["Gref"][k].ravel())
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=A.shape)


@pytest.mark.parametrize("d,N,p", [(2, 16, 2), (2, 16, 3), (3, 8, 2)])
def test_assembled_ghost_energy_of_kinks_counts_faces_on_the_plane(d, N, p):
    """On a whole level: g(u_j, u_j) = gamma_j h^(2j-1) h^(d-1) times the
    number of ghost faces normal to e_k that lie in the plane x_k = x_F."""
    lev = Level(Sphere([0.02] * d, 0.7), d, N, p)
    A, info = assemble_level(lev, 20.0 * p * p, GAMMAS[:p], p + 2)
    G = _ghost_operator(lev, A, info)
    X = lev.node_coords(lev.dof_nodes)
    h = lev.h
    for k in range(d):
        for plane in (N // 4, 3 * N // 4):
            xF = lev.lo + plane * h
            nf = sum(1 for (kk, c1, _) in info["ghost_faces"]
                     if kk == k and lev.cell_multi[c1, k] == plane - 1)
            assert nf > 0
            for j in range(1, p + 1):
                u = np.maximum(X[:, k] - xF, 0.0) ** j
                expect = nf * GAMMAS[j - 1] * h ** (2 * j - 1) * h ** (d - 1)
                assert u @ (G @ u) == pytest.approx(expect, rel=1e-12), (k, plane, j)


def test_printed_face_weight_makes_the_operator_indefinite():
    """Reading of eq. "cutfem-ghost": with the printed weight h^(2m+1) (h^2
    times the one used) the level operator of a plane cut that leaves a 1 %
    sliver of a cell column has a negative eigenvalue (2D Q1, 8^2); with
    h^(2m-1) it is positive definite."""
    d, N, p = 2, 8, 1
    h = 2.0 / N
    lev = Level(Plane([1.0, 0.0], -1.0 + (N // 2 + 0.01) * h), d, N, p)
    A, info = assemble_level(lev, 20.0 * p * p, [0.1], p + 2)
    G = _ghost_operator(lev, A, info)
    used = np.linalg.eigvalsh(A.toarray())[0]
    printed = np.linalg.eigvalsh((A - G + h * h * G).toarray())[0]
    assert used > 1e-2
    assert printed < -1e-2
