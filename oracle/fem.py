"""Assembled CutFEM operator of one level (Sec. 2.1), FP64, as a scipy CSR
matrix: the plain definition of A_l.

  a_l(u, v) = (grad u, grad v)_Omega - (d_n u, v)_Gamma - (u, d_n v)_Gamma
              + (gamma_D / h) (u, v)_Gamma                       eq. "cutfem_nitsche"
  g_l(u, v) = sum_{F in F_G} sum_{k=1..p} gamma_k h^(2k-1)/(k!)^2
              ([d_n^k u], [d_n^k v])_F                           eq. "cutfem-ghost"

Readings (the paper leaves them open):
* active cell: min_T phi < 0; cut cell: min_T phi < 0 < max_T phi;
* the k = 0 ghost term vanishes for continuous V_l and is dropped;
* the face weight is h_F^(2k-1)/(k!)^2, the scaling of the face ghost penalty
  the paper cites (Burman-Hansbo 2012, and the deal.II step-85 construction it
  says it follows); the printed h_F^(2k+1) weakens the penalty by h^2 against
  the stiffness, and with it A_l is indefinite on a 64^3 ball (a sliver cut at
  the top cap gives a negative eigenvalue of a patch matrix);
* h_F = h; gamma_D is one constant per level, used as gamma_D / h;
* right-hand side b_i = (f, phi_i)_Omega + (g, gamma_D/h phi_i - d_n phi_i)_Gamma
  (the consistent Nitsche data term for u = g on Gamma);
* uncut cells and faces use tensor Gauss rules exact for the integrands.

Lattice conventions: cell (c_0, .., c_{d-1}) has flat index sum c_k N^k;
node (i_0, ..) of the (pN+1)^d lattice has flat index sum i_k n^k; active
nodes are numbered in increasing flat index (first coordinate fastest).
"""

import math

import numpy as np
import scipy.sparse as sp

from .basis import Basis1D, local_multi_indices, tensor_values_grads
from .quadrature import cut_cell_rule, gauss01


def tensor_rule01(q, d):
    """q^d tensor Gauss points on [0,1]^d and their weights."""
    x, w = gauss01(q)
    X = np.meshgrid(*([x] * d), indexing="ij")
    W = np.meshgrid(*([w] * d), indexing="ij")
    xi = np.stack([g.ravel() for g in X], axis=-1)
    wq = np.ones(xi.shape[0])
    for g in W:
        wq = wq * g.ravel()
    return xi, wq


def _unflat(flat, n, d):
    out = []
    for _ in range(d):
        out.append(flat % n)
        flat = flat // n
    return np.stack(out, axis=-1)


class Level:
    """Mesh level: classification, node numbering, cell -> DoF maps."""

    def __init__(self, ls, d, N, p, lo=-1.0, hi=1.0):
        self.ls, self.d, self.N, self.p = ls, d, N, p
        self.lo, self.hi = float(lo), float(hi)
        self.h = (self.hi - self.lo) / N
        self.n = p * N + 1
        ncell = N ** d
        cidx = _unflat(np.arange(ncell), N, d)
        self.cell_multi = cidx
        clo = self.lo + self.h * cidx
        chi = self.lo + self.h * (cidx + 1)
        mn = np.empty(ncell)
        mx = np.empty(ncell)
        for c in range(ncell):
            mn[c], mx[c] = ls.box_minmax(clo[c], chi[c])
        self.active = mn < 0
        self.cut = (mn < 0) & (mx > 0)
        self.cell_lo = clo
        # local node offsets in the lattice
        mi = np.array(local_multi_indices(p, d))
        self.local_mi = mi
        strides = self.n ** np.arange(d)
        self.local_off = mi @ strides
        base = (p * cidx) @ strides
        self.cell_nodes = base[:, None] + self.local_off[None, :]
        node_act = np.zeros(self.n ** d, dtype=bool)
        node_act[self.cell_nodes[self.active].ravel()] = True
        self.node_active = node_act
        self.dof_nodes = np.nonzero(node_act)[0]
        self.ndof = self.dof_nodes.size
        self.node_to_dof = -np.ones(self.n ** d, dtype=np.int64)
        self.node_to_dof[self.dof_nodes] = np.arange(self.ndof)
        self.basis = Basis1D(p)

    def node_coords(self, nodes):
        """Physical coordinates of lattice nodes."""
        m = _unflat(np.asarray(nodes), self.n, self.d)
        c = np.minimum(m // self.p, self.N - 1)
        a = m - self.p * c
        return self.lo + self.h * (c + self.basis.nodes[a])

    def cell_dofs(self, c):
        return self.node_to_dof[self.cell_nodes[c]]

    def ghost_faces(self):
        """All (direction k, lower cell, upper cell) with both cells active
        and at least one of them cut: the set F_G."""
        out = []
        N, d = self.N, self.d
        for k in range(d):
            stride = N ** k
            for c in range(N ** d):
                if self.cell_multi[c, k] == N - 1:
                    continue
                u = c + stride
                if self.active[c] and self.active[u] and (self.cut[c] or self.cut[u]):
                    out.append((k, c, u))
        return out


def uncut_stiffness(lev):
    """Element stiffness of a cell inside Omega by (p+1)^d tensor Gauss points."""
    d, h = lev.d, lev.h
    xi, wq = tensor_rule01(lev.p + 1, d)
    _, G = tensor_values_grads(lev.basis, xi, d)
    G = G / h
    K = np.zeros((G.shape[1], G.shape[1]))
    for k in range(d):
        K += (G[k] * wq) @ G[k].T
    return K * h ** d


def cut_cell_matrix(lev, c, gamma_D, q):
    """Volume and Nitsche terms of a cut cell by the cut-cell rule."""
    lo = lev.cell_lo[c]
    hi = lo + lev.h
    vp, vw, spts, sw, sn = cut_cell_rule(lev.ls, lo, hi, q)
    h = lev.h
    _, G = tensor_values_grads(lev.basis, (vp - lo) / h, lev.d)
    G = G / h
    K = np.zeros((G.shape[1], G.shape[1]))
    for k in range(lev.d):
        K += (G[k] * vw) @ G[k].T
    if sw.size:
        V, Gs = tensor_values_grads(lev.basis, (spts - lo) / h, lev.d)
        Gs = Gs / h
        dn = np.einsum("kiq,qk->iq", Gs, sn)
        K -= (dn * sw) @ V.T + (V * sw) @ dn.T
        K += (gamma_D / h) * (V * sw) @ V.T
    return K


def ghost_face_matrix(lev, k, gammas):
    """Ghost penalty matrix of one face normal to direction k between a lower
    cell T1 and an upper cell T2, on the 2 (p+1)^d local DoFs [T1 | T2]."""
    d, p, h = lev.d, lev.p, lev.h
    tdims = [j for j in range(d) if j != k]
    tpts, tw = tensor_rule01(p + 1, len(tdims))
    nq = tw.size
    mi = lev.local_mi
    nb = len(mi)
    Gm = np.zeros((2 * nb, 2 * nb))
    for m in range(1, p + 1):
        J = np.zeros((2 * nb, nq))
        for side, xi_k in ((0, 1.0), (1, 0.0)):
            dk = lev.basis.eval(np.array([xi_k]), m)[:, 0] / h ** m
            for i, a in enumerate(mi):
                val = np.full(nq, dk[a[k]])
                for jj, j in enumerate(tdims):
                    val = val * lev.basis.eval(tpts[:, jj])[a[j]]
                J[side * nb + i] = val if side == 0 else -val
        coef = gammas[m - 1] * h ** (2 * m - 1) / math.factorial(m) ** 2
        Gm += coef * (J * tw) @ J.T * h ** (d - 1)
    return Gm


def assemble_level(lev, gamma_D, gammas, q):
    """Assembled A_l (CSR, ndof x ndof) and the per-cut-cell matrices."""
    rows, cols, vals = [], [], []
    Kref = uncut_stiffness(lev)
    unc = np.nonzero(lev.active & ~lev.cut)[0]
    if unc.size:
        D = lev.node_to_dof[lev.cell_nodes[unc]]
        nb = D.shape[1]
        rows.append(np.repeat(D, nb, axis=1).ravel())
        cols.append(np.tile(D, (1, nb)).ravel())
        vals.append(np.tile(Kref.ravel(), unc.size))
    cutmats = {}
    for c in np.nonzero(lev.cut)[0]:
        K = cut_cell_matrix(lev, c, gamma_D, q)
        cutmats[int(c)] = K
        D = lev.cell_dofs(c)
        rows.append(np.repeat(D, D.size))
        cols.append(np.tile(D, D.size))
        vals.append(K.ravel())
    faces = lev.ghost_faces()
    Gref = [ghost_face_matrix(lev, k, gammas) for k in range(lev.d)]
    for (k, c1, c2) in faces:
        D = np.concatenate([lev.cell_dofs(c1), lev.cell_dofs(c2)])
        rows.append(np.repeat(D, D.size))
        cols.append(np.tile(D, D.size))
        vals.append(Gref[k].ravel())
    r = np.concatenate(rows)
    cc = np.concatenate(cols)
    v = np.concatenate(vals)
    A = sp.csr_matrix((v, (r, cc)), shape=(lev.ndof, lev.ndof))
    A.sum_duplicates()
    return A, {"Kref": Kref, "cut": cutmats, "ghost_faces": faces, "Gref": Gref}


def sine_solution(X):
    """u(x) = prod_k sin(pi x_k): the manufactured solution of the workloads."""
    u = np.ones(X.shape[0])
    for k in range(X.shape[1]):
        u = u * np.sin(np.pi * X[:, k])
    return u


def assemble_rhs(lev, gamma_D, q, u=sine_solution, f=None):
    """b_i = (f, phi_i)_Omega + (g, gamma_D/h phi_i - d_n phi_i)_Gamma with
    g = u on Gamma and f = -Laplace u (= d pi^2 u for the sine solution)."""
    d, h = lev.d, lev.h
    if f is None:
        f = lambda X: d * np.pi ** 2 * u(X)
    b = np.zeros(lev.ndof)
    xi, wq = tensor_rule01(q, d)
    Vref, _ = tensor_values_grads(lev.basis, xi, d)
    for c in np.nonzero(lev.active & ~lev.cut)[0]:
        X = lev.cell_lo[c] + h * xi
        np.add.at(b, lev.cell_dofs(c), Vref @ (wq * f(X)) * h ** d)
    for c in np.nonzero(lev.cut)[0]:
        lo = lev.cell_lo[c]
        vp, vw, spts, sw, sn = cut_cell_rule(lev.ls, lo, lo + h, q)
        D = lev.cell_dofs(c)
        if vw.size:
            V, _ = tensor_values_grads(lev.basis, (vp - lo) / h, d)
            np.add.at(b, D, V @ (vw * f(vp)))
        if sw.size:
            V, G = tensor_values_grads(lev.basis, (spts - lo) / h, d)
            dn = np.einsum("kiq,qk->iq", G / h, sn)
            np.add.at(b, D, ((gamma_D / h) * V - dn) @ (sw * u(spts)))
    return b


def l2_error(lev, xvec, q, u=sine_solution):
    """||u_h - u||_{L2(Omega)} with the same volume rules."""
    d, h = lev.d, lev.h
    xi, wq = tensor_rule01(q, d)
    Vref, _ = tensor_values_grads(lev.basis, xi, d)
    err2 = 0.0
    for c in np.nonzero(lev.active)[0]:
        lo = lev.cell_lo[c]
        xc = xvec[lev.cell_dofs(c)]
        if lev.cut[c]:
            vp, vw, _, _, _ = cut_cell_rule(lev.ls, lo, lo + h, q)
            if not vw.size:
                continue
            V, _ = tensor_values_grads(lev.basis, (vp - lo) / h, d)
            e = xc @ V - u(vp)
            err2 += np.sum(vw * e * e)
        else:
            X = lo + h * xi
            e = xc @ Vref - u(X)
            err2 += np.sum(wq * e * e) * h ** d
    return math.sqrt(err2)
