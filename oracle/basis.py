"""Tensor-product Q_p basis with nodes in the Gauss-Lobatto points (Sec. 2.1,
after eq. "spaces"), on the reference interval [0, 1]."""

import math

import numpy as np
from numpy.polynomial import Polynomial


def gll_nodes(p):
    """Gauss-Lobatto points on [0, 1] for degree p = 1, 2, 3, 4 (closed forms:
    the end points plus the roots of P_p', mapped from [-1, 1]: 0 for p = 2,
    +-1/sqrt(5) for p = 3, 0 and +-sqrt(3/7) for p = 4)."""
    if p == 1:
        return np.array([0.0, 1.0])
    if p == 2:
        return np.array([0.0, 0.5, 1.0])
    if p == 3:
        s = 1.0 / math.sqrt(5.0)
        return np.array([0.0, 0.5 * (1.0 - s), 0.5 * (1.0 + s), 1.0])
    if p == 4:
        s = math.sqrt(3.0 / 7.0)
        return np.array([0.0, 0.5 * (1.0 - s), 0.5, 0.5 * (1.0 + s), 1.0])
    raise ValueError("degree must be 1, 2, 3 or 4")


class Basis1D:
    """Lagrange polynomials l_a through the GLL nodes, with derivatives."""

    def __init__(self, p):
        self.p = p
        self.nodes = gll_nodes(p)
        self.polys = []
        for a in range(p + 1):
            others = [self.nodes[b] for b in range(p + 1) if b != a]
            den = 1.0
            for o in others:
                den *= self.nodes[a] - o
            self.polys.append(Polynomial.fromroots(others) / den)

    def eval(self, xi, m=0):
        """Array (p+1, len(xi)) of the m-th derivatives l_a^(m)(xi)."""
        xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
        out = np.empty((self.p + 1, xi.size))
        for a, P in enumerate(self.polys):
            out[a] = (P.deriv(m) if m > 0 else P)(xi)
        return out


def local_multi_indices(p, d):
    """Local node multi-indices of a cell, first coordinate fastest."""
    n1 = p + 1
    idx = []
    for flat in range((n1) ** d):
        a = []
        t = flat
        for _ in range(d):
            a.append(t % n1)
            t //= n1
        idx.append(tuple(a))
    return idx


def tensor_values_grads(basis, xi, d):
    """Values (nb, n) and reference gradients (d, nb, n) of the cell basis at
    reference points xi (n, d)."""
    xi = np.atleast_2d(xi)
    V1 = [basis.eval(xi[:, k]) for k in range(d)]
    D1 = [basis.eval(xi[:, k], 1) for k in range(d)]
    mi = local_multi_indices(basis.p, d)
    nb = len(mi)
    n = xi.shape[0]
    V = np.ones((nb, n))
    G = np.ones((d, nb, n))
    for i, a in enumerate(mi):
        for k in range(d):
            V[i] *= V1[k][a[k]]
            for j in range(d):
                G[j, i] *= (D1 if j == k else V1)[k][a[k]]
    return V, G
