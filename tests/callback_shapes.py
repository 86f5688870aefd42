"""Level sets given only as point callbacks (phi, grad), for the tests of the
user level-set path.  Vectorised over X of shape (..., d) with +, -, *, / and
sqrt only, so one point at a time and a whole array give the same bits."""

import numpy as np


def superellipse(center, axes):
    """phi(x) = (sum_k ((x_k - c_k) / a_k)^4)^(1/4) - 1: a rounded box, not a
    distance function (|grad phi| varies), with area 4 a b G(5/4)^2 / G(3/2)
    in 2D and volume 8 a b c G(5/4)^3 / G(7/4) in 3D."""
    c = np.asarray(center, dtype=np.float64)
    a = np.asarray(axes, dtype=np.float64)
    d = len(c)

    def parts(X):
        X = np.asarray(X, dtype=np.float64)
        U = [(X[..., k] - c[k]) / a[k] for k in range(d)]
        s = U[0] * U[0] * U[0] * U[0]
        for k in range(1, d):
            s = s + U[k] * U[k] * U[k] * U[k]
        return U, np.sqrt(np.sqrt(s))

    def phi(X):
        return parts(X)[1] - 1.0

    def grad(X):
        U, q = parts(X)
        q3 = q * q * q
        return np.stack([U[k] * U[k] * U[k] / (a[k] * q3) for k in range(d)], axis=-1)

    return {"kind": "callback", "dim": d, "phi": phi, "grad": grad}


def distance_sphere(center, radius):
    """|x - c| - r through callbacks (a distance function: |grad phi| = 1)."""
    c = np.asarray(center, dtype=np.float64)
    d = len(c)

    def dist(X):
        X = np.asarray(X, dtype=np.float64)
        s = None
        for k in range(d):
            t = X[..., k] - c[k]
            s = t * t if s is None else s + t * t
        return np.sqrt(s)

    def phi(X):
        return dist(X) - radius

    def grad(X):
        X = np.asarray(X, dtype=np.float64)
        return (X - c) / dist(X)[..., None]

    return {"kind": "callback", "dim": d, "phi": phi, "grad": grad}
