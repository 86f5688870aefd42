"""Level-set functions for the oracle (Sec. 2, "analytic level set function",
Sec. 4 setup).  Omega = {phi < 0}, Gamma = {phi = 0}.

Each level set provides
  phi(X)                 values at points X (..., d)
  grad(X)                gradient at points
  box_minmax(lo, hi)     exact min and max of phi over a closed box (degenerate
                         sides allowed), used for classification and to drop
                         functions without a zero in a box
  grad_sign_const(k, lo, hi)
                         True when d phi / d x_k has one strict sign on the box
                         (monotonicity test of the dimension-reduction rule)
"""

import numpy as np


class Sphere:
    """phi(x) = |x - c| - r: a disk (d = 2) or ball (d = 3)."""

    kind = "sphere"

    def __init__(self, center, radius):
        self.c = np.asarray(center, dtype=np.float64)
        self.r = float(radius)
        self.d = len(self.c)

    def _dist2(self, X):
        X = np.asarray(X, dtype=np.float64)
        s = None
        for k in range(self.d):
            dk = X[..., k] - self.c[k]
            s = dk * dk if s is None else s + dk * dk
        return s

    def phi(self, X):
        return np.sqrt(self._dist2(X)) - self.r

    def grad(self, X):
        X = np.asarray(X, dtype=np.float64)
        nrm = np.sqrt(self._dist2(X))
        return (X - self.c) / nrm[..., None]

    def box_minmax(self, lo, hi):
        smin = 0.0
        smax = 0.0
        for k in range(self.d):
            a = lo[k] - self.c[k]
            b = hi[k] - self.c[k]
            near = a if a > 0 else (-b if b < 0 else 0.0)
            far = max(abs(a), abs(b))
            smin = smin + near * near
            smax = smax + far * far
        return np.sqrt(smin) - self.r, np.sqrt(smax) - self.r

    def grad_sign_const(self, k, lo, hi):
        return bool(self.c[k] < lo[k] or self.c[k] > hi[k])


class Plane:
    """phi(x) = n . x - a (a half space); flat interfaces make every cut rule
    exact for polynomials, which the tests use as a pin."""

    kind = "plane"

    def __init__(self, normal, offset):
        self.n = np.asarray(normal, dtype=np.float64)
        self.a = float(offset)
        self.d = len(self.n)

    def phi(self, X):
        X = np.asarray(X, dtype=np.float64)
        s = None
        for k in range(self.d):
            t = self.n[k] * X[..., k]
            s = t if s is None else s + t
        return s - self.a

    def grad(self, X):
        X = np.asarray(X, dtype=np.float64)
        return np.broadcast_to(self.n, X.shape).copy()

    def box_minmax(self, lo, hi):
        mn = -self.a
        mx = -self.a
        for k in range(self.d):
            u = self.n[k] * lo[k]
            v = self.n[k] * hi[k]
            mn += min(u, v)
            mx += max(u, v)
        return mn, mx

    def grad_sign_const(self, k, lo, hi):
        return bool(self.n[k] != 0.0)


def make_levelset(spec):
    """Build a level set from a plain dict: {"kind": "sphere", "center": [...],
    "radius": r} or {"kind": "plane", "normal": [...], "offset": a}."""
    kind = spec["kind"]
    if kind == "sphere":
        return Sphere(spec["center"], spec["radius"])
    if kind == "plane":
        return Plane(spec["normal"], spec["offset"])
    raise ValueError(f"unknown level set kind {kind!r}")
