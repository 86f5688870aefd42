"""Level-set functions for the oracle (Sec. 2, "analytic level set function",
Sec. 4 setup).  Omega = {phi < 0}, Gamma = {phi = 0}.

Each level set provides
  phi(X)                 values at points X (..., d)
  grad(X)                gradient at points
  box_minmax(lo, hi)     bounds of phi over a closed box (degenerate sides
                         allowed): exact for the sphere and the plane; for the
                         other shapes an interval enclosure, refined by
                         halving the box (all directions) while the sign is
                         undecided, at most BOX_DEPTH times
  grad_sign_const(k, lo, hi)
                         True when d phi / d x_k provably keeps one strict sign
                         on the box (monotonicity test of the cut quadrature)

A user level set given by point callbacks (Callback) has sampled bounds
instead; its docstring states them.

Interval enclosures use plain floating point (no outward rounding); the
library's setup evaluates the same expressions in the same order.
"""

import math

import numpy as np

BOX_DEPTH = 2


# ---------------------------------------------------------------------------
# closed intervals as (lo, hi) tuples

def iadd(a, b):
    return (a[0] + b[0], a[1] + b[1])


def isub(a, b):
    return (a[0] - b[1], a[1] - b[0])


def iscale(s, a):
    u, v = s * a[0], s * a[1]
    return (min(u, v), max(u, v))


def imul(a, b):
    p = (a[0] * b[0], a[0] * b[1], a[1] * b[0], a[1] * b[1])
    return (min(p), max(p))


def isqr(a):
    u, v = a[0] * a[0], a[1] * a[1]
    if a[0] <= 0.0 <= a[1]:
        return (0.0, max(u, v))
    return (min(u, v), max(u, v))


def isqrt(a):
    return (math.sqrt(max(a[0], 0.0)), math.sqrt(max(a[1], 0.0)))


def idiv(a, b):
    """a / b for an interval b not containing 0 (caller checks)."""
    return imul(a, (1.0 / b[1], 1.0 / b[0]))


def icos(a):
    lo, hi = a
    if hi - lo >= 2.0 * math.pi:
        return (-1.0, 1.0)
    c0, c1 = math.cos(lo), math.cos(hi)
    mn, mx = min(c0, c1), max(c0, c1)
    # a multiple of 2 pi inside -> max 1; an odd multiple of pi inside -> min -1
    k = math.ceil(lo / (2.0 * math.pi))
    if 2.0 * math.pi * k <= hi:
        mx = 1.0
    k = math.ceil((lo - math.pi) / (2.0 * math.pi))
    if math.pi + 2.0 * math.pi * k <= hi:
        mn = -1.0
    return (mn, mx)


def isin(a):
    return icos((a[0] - 0.5 * math.pi, a[1] - 0.5 * math.pi))


def _box_dist(lo, hi, c, d):
    """Exact min and max of |x - c| over a box."""
    smin = 0.0
    smax = 0.0
    for k in range(d):
        a = lo[k] - c[k]
        b = hi[k] - c[k]
        near = a if a > 0 else (-b if b < 0 else 0.0)
        far = max(abs(a), abs(b))
        smin = smin + near * near
        smax = smax + far * far
    return math.sqrt(smin), math.sqrt(smax)


def _refined(fn, lo, hi, d, depth=0):
    mn, mx = fn(lo, hi)
    if mn < 0.0 < mx and depth < BOX_DEPTH:
        free = [k for k in range(d) if hi[k] > lo[k]]
        mn, mx = math.inf, -math.inf
        for bits in range(1 << len(free)):
            clo = list(lo)
            chi = list(hi)
            for i, k in enumerate(free):
                mid = 0.5 * (lo[k] + hi[k])
                if (bits >> i) & 1:
                    clo[k] = mid
                else:
                    chi[k] = mid
            a, b = _refined(fn, clo, chi, d, depth + 1)
            mn, mx = min(mn, a), max(mx, b)
    return mn, mx


# ---------------------------------------------------------------------------

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
        dmin, dmax = _box_dist(lo, hi, self.c, self.d)
        return dmin - self.r, dmax - self.r

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


class Ellipsoid:
    """phi(x) = sqrt(sum_i (y_i / a_i)^2) - 1 with y = R (x - c): the
    ellipsoid with semi-axes a_i along the rows of the rotation R (d = 3)."""

    kind = "ellipsoid"

    def __init__(self, center, axes, rot):
        self.c = np.asarray(center, dtype=np.float64)
        self.a = np.asarray(axes, dtype=np.float64)
        self.R = np.asarray(rot, dtype=np.float64).reshape(3, 3)
        self.d = 3

    def _y(self, X):
        X = np.asarray(X, dtype=np.float64)
        D = [X[..., j] - self.c[j] for j in range(3)]
        return [self.R[i, 0] * D[0] + self.R[i, 1] * D[1] + self.R[i, 2] * D[2] for i in range(3)]

    def phi(self, X):
        y = self._y(X)
        s = None
        for i in range(3):
            t = y[i] / self.a[i]
            s = t * t if s is None else s + t * t
        return np.sqrt(s) - 1.0

    def grad(self, X):
        y = self._y(X)
        s = None
        for i in range(3):
            t = y[i] / self.a[i]
            s = t * t if s is None else s + t * t
        q = np.sqrt(s)
        g = [y[i] / (self.a[i] * self.a[i]) / q for i in range(3)]
        return np.stack([self.R[0, j] * g[0] + self.R[1, j] * g[1] + self.R[2, j] * g[2]
                         for j in range(3)], axis=-1)

    def _iy(self, lo, hi):
        D = [(lo[j] - self.c[j], hi[j] - self.c[j]) for j in range(3)]
        out = []
        for i in range(3):
            t = iscale(self.R[i, 0], D[0])
            t = iadd(t, iscale(self.R[i, 1], D[1]))
            t = iadd(t, iscale(self.R[i, 2], D[2]))
            out.append(t)
        return out

    def _natural(self, lo, hi):
        y = self._iy(lo, hi)
        s = isqr(iscale(1.0 / self.a[0], y[0]))
        s = iadd(s, isqr(iscale(1.0 / self.a[1], y[1])))
        s = iadd(s, isqr(iscale(1.0 / self.a[2], y[2])))
        q = isqrt(s)
        return q[0] - 1.0, q[1] - 1.0

    def box_minmax(self, lo, hi):
        return _refined(self._natural, lo, hi, 3)

    def grad_sign_const(self, k, lo, hi):
        # sign of sum_i R_ik y_i / a_i^2 (the positive factor 1/|.| dropped)
        y = self._iy(lo, hi)
        t = iscale(self.R[0, k] / (self.a[0] * self.a[0]), y[0])
        t = iadd(t, iscale(self.R[1, k] / (self.a[1] * self.a[1]), y[1]))
        t = iadd(t, iscale(self.R[2, k] / (self.a[2] * self.a[2]), y[2]))
        return bool(t[0] > 0.0 or t[1] < 0.0)


class Torus:
    """phi(x) = sqrt((sqrt(y_0^2 + y_1^2) - R0)^2 + y_2^2) - r0 with
    y = Q (x - c): the torus around the axis Q[2] (d = 3)."""

    kind = "torus"

    def __init__(self, center, rot, major, minor):
        self.c = np.asarray(center, dtype=np.float64)
        self.Q = np.asarray(rot, dtype=np.float64).reshape(3, 3)
        self.R0 = float(major)
        self.r0 = float(minor)
        self.d = 3

    def _y(self, X):
        X = np.asarray(X, dtype=np.float64)
        D = [X[..., j] - self.c[j] for j in range(3)]
        return [self.Q[i, 0] * D[0] + self.Q[i, 1] * D[1] + self.Q[i, 2] * D[2] for i in range(3)]

    def phi(self, X):
        y = self._y(X)
        rho = np.sqrt(y[0] * y[0] + y[1] * y[1])
        t = rho - self.R0
        return np.sqrt(t * t + y[2] * y[2]) - self.r0

    def grad(self, X):
        y = self._y(X)
        rho = np.sqrt(y[0] * y[0] + y[1] * y[1])
        t = rho - self.R0
        q = np.sqrt(t * t + y[2] * y[2])
        g = [t / q * y[0] / rho, t / q * y[1] / rho, y[2] / q]
        return np.stack([self.Q[0, j] * g[0] + self.Q[1, j] * g[1] + self.Q[2, j] * g[2]
                         for j in range(3)], axis=-1)

    def _iy(self, lo, hi):
        D = [(lo[j] - self.c[j], hi[j] - self.c[j]) for j in range(3)]
        out = []
        for i in range(3):
            t = iscale(self.Q[i, 0], D[0])
            t = iadd(t, iscale(self.Q[i, 1], D[1]))
            t = iadd(t, iscale(self.Q[i, 2], D[2]))
            out.append(t)
        return out

    def _natural(self, lo, hi):
        y = self._iy(lo, hi)
        rho = isqrt(iadd(isqr(y[0]), isqr(y[1])))
        t = (rho[0] - self.R0, rho[1] - self.R0)
        q = isqrt(iadd(isqr(t), isqr(y[2])))
        return q[0] - self.r0, q[1] - self.r0

    def box_minmax(self, lo, hi):
        return _refined(self._natural, lo, hi, 3)

    def grad_sign_const(self, k, lo, hi):
        y = self._iy(lo, hi)
        rho2 = iadd(isqr(y[0]), isqr(y[1]))
        if rho2[0] <= 0.0:
            return False
        rho = isqrt(rho2)
        t = (rho[0] - self.R0, rho[1] - self.R0)
        # q * dphi/dx_k = t/rho (Q0k y0 + Q1k y1) + Q2k y2  (q > 0 dropped)
        w = iadd(iscale(self.Q[0, k], y[0]), iscale(self.Q[1, k], y[1]))
        a = imul(idiv(t, rho), w)
        s = iadd(a, iscale(self.Q[2, k], y[2]))
        return bool(s[0] > 0.0 or s[1] < 0.0)


class Flower:
    """phi(x) = |x - c| - (r0 + a0 cos(m (theta - theta0))), theta the polar
    angle of x - c (d = 2): the curve r(theta) = 0.6 + 0.1 cos(m theta)
    rotated by theta0."""

    kind = "flower"

    def __init__(self, center, lobes, phase, base=0.6, amplitude=0.1):
        self.c = np.asarray(center, dtype=np.float64)
        self.m = int(lobes)
        self.t0 = float(phase)
        self.r0 = float(base)
        self.a0 = float(amplitude)
        self.d = 2

    def phi(self, X):
        X = np.asarray(X, dtype=np.float64)
        dx = X[..., 0] - self.c[0]
        dy = X[..., 1] - self.c[1]
        rho = np.sqrt(dx * dx + dy * dy)
        th = np.arctan2(dy, dx)
        return rho - (self.r0 + self.a0 * np.cos(self.m * (th - self.t0)))

    def grad(self, X):
        X = np.asarray(X, dtype=np.float64)
        dx = X[..., 0] - self.c[0]
        dy = X[..., 1] - self.c[1]
        r2 = dx * dx + dy * dy
        rho = np.sqrt(r2)
        th = np.arctan2(dy, dx)
        s = self.a0 * self.m * np.sin(self.m * (th - self.t0))
        return np.stack([dx / rho - s * dy / r2, dy / rho + s * dx / r2], axis=-1)

    def _theta(self, lo, hi):
        """Range of the polar angle over a box not containing c, in radians,
        possibly beyond pi when the box crosses the negative x half-axis."""
        xs = (lo[0] - self.c[0], hi[0] - self.c[0])
        ys = (lo[1] - self.c[1], hi[1] - self.c[1])
        ang = [math.atan2(y, x) for x in xs for y in ys]
        if xs[1] < 0.0 and ys[0] <= 0.0 <= ys[1]:
            ang = [a + 2.0 * math.pi if a < 0.0 else a for a in ang]
        return (min(ang), max(ang))

    def _contains_c(self, lo, hi):
        return lo[0] <= self.c[0] <= hi[0] and lo[1] <= self.c[1] <= hi[1]

    def _wave(self, lo, hi):
        if self._contains_c(lo, hi):
            return (-1.0, 1.0), None
        th = self._theta(lo, hi)
        arg = (self.m * (th[0] - self.t0), self.m * (th[1] - self.t0))
        return icos(arg), arg

    def _natural(self, lo, hi):
        dmin, dmax = _box_dist(lo, hi, self.c, 2)
        cw, _ = self._wave(lo, hi)
        return dmin - (self.r0 + self.a0 * cw[1]), dmax - (self.r0 + self.a0 * cw[0])

    def box_minmax(self, lo, hi):
        return _refined(self._natural, lo, hi, 2)

    def grad_sign_const(self, k, lo, hi):
        if self._contains_c(lo, hi):
            return False
        dx = (lo[0] - self.c[0], hi[0] - self.c[0])
        dy = (lo[1] - self.c[1], hi[1] - self.c[1])
        dmin, dmax = _box_dist(lo, hi, self.c, 2)
        _, arg = self._wave(lo, hi)
        sw = iscale(self.a0 * self.m, isin(arg))
        # rho^2 dphi/dx = dx rho - s dy ; rho^2 dphi/dy = dy rho + s dx
        rho = (dmin, dmax)
        if k == 0:
            v = isub(imul(dx, rho), imul(sw, dy))
        else:
            v = iadd(imul(dy, rho), imul(sw, dx))
        return bool(v[0] > 0.0 or v[1] < 0.0)


SAMPLE_INTERVALS = 4


class Callback:
    """A user level set known only through point values phi(X) and gradients
    grad(X) (vectorised callables over X of shape (..., d)).  The paper's
    examples are closed forms; for these no enclosure exists, so both bounds
    come from samples (a reading of the classification and the quadrature's
    monotonicity test for point-only level sets):

    * samples: the lattice of SAMPLE_INTERVALS + 1 points per free direction
      of the box, x_k = lo_k + (hi_k - lo_k) i / SAMPLE_INTERVALS (one point
      in a degenerate direction);
    * delta = half the diagonal of one lattice cell: every box point lies
      within delta of a sample;
    * box_minmax = (min phi - L delta, max phi + L delta), L the largest
      sampled |grad phi| (an exact enclosure when L bounds |grad phi| on the
      box, e.g. for distance functions, where L = 1);
    * grad_sign_const(k): every sampled d phi/d x_k has one strict sign and
      its smallest magnitude exceeds C_k delta, C_k the largest difference
      quotient of d phi/d x_k between neighbouring samples."""

    kind = "callback"

    def __init__(self, phi, grad, d):
        self._phi = phi
        self._grad = grad
        self.d = int(d)

    def phi(self, X):
        return np.asarray(self._phi(np.asarray(X, dtype=np.float64)), dtype=np.float64)

    def grad(self, X):
        return np.asarray(self._grad(np.asarray(X, dtype=np.float64)), dtype=np.float64)

    def _samples(self, lo, hi):
        d = len(lo)
        cnt = [SAMPLE_INTERVALS + 1 if hi[k] > lo[k] else 1 for k in range(d)]
        axes = [np.array([lo[k] + (hi[k] - lo[k]) * i / SAMPLE_INTERVALS for i in range(cnt[k])])
                for k in range(d)]
        # lexicographic with the first direction fastest
        grids = np.meshgrid(*axes, indexing="ij")
        X = np.stack([g.transpose(tuple(range(d))[::-1]).ravel() for g in grids], axis=-1)
        s = 0.0
        for k in range(d):
            t = (hi[k] - lo[k]) / SAMPLE_INTERVALS
            s = t * t if k == 0 else s + t * t
        delta = 0.5 * math.sqrt(s)
        return X, cnt, delta

    def box_minmax(self, lo, hi):
        X, _, delta = self._samples(lo, hi)
        v = self.phi(X)
        G = self.grad(X)
        nrm = G[:, 0] * G[:, 0]
        for k in range(1, G.shape[1]):
            nrm = nrm + G[:, k] * G[:, k]
        lip = float(np.sqrt(nrm).max())
        return float(v.min()) - lip * delta, float(v.max()) + lip * delta

    def grad_sign_const(self, k, lo, hi):
        X, cnt, delta = self._samples(lo, hi)
        gk = self.grad(X)[:, k]
        if not (np.all(gk > 0.0) or np.all(gk < 0.0)):
            return False
        d = len(lo)
        A = gk.reshape(tuple(cnt[::-1]))  # axis d-1-j is direction j
        curv = 0.0
        for j in range(d):
            if cnt[j] == 1:
                continue
            step = (hi[j] - lo[j]) / SAMPLE_INTERVALS
            diff = np.abs(np.diff(A, axis=d - 1 - j)) / step
            curv = max(curv, float(diff.max()))
        return bool(float(np.abs(gk).min()) > curv * delta)


def make_levelset(spec):
    """Build a level set from a plain dict (kind and its parameters)."""
    kind = spec["kind"]
    if kind == "callback":
        return Callback(spec["phi"], spec["grad"], spec["dim"])
    if kind == "sphere":
        return Sphere(spec["center"], spec["radius"])
    if kind == "plane":
        return Plane(spec["normal"], spec["offset"])
    if kind == "ellipsoid":
        return Ellipsoid(spec["center"], spec["axes"], spec["rot"])
    if kind == "torus":
        return Torus(spec["center"], spec["rot"], spec["major"], spec["minor"])
    if kind == "flower":
        return Flower(spec["center"], spec["lobes"], spec["phase"], spec.get("base", 0.6),
                      spec.get("amplitude", 0.1))
    raise ValueError(f"unknown level set kind {kind!r}")
