"""Cut-cell quadrature by dimension reduction, the algorithm the paper uses for
the rules on intersected cells (Sec. 3: "substitute quadrature ... computed
upfront on the CPU", citing Saye 2015).

The paper names the algorithm but fixes none of its parameters.  This oracle
fixes them as follows (the CUDA library's own setup implements the same
reading independently):

* q Gauss-Legendre points on every one-dimensional sub-interval;
* height direction: the free directions ordered by |d phi/d x_k| at the box
  centre (descending, ties to the lower k); the first one in which every
  function of the current stage is strictly monotone over its box is taken;
* when no direction qualifies the box is halved in every free direction, at
  most MAX_DEPTH times; past that the first direction in the order is used
  and roots are searched on 2q equal sub-intervals;
* a function with no zero on its box (exact min/max test) is dropped;
* every root is found by N_BISECT bisection steps from a strict sign change.

Recursion: to integrate over {phi < 0} in a d-box, pick the height direction
k; the two face restrictions phi(., lo_k) and phi(., hi_k) become the
functions of a (d-1)-dimensional rule on the base box (split at their zero
sets, itself built the same way); above every base node the interval in x_k
is split at the root of phi, Gauss points are placed on the sub-intervals with
phi < 0, and the root itself is a surface node with weight
w' |grad phi| / |d_k phi| and normal grad phi / |grad phi|.
"""

import numpy as np

MAX_DEPTH = 4
N_BISECT = 64


def gauss01(q):
    """Gauss-Legendre nodes and weights on [0, 1] (numpy's leggauss)."""
    x, w = np.polynomial.legendre.leggauss(q)
    return 0.5 * (x + 1.0), 0.5 * w


def bisect(g, a, b, ga):
    """Root of g in [a, b] (arrays) given g(a) = ga with g(a) g(b) < 0.
    N_BISECT halvings; the result is the final midpoint."""
    a = np.array(a, dtype=np.float64)
    b = np.array(b, dtype=np.float64)
    neg_a = np.asarray(ga) < 0
    for _ in range(N_BISECT):
        m = 0.5 * (a + b)
        gm = g(m)
        zero = gm == 0
        same = (gm < 0) == neg_a
        a = np.where(zero | same, m, a)
        b = np.where(zero | ~same, m, b)
    return 0.5 * (a + b)


def _fbox(lo, hi, f):
    blo = lo.copy()
    bhi = hi.copy()
    for dim, v in f.items():
        blo[dim] = v
        bhi[dim] = v
    return blo, bhi


def _changes_sign(ls, lo, hi, f):
    mn, mx = ls.box_minmax(*_fbox(lo, hi, f))
    return mn < 0 < mx


def _monotone(ls, k, lo, hi, funcs):
    return all(ls.grad_sign_const(k, *_fbox(lo, hi, f)) for f in funcs)


def _dir_order(ls, lo, hi, free, f0):
    blo, bhi = _fbox(lo, hi, f0)
    ctr = 0.5 * (blo + bhi)
    g = ls.grad(ctr[None, :])[0]
    return sorted(free, key=lambda k: (-abs(g[k]), k))


def _children(lo, hi, free):
    out = []
    for bits in range(1 << len(free)):
        clo = lo.copy()
        chi = hi.copy()
        for i, k in enumerate(free):
            mid = 0.5 * (lo[k] + hi[k])
            if (bits >> i) & 1:
                clo[k] = mid
            else:
                chi[k] = mid
        out.append((clo, chi))
    return out


def _tensor_gauss(lo, hi, free, q, d):
    x, w = gauss01(q)
    pts = np.zeros((1, d))
    wt = np.ones(1)
    for k in free:
        L = hi[k] - lo[k]
        n = pts.shape[0]
        pts = np.repeat(pts, q, axis=0)
        wt = np.repeat(wt, q) * np.tile(w * L, n)
        pts[:, k] = np.tile(lo[k] + L * x, n)
    return pts, wt


def _eval_line(ls, f, P, k, t):
    X = P.copy()
    for dim, v in f.items():
        X[:, dim] = v
    X[:, k] = t
    return ls.phi(X)


def _line_roots(ls, f, P, k, a, b, monotone, q):
    """Roots in (a, b) of t -> phi_f(P, t) for every row of P.  Returns a list
    of arrays (one per candidate bracket) with NaN where there is none."""
    n = P.shape[0]
    if monotone:
        edges = [a, b]
    else:
        edges = list(a + (b - a) * np.arange(2 * q + 1) / (2 * q))
        edges[-1] = b
    out = []
    for s in range(len(edges) - 1):
        ta = np.full(n, edges[s])
        tb = np.full(n, edges[s + 1])
        ga = _eval_line(ls, f, P, k, ta)
        gb = _eval_line(ls, f, P, k, tb)
        br = ((ga < 0) & (gb > 0)) | ((ga > 0) & (gb < 0))
        r = np.full(n, np.nan)
        if br.any():
            g = lambda t, idx=np.nonzero(br)[0]: _eval_line(ls, f, P[idx], k, t)
            r[br] = bisect(g, ta[br], tb[br], ga[br])
        out.append(r)
    return out


def _pieces(a, b, roots):
    """Sub-intervals of [a, b] cut at the given roots (NaNs ignored)."""
    rs = sorted(float(r) for r in roots if not np.isnan(r))
    pts = [a] + rs + [b]
    return [(pts[i], pts[i + 1]) for i in range(len(pts) - 1)]


def base_rule(ls, lo, hi, free, funcs, q, depth):
    """Rule on the box restricted to the free directions (all other coordinates
    are fixed by every function in funcs), split at the zero sets of funcs so
    that a smooth integrand in between is integrated to Gauss accuracy.
    Returns points (n, d) (non-free coordinates unused) and weights (n,)."""
    d = ls.d
    kept = [f for f in funcs if _changes_sign(ls, lo, hi, f)]
    if not kept:
        return _tensor_gauss(lo, hi, free, q, d)
    order = _dir_order(ls, lo, hi, free, kept[0])
    k = next((j for j in order if _monotone(ls, j, lo, hi, kept)), None)
    monotone = k is not None
    if not monotone:
        if depth < MAX_DEPTH:
            parts = [base_rule(ls, clo, chi, free, kept, q, depth + 1)
                     for clo, chi in _children(lo, hi, free)]
            return (np.concatenate([p[0] for p in parts]),
                    np.concatenate([p[1] for p in parts]))
        k = order[0]
    sub = [j for j in free if j != k]
    if sub:
        sub_funcs = []
        for f in kept:
            sub_funcs.append({**f, k: lo[k]})
            sub_funcs.append({**f, k: hi[k]})
        bp, bw = base_rule(ls, lo, hi, sub, sub_funcs, q, depth)
    else:
        bp, bw = np.zeros((1, d)), np.ones(1)
    roots = []
    for f in kept:
        roots.extend(_line_roots(ls, f, bp, k, lo[k], hi[k], monotone, q))
    x, w = gauss01(q)
    P_out, W_out = [], []
    for i in range(bp.shape[0]):
        for (ta, tb) in _pieces(lo[k], hi[k], [r[i] for r in roots]):
            L = tb - ta
            P = np.repeat(bp[i:i + 1], q, axis=0)
            P[:, k] = ta + L * x
            P_out.append(P)
            W_out.append(bw[i] * L * w)
    return np.concatenate(P_out), np.concatenate(W_out)


def cut_cell_rule(ls, lo, hi, q, depth=0):
    """Volume rule on {phi < 0} within the box [lo, hi] and surface rule on
    {phi = 0} within it.

    Returns (vp, vw, sp, sw, sn): volume points/weights, surface points,
    weights and unit normals (grad phi / |grad phi|, pointing out of Omega)."""
    d = ls.d
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    empty = (np.zeros((0, d)), np.zeros(0), np.zeros((0, d)), np.zeros(0), np.zeros((0, d)))
    mn, mx = ls.box_minmax(lo, hi)
    if mn >= 0:
        return empty
    if mx <= 0:
        vp, vw = _tensor_gauss(lo, hi, list(range(d)), q, d)
        return vp, vw, empty[2], empty[3], empty[4]
    free = list(range(d))
    order = _dir_order(ls, lo, hi, free, {})
    k = next((j for j in order if _monotone(ls, j, lo, hi, [{}])), None)
    monotone = k is not None
    if not monotone:
        if depth < MAX_DEPTH:
            parts = [cut_cell_rule(ls, clo, chi, q, depth + 1)
                     for clo, chi in _children(lo, hi, free)]
            return tuple(np.concatenate([p[i] for p in parts]) for i in range(5))
        k = order[0]
    sub = [j for j in free if j != k]
    bp, bw = base_rule(ls, lo, hi, sub, [{k: lo[k]}, {k: hi[k]}], q, depth)
    roots = _line_roots(ls, {}, bp, k, lo[k], hi[k], monotone, q)
    x, w = gauss01(q)
    VP, VW, SP, SW = [], [], [], []
    for i in range(bp.shape[0]):
        ri = [r[i] for r in roots]
        for (ta, tb) in _pieces(lo[k], hi[k], ri):
            pm = bp[i].copy()
            pm[k] = 0.5 * (ta + tb)
            if ls.phi(pm[None, :])[0] < 0:
                L = tb - ta
                P = np.repeat(bp[i:i + 1], q, axis=0)
                P[:, k] = ta + L * x
                VP.append(P)
                VW.append(bw[i] * L * w)
        for r in ri:
            if np.isnan(r):
                continue
            ps = bp[i].copy()
            ps[k] = r
            SP.append(ps[None, :])
            SW.append(np.array([bw[i]]))
    vp = np.concatenate(VP) if VP else empty[0]
    vw = np.concatenate(VW) if VW else empty[1]
    if SP:
        sp = np.concatenate(SP)
        g = ls.grad(sp)
        gn = np.sqrt((g * g).sum(axis=1))
        sw = np.concatenate(SW) * gn / np.abs(g[:, k])
        sn = g / gn[:, None]
    else:
        sp, sw, sn = empty[2], empty[3], empty[4]
    return vp, vw, sp, sw, sn
