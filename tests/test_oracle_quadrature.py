"""Pins of the oracle's cut-cell quadrature (Sec. 3: substitute quadrature on
cut cells by dimension reduction) against closed forms.

A dropped sub-interval, a wrong surface weight |grad phi|/|d_k phi|, a wrong
normal or a missed root each break one of these."""

import math

import numpy as np
import pytest

from oracle.levelset import Plane, Sphere
from oracle.quadrature import cut_cell_rule, gauss01


def plane_volume_unit(n, a):
    """Volume of {xi in [0,1]^d : n.xi < a} for n > 0 (inclusion-exclusion
    over the cube's vertices)."""
    d = len(n)
    s = 0.0
    for v in range(1 << d):
        bits = [(v >> k) & 1 for k in range(d)]
        t = a - sum(n[k] * bits[k] for k in range(d))
        s += (-1) ** sum(bits) * max(0.0, t) ** d
    return s / (math.factorial(d) * np.prod(n))


def plane_dvolume_unit(n, a):
    d = len(n)
    s = 0.0
    for v in range(1 << d):
        bits = [(v >> k) & 1 for k in range(d)]
        t = a - sum(n[k] * bits[k] for k in range(d))
        s += (-1) ** sum(bits) * max(0.0, t) ** (d - 1)
    return s / (math.factorial(d - 1) * np.prod(n))


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("a", [0.37, 0.9, 1.31])
def test_plane_cut_volume_and_area_exact(d, a):
    n = np.array([0.6, 0.8, 0.45][:d])
    lo = np.array([0.25, -0.5, 0.125][:d])
    h = 0.5
    ls = Plane(n, n @ lo + h * a)
    vp, vw, sp, sw, sn = cut_cell_rule(ls, lo, lo + h, 4)
    assert vw.sum() == pytest.approx(h ** d * plane_volume_unit(n, a), rel=1e-13)
    # area of the plane piece: |n| dV/da, with V(a) the physical volume
    assert sw.sum() == pytest.approx(np.linalg.norm(n) * h ** (d - 1) * plane_dvolume_unit(n, a), rel=1e-13)
    assert np.allclose(sn, n / np.linalg.norm(n))
    assert np.all(ls.phi(vp) < 0)
    assert np.allclose(ls.phi(sp), 0, atol=1e-15)


def test_plane_cut_polynomial_exact_2d():
    """Volume moments of a polygon (square clipped by a line) against Green's
    theorem on its edges, which is exact for polynomials with enough Gauss
    points per edge."""
    lo = np.array([0.0, 0.0])
    n = np.array([1.0, 0.7])
    a = 1.05
    ls = Plane(n, a)
    vp, vw, _, _, _ = cut_cell_rule(ls, lo, lo + 1.0, 4)
    # polygon vertices (counter-clockwise): clip unit square with x + 0.7 y < a
    poly = [(0, 0), (1, 0), (1, (a - 1) / 0.7), (a - 0.7, 1), (0, 1)]
    x, w = gauss01(8)
    for (pa, pb) in [(2, 0), (1, 3), (3, 1), (2, 2)]:
        # int x^pa y^pb dA = oint x^(pa+1)/(pa+1) y^pb dy
        ref = 0.0
        for i in range(len(poly)):
            x0, y0 = poly[i]
            x1, y1 = poly[(i + 1) % len(poly)]
            X = x0 + (x1 - x0) * x
            Y = y0 + (y1 - y0) * x
            ref += np.sum(w * X ** (pa + 1) / (pa + 1) * Y ** pb) * (y1 - y0)
        got = np.sum(vw * vp[:, 0] ** pa * vp[:, 1] ** pb)
        assert got == pytest.approx(ref, rel=1e-13, abs=1e-15)


def _sphere_totals(ls, d, N, q=4):
    h = 2.0 / N
    V = 0.0
    rules = []
    for flat in range(N ** d):
        c = [(flat // N ** k) % N for k in range(d)]
        lo = -1.0 + h * np.array(c, dtype=float)
        mn, mx = ls.box_minmax(lo, lo + h)
        if mn >= 0:
            continue
        if mx <= 0:
            V += h ** d
            rules.append((lo, None))
            continue
        rules.append((lo, cut_cell_rule(ls, lo, lo + h, q)))
    return V, rules, h


def test_disk_area_perimeter_moments():
    c = np.array([0.031, 0.017])
    r = 0.7
    ls = Sphere(c, r)
    V_unc, rules, h = _sphere_totals(ls, 2, 32)
    xg, wg = gauss01(3)
    vol = V_unc
    per = 0.0
    m2 = 0.0
    surf_xn = 0.0
    for lo, rule in rules:
        if rule is None:
            X, Y = np.meshgrid(lo[0] + h * xg, lo[1] + h * xg, indexing="ij")
            W = np.outer(wg, wg) * h * h
            m2 += np.sum(W * ((X - c[0]) ** 2 + (Y - c[1]) ** 2))
            continue
        vp, vw, sp, sw, sn = rule
        vol += vw.sum()
        per += sw.sum()
        m2 += np.sum(vw * ((vp - c) ** 2).sum(axis=1))
        surf_xn += np.sum(sw * ((sp - c) * sn).sum(axis=1))
    assert vol == pytest.approx(math.pi * r * r, rel=1e-11)
    assert per == pytest.approx(2 * math.pi * r, rel=1e-10)
    assert m2 == pytest.approx(math.pi * r ** 4 / 2, rel=1e-10)
    assert surf_xn == pytest.approx(r * 2 * math.pi * r, rel=1e-10)


def test_ball_volume_area_and_divergence_theorem():
    c = np.array([0.05, 0.03, 0.02])
    r = 0.7
    ls = Sphere(c, r)
    V_unc, rules, h = _sphere_totals(ls, 3, 16)
    xg, wg = gauss01(4)
    vol = V_unc
    area = 0.0
    div_vol = 0.0
    flux = 0.0
    # F = (x^3, x y^2, z^2 y): div F = 3x^2 + 2xy + 2zy
    F = lambda X: np.stack([X[:, 0] ** 3, X[:, 0] * X[:, 1] ** 2, X[:, 2] ** 2 * X[:, 1]], axis=1)
    divF = lambda X: 3 * X[:, 0] ** 2 + 2 * X[:, 0] * X[:, 1] + 2 * X[:, 2] * X[:, 1]
    G = np.array(np.meshgrid(xg, xg, xg, indexing="ij")).reshape(3, -1).T
    WG = np.einsum("i,j,k->ijk", wg, wg, wg).ravel()
    for lo, rule in rules:
        if rule is None:
            X = lo + h * G
            div_vol += np.sum(WG * divF(X)) * h ** 3
            continue
        vp, vw, sp, sw, sn = rule
        vol += vw.sum()
        area += sw.sum()
        div_vol += np.sum(vw * divF(vp))
        flux += np.sum(sw * (F(sp) * sn).sum(axis=1))
    assert vol == pytest.approx(4 / 3 * math.pi * r ** 3, rel=2e-9)
    assert area == pytest.approx(4 * math.pi * r ** 2, rel=1e-8)
    assert div_vol == pytest.approx(flux, rel=1e-8)


def test_quadrature_converges_under_refinement():
    """Geometric error of the disk area falls by far more than h^2 per
    refinement (high order in h)."""
    ls = Sphere([0.031, 0.017], 0.7)
    errs = []
    for N in (4, 8, 16):
        V_unc, rules, h = _sphere_totals(ls, 2, N)
        vol = V_unc + sum(rule[1].sum() for _, rule in rules if rule is not None)
        errs.append(abs(vol - math.pi * 0.49))
    assert errs[1] < errs[0] / 16 and errs[2] < errs[1] / 16
