"""Pins of the oracle's general level sets (ellipsoid, torus, flower): the
interval bounds enclose sampled values and gradients, and the cut-cell
quadrature over them reproduces closed-form volumes and areas."""

import math

import numpy as np
import pytest

from oracle.levelset import Ellipsoid, Flower, Sphere, Torus
from oracle.quadrature import cut_cell_rule


def rot(a, b, c):
    ca, sa, cb, sb, cc, sc = math.cos(a), math.sin(a), math.cos(b), math.sin(b), math.cos(c), math.sin(c)
    Rz = np.array([[ca, -sa, 0], [sa, ca, 0], [0, 0, 1]])
    Ry = np.array([[cb, 0, sb], [0, 1, 0], [-sb, 0, cb]])
    Rx = np.array([[1, 0, 0], [0, cc, -sc], [0, sc, cc]])
    return Rz @ Ry @ Rx


SHAPES = {
    "ellipsoid": lambda: Ellipsoid([0.03, -0.02, 0.01], [0.7, 0.5, 0.4], rot(0.3, 0.5, 0.2)),
    "torus": lambda: Torus([0.02, 0.01, -0.03], rot(0.4, 0.7, 0.1), 0.6, 0.2),
    "flower": lambda: Flower([0.02, -0.03], 5, 0.4),
}


@pytest.mark.parametrize("name", list(SHAPES))
def test_bounds_enclose_samples(name):
    ls = SHAPES[name]()
    d = ls.d
    rng = np.random.default_rng(3)
    for _ in range(300):
        lo = rng.uniform(-1, 0.9, d)
        hi = lo + rng.uniform(0.01, 0.3, d)
        X = lo + (hi - lo) * rng.uniform(0, 1, (400, d))
        mn, mx = ls.box_minmax(lo, hi)
        v = ls.phi(X)
        assert v.min() >= mn - 1e-12 and v.max() <= mx + 1e-12
        g = ls.grad(X)
        for k in range(d):
            if ls.grad_sign_const(k, lo, hi):
                assert (g[:, k] > 0).all() or (g[:, k] < 0).all()


@pytest.mark.parametrize("name", list(SHAPES))
def test_gradient_matches_finite_differences(name):
    ls = SHAPES[name]()
    rng = np.random.default_rng(4)
    X = rng.uniform(-0.9, 0.9, (50, ls.d))
    g = ls.grad(X)
    for k in range(ls.d):
        e = np.zeros(ls.d)
        e[k] = 1e-6
        fd = (ls.phi(X + e) - ls.phi(X - e)) / 2e-6
        assert np.abs(fd - g[:, k]).max() < 1e-6


def _totals(ls, N):
    d = ls.d
    h = 2.0 / N
    vol = 0.0
    area = 0.0
    for flat in range(N ** d):
        c = [(flat // N ** k) % N for k in range(d)]
        lo = -1.0 + h * np.array(c, dtype=float)
        mn, mx = ls.box_minmax(lo, lo + h)
        if mn >= 0:
            continue
        if mx <= 0:
            vol += h ** d
            continue
        _, vw, _, sw, _ = cut_cell_rule(ls, lo, lo + h, 4)
        vol += vw.sum()
        area += sw.sum()
    return vol, area


def test_flower_area_and_perimeter():
    ls = SHAPES["flower"]()
    vol, per = _totals(ls, 64)
    assert vol == pytest.approx(math.pi * (0.6 ** 2 + 0.1 ** 2 / 2), rel=1e-7)
    th = np.linspace(0, 2 * math.pi, 200001)
    r = 0.6 + 0.1 * np.cos(5 * th)
    dr = -0.5 * np.sin(5 * th)
    ref = np.trapezoid(np.sqrt(r * r + dr * dr), th)
    assert per == pytest.approx(ref, rel=1e-6)


def test_ellipsoid_volume():
    ls = SHAPES["ellipsoid"]()
    vol, _ = _totals(ls, 16)
    assert vol == pytest.approx(4.0 / 3.0 * math.pi * 0.7 * 0.5 * 0.4, rel=2e-6)


def test_torus_volume_and_area():
    ls = SHAPES["torus"]()
    vol, area = _totals(ls, 16)
    assert vol == pytest.approx(2 * math.pi ** 2 * 0.6 * 0.2 ** 2, rel=1e-5)
    assert area == pytest.approx(4 * math.pi ** 2 * 0.6 * 0.2, rel=1e-4)


def test_sphere_bounds_are_exact():
    ls = Sphere([0.1, 0.2, -0.1], 0.5)
    mn, mx = ls.box_minmax(np.array([0.0, 0.0, 0.0]), np.array([0.2, 0.3, 0.1]))
    assert mn == pytest.approx(0.1 - 0.5)
    assert mx == pytest.approx(math.sqrt(0.1 ** 2 + 0.2 ** 2 + 0.2 ** 2) - 0.5)


# ---------------------------------------------------------------------------
# level sets known only through point callbacks (sampled bounds)

from callback_shapes import distance_sphere, superellipse  # noqa: E402
from oracle.levelset import make_levelset  # noqa: E402


def test_sampled_bounds_enclose_a_distance_function_exactly():
    """For a distance function the sampled gradient norm (1) bounds |grad phi|
    everywhere, so the widened sample range must contain the exact range of
    the sphere, on full boxes and on degenerate (face and edge) boxes."""
    for c in ([0.1, -0.05], [0.1, -0.05, 0.02]):
        d = len(c)
        cb = make_levelset(distance_sphere(c, 0.6))
        ex = Sphere(c, 0.6)
        rng = np.random.default_rng(11 + d)
        for i in range(300):
            lo = rng.uniform(-1, 0.9, d)
            hi = lo + rng.uniform(0.01, 0.3, d)
            if i % 3 == 1:
                hi[i % d] = lo[i % d]
            mn, mx = cb.box_minmax(lo, hi)
            emn, emx = ex.box_minmax(lo, hi)
            assert mn <= emn + 1e-15 and mx >= emx - 1e-15
            # and no wider than the lattice spacing allows
            delta = 0.5 * np.linalg.norm((hi - lo) / 4)
            assert mn >= emn - 2 * delta - 1e-15 and mx <= emx + 2 * delta + 1e-15


def test_sampled_bounds_and_monotonicity_hold_on_dense_samples():
    ls = make_levelset(superellipse([0.03, -0.02], [0.7, 0.55]))
    rng = np.random.default_rng(12)
    mono = 0
    for _ in range(300):
        lo = rng.uniform(-0.95, 0.8, 2)
        hi = lo + rng.uniform(0.02, 0.15, 2)
        X = lo + (hi - lo) * rng.uniform(0, 1, (400, 2))
        mn, mx = ls.box_minmax(lo, hi)
        v = ls.phi(X)
        assert v.min() >= mn - 1e-12 and v.max() <= mx + 1e-12
        g = ls.grad(X)
        for k in range(2):
            if ls.grad_sign_const(k, lo, hi):
                mono += 1
                assert (g[:, k] > 0).all() or (g[:, k] < 0).all()
    assert mono > 200  # the test is not vacuous


def test_callback_quadrature_reproduces_closed_form_measures():
    disk = make_levelset(distance_sphere([0.031, 0.017], 0.7))
    vol, per = _totals(disk, 32)
    assert vol == pytest.approx(math.pi * 0.49, rel=1e-8)
    assert per == pytest.approx(2 * math.pi * 0.7, rel=1e-7)
    g = math.gamma
    se = make_levelset(superellipse([0.03, -0.02], [0.7, 0.55]))
    vol, _ = _totals(se, 64)
    assert vol == pytest.approx(4 * 0.7 * 0.55 * g(1.25) ** 2 / g(1.5), rel=1e-6)
    se3 = make_levelset(superellipse([0.03, -0.02, 0.01], [0.7, 0.55, 0.6]))
    vol, _ = _totals(se3, 8)
    assert vol == pytest.approx(8 * 0.7 * 0.55 * 0.6 * g(1.25) ** 3 / g(1.75), rel=1e-4)


def test_callback_classification_contains_the_exact_one():
    """Cells the exact sphere calls active (cut) are active (cut) for the same
    sphere given as callbacks: the sampled bounds only widen."""
    from oracle.fem import Level
    lev_ex = Level(Sphere([0.031, 0.017], 0.7), 2, 32, 2)
    lev_cb = Level(make_levelset(distance_sphere([0.031, 0.017], 0.7)), 2, 32, 2)
    assert np.all(lev_cb.active[lev_ex.active])
    assert np.all(lev_cb.cut[lev_ex.cut])
    # the extra ones lie within the widening (2 delta) of the interface
    ex = Sphere([0.031, 0.017], 0.7)
    delta = 0.5 * math.sqrt(2.0) * lev_ex.h / 4
    extra = np.nonzero((lev_cb.cut & ~lev_ex.cut) | (lev_cb.active & ~lev_ex.active))[0]
    assert extra.size > 0
    for c in extra:
        emn, emx = ex.box_minmax(lev_ex.cell_lo[c], lev_ex.cell_lo[c] + lev_ex.h)
        assert (0 <= emn <= 2 * delta) or (-2 * delta <= emx <= 0)
