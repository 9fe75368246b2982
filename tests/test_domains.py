"""Input generators: parametrisations, graded mesh (Sec. 6), orientation, and
the workload recipes."""
import math

import numpy as np
import pytest

from paper_1308_5351_gb300 import domains as Dm


def _fd_check(curve, tol=1e-6):
    t = np.linspace(0.1, 6.1, 37)
    h = 1e-5
    z, zp, zpp = curve.eval(t)
    zph = (curve.eval(t + h)[0] - curve.eval(t - h)[0]) / (2 * h)
    zpph = (curve.eval(t + h)[1] - curve.eval(t - h)[1]) / (2 * h)
    scale = max(1.0, np.abs(zp).max())
    assert np.abs(zp - zph).max() < tol * scale
    assert np.abs(zpp - zpph).max() < tol * max(1.0, np.abs(zpp).max())


def test_curve_derivatives_match_finite_differences():
    rng = np.random.default_rng(0)
    _fd_check(Dm.Circle(0.3j, 0.7, ccw=True))
    _fd_check(Dm.Circle(0.3j, 0.7, ccw=False))
    _fd_check(Dm.Ellipse(1 + 1j, 0.4, 0.2, 0.7, ccw=False))
    k = np.arange(1, 9)
    _fd_check(Dm.Star(0j, 0.3, rng.normal(0, 0.05 / k), rng.normal(0, 0.05 / k)), tol=1e-5)
    # away from corners the graded polygon is smooth
    sq = Dm.square(0j, 0.5, ccw=True)
    t = np.array([0.3, 1.2, 2.0, 3.5, 4.4, 5.9])
    h = 1e-6
    z, zp, zpp = sq.eval(t)
    assert np.abs(zp - (sq.eval(t + h)[0] - sq.eval(t - h)[0]) / (2 * h)).max() < 1e-5
    assert np.abs(zpp - (sq.eval(t + h)[1] - sq.eval(t - h)[1]) / (2 * h)).max() < 1e-4


@pytest.mark.parametrize("p", [2, 3, 4])
def test_grading_function_properties(p):
    """omega is a bijection of [0, 2pi], strictly increasing, with omega' = 0 at
    the ends (Eq. omega); delta_j fixes the corners and has delta' = 0 there."""
    u = np.linspace(0, 2 * math.pi, 2001)
    om, dom, ddom = Dm.grading_omega(u, p)
    assert abs(om[0]) < 1e-15 and abs(om[-1] - 2 * math.pi) < 1e-12
    assert np.all(np.diff(om) > 0)
    assert abs(dom[0]) < 1e-14 and abs(dom[-1]) < 1e-12
    # symmetry omega(2pi - u) = 2pi - omega(u)
    assert np.abs(om[::-1] - (2 * math.pi - om)).max() < 1e-12
    h = 1e-6
    uu = np.linspace(0.2, 6.0, 23)
    assert np.abs(Dm.grading_omega(uu, p)[1] - (Dm.grading_omega(uu + h, p)[0] - Dm.grading_omega(uu - h, p)[0]) / (2 * h)).max() < 1e-6
    assert np.abs(Dm.grading_omega(uu, p)[2] - (Dm.grading_omega(uu + h, p)[1] - Dm.grading_omega(uu - h, p)[1]) / (2 * h)).max() < 1e-5
    pj = 4
    ck = np.arange(pj) * 2 * math.pi / pj
    dl, ddl, _ = Dm.grading_delta(ck, pj, p)
    assert np.abs(dl - ck).max() < 1e-14 and np.abs(ddl).max() < 1e-14


def test_graded_polygon_perimeter_and_area():
    """Trapezoidal rule on the graded mesh integrates |eta'| to the perimeter and
    (1/2) Im(conj(eta) eta') to the signed area (Eq. trap-cr)."""
    sq = Dm.square(0.2 + 0.1j, 0.5, ccw=True)
    n = 256
    t = Dm.nodes(n)
    z, zp, _ = sq.eval(t)
    per = (2 * math.pi / n) * np.abs(zp).sum()
    area = (2 * math.pi / n) * 0.5 * np.imag(np.conj(z) * zp).sum()
    assert abs(per - 4.0) < 1e-6 and abs(area - 1.0) < 1e-6


def test_orientation_and_sizes():
    d = Dm.three_circles(64)
    t = Dm.nodes(64)
    areas = [(2 * math.pi / 64) * 0.5 * np.imag(np.conj(d.et[k * 64:(k + 1) * 64]) * d.etp[k * 64:(k + 1) * 64]).sum()
             for k in range(3)]
    assert areas[0] > 0 and areas[1] < 0 and areas[2] < 0  # G on the left
    assert d.N == 192 and d.m1 == 3 and d.c == 1
    assert np.allclose(d.A, d.et - 0.05j)
    du = Dm.ex4_circles(0.01, 32)
    assert du.c == -1 and np.allclose(du.A, 1.0) and np.all(du.Ap == 0)
    with pytest.raises(ValueError):
        Dm.three_circles(63)


def test_example_geometries_as_printed():
    """Ex. 4: gaps are exactly eps; Ex. 2: radius (2 - eps(2+2 sqrt 2))/(2+2 sqrt 2),
    centres +-(2-eps)/(2+2 sqrt 2) (1 +- i)."""
    for eps in (1e-1, 1e-2, 1e-3, 1e-4):
        d = Dm.ex4_circles(eps, 8)
        c0, cs = d.curves[0], d.curves[1:]
        for c in cs:
            assert abs(abs(c.centre - c0.centre) - c.radius - c0.radius - eps) < 1e-14
        d2 = Dm.ex2_circles(eps, 8)
        s = 2 + 2 * math.sqrt(2)
        for c in d2.curves[1:]:
            assert abs(c.radius - (2 - eps * s) / s) < 1e-15
            assert abs(abs(c.centre.real) - (2 - eps) / s) < 1e-15


def test_workload_recipes_small():
    d = Dm.ellipses64(2, 16)
    assert d.m1 == 64 and d.N == 1024 and not d.bounded
    pts = [Dm._polyline(c, 256) for c in d.curves]
    gmin = min(Dm._min_gap(pts[i], pts[j]) for i in range(64) for j in range(i + 1, 64)
               if abs(d.curves[i].centre - d.curves[j].centre) < 1.0)
    assert gmin >= 0.05 - 1e-3
    d3 = Dm.close_curves(3, 8)
    assert d3.m1 == 1024 and sum(isinstance(c, Dm.GradedPolygon) for c in d3.curves) == 32
    d5 = Dm.stars_and_polygons(5, 32)
    assert d5.m1 == 20 and sum(isinstance(c, Dm.GradedPolygon) for c in d5.curves) == 4
    b = Dm.batch_domains(4, count=3)
    assert len(b) == 3 and all(2 <= x.m1 <= 64 for x in b)
