"""Cauchy integral formula with singularity subtraction (Sec. 5, Eqs. cauchy4,
cauchy6): values of an analytic function at points of G from its boundary
values.

CPU pins: for f analytic in G the oracle's ratio formula reproduces f(z) at
interior points (closed form), including points close to the boundary, where
the plain trapezoidal rule of Eq. (cauchy) fails; exponential convergence in n.
GPU: gnk_cauchy_eval against the oracle (FP64 and double-float), relative
1e-11 of |f(z)| for points whose distance to Gamma exceeds a node spacing."""
import math

import numpy as np
import pytest

from oracle import gnk_dense as O
from paper_1308_5351_gb300 import domains as Dm


def _interior_points_three_circles(rng, count):
    pts = []
    while len(pts) < count:
        z = complex(rng.uniform(-0.95, 0.95), rng.uniform(-0.95, 0.95))
        if abs(z) < 0.97 and abs(z - 0.45) > 0.23 and abs(z + 0.45) > 0.23:
            pts.append(z)
    return np.array(pts)


def test_formula_reproduces_analytic_function_bounded():
    rng = np.random.default_rng(0)
    z = _interior_points_three_circles(rng, 40)
    errs = []
    for n in (32, 64, 128):
        d = Dm.three_circles(n)
        fz = O.cauchy_formula(d.et, d.etp, n, Dm.f_bounded_ex1(d.et), z, True)
        errs.append(np.abs(fz - Dm.f_bounded_ex1(z)).max())
    assert errs[-1] < 1e-10 and errs[1] < errs[0] / 10


def test_formula_unbounded_ex4():
    d = Dm.ex4_circles(0.1, 256)
    rng = np.random.default_rng(1)
    z = []
    while len(z) < 30:
        c = complex(rng.uniform(-2.5, 2.5), rng.uniform(-2.5, 2.5))
        if all(abs(c - cv.centre) > cv.radius + 0.05 for cv in d.curves):
            z.append(c)
    z = np.array(z)
    f = Dm.f_unbounded_ex1
    fz = O.cauchy_formula(d.et, d.etp, d.n, f(d.et), z, False, finf=0.0)
    assert np.abs(fz - f(z)).max() < 1e-9


def test_formula_unbounded_constant_at_infinity():
    """f = c + poles inside the holes: f(inf) = c enters through f_inf only;
    dropping it (f_inf = 0) shifts every value."""
    d = Dm.ex4_circles(0.1, 256)
    rng = np.random.default_rng(5)
    cst = 0.7 - 1.3j
    fp = Dm.f_poles([cv.centre for cv in d.curves], [0.3 + 0.1j] * len(d.curves))

    def f(x):
        return cst + fp(x)
    z = []
    while len(z) < 20:
        c = complex(rng.uniform(-2.5, 2.5), rng.uniform(-2.5, 2.5))
        if all(abs(c - cv.centre) > cv.radius + 0.05 for cv in d.curves):
            z.append(c)
    z = np.array(z)
    good = O.cauchy_formula(d.et, d.etp, d.n, f(d.et), z, False, cst)
    bad = O.cauchy_formula(d.et, d.etp, d.n, f(d.et), z, False, 0.0)
    assert np.abs(good - f(z)).max() < 1e-9 and np.abs(bad - f(z)).min() > 1e-3


def test_ratio_form_beats_plain_rule_near_boundary():
    """Points at distance 1e-3 from the outer circle: the subtracted form stays
    accurate while the plain trapezoidal rule of Eq. (cauchy) does not."""
    d = Dm.three_circles(128)
    th = np.linspace(0.1, 2.0, 7)
    z = (1 - 1e-3) * np.exp(1j * th)
    f = Dm.f_bounded_ex1
    fz = O.cauchy_formula(d.et, d.etp, d.n, f(d.et), z, True)
    plain = np.array([(2 * math.pi / d.n) / (2j * math.pi) * np.sum(f(d.et) * d.etp / (d.et - zk)) for zk in z])
    assert np.abs(fz - f(z)).max() < 1e-6 < np.abs(plain - f(z)).max()


# ------------------------------------------------------------------ GPU
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def G():
    from paper_1308_5351_gb300 import build, gnk
    build.build()
    gnk.load()
    return gnk


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [0, 3])
@pytest.mark.parametrize("case", ["bounded", "unbounded"])
def test_cauchy_eval_matches_oracle(G, prec, case):
    rng = np.random.default_rng(7)
    if case == "bounded":
        d = Dm.three_circles(256)
        z = _interior_points_three_circles(rng, 1000)
        f = Dm.f_bounded_ex1
        finf = None
    else:
        d = Dm.ex4_circles(0.1, 256)
        z = []
        while len(z) < 777:
            c = complex(rng.uniform(-2.5, 2.5), rng.uniform(-2.5, 2.5))
            if all(abs(c - cv.centre) > cv.radius + 0.02 for cv in d.curves):
                z.append(c)
        z = np.array(z)
        f = Dm.f_unbounded_ex1
        finf = 0.0 + 0.0j
    ref = O.cauchy_formula(d.et, d.etp, d.n, f(d.et), z, d.bounded, 0.0 if finf is None else finf)
    with G.Boundary.from_domain(d, adjoint=False, device="cuda") as b:
        fz = b.cauchy_eval(torch.as_tensor(z, device="cuda"), torch.as_tensor(f(d.et), device="cuda"),
                           finf=finf, precision=prec).cpu().numpy()
    assert np.all(np.abs(fz - ref) <= 1e-11 * np.maximum(1.0, np.abs(ref)))
    assert np.abs(fz - f(z)).max() < 1e-8


def _exterior_points(d, rng, count, box, margin):
    """Points of the unbounded G (outside every ellipse) at distance > margin
    from all boundary nodes."""
    out = []
    while len(out) < count:
        c = rng.uniform(-box, box, size=4 * count) + 1j * rng.uniform(-box, box, size=4 * count)
        keep = np.ones(c.size, dtype=bool)
        for cv in d.curves:
            w = np.exp(-1j * cv.phi) * (c - cv.centre)
            keep &= (w.real / cv.a) ** 2 + (w.imag / cv.b) ** 2 > 1.0
        c = c[keep]
        far = np.ones(c.size, dtype=bool)
        for k in range(0, c.size, 32):
            far[k:k + 32] = np.abs(c[k:k + 32, None] - d.et[None, :]).min(axis=1) > margin
        out.extend(c[far].tolist())
    return np.array(out[:count])


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [0, 3])
def test_cauchy_eval_fullsize_ellipses(G, prec):
    """64 ellipses, N = 65,536 nodes (the headline boundary), 4099 exterior
    points (ragged against every tile size): f = c + sum of poles inside the
    ellipses, so f(inf) = c != 0.  Sampled points against the oracle, all
    points against the closed form."""
    d = Dm.ellipses64()
    rng = np.random.default_rng(11)
    z = _exterior_points(d, rng, 4099, 4.6, 0.03)
    cst = 0.7 - 1.3j
    poles = [cv.centre for cv in d.curves]
    fp = Dm.f_poles(poles, rng.uniform(-0.2, 0.2, len(poles)) + 1j * rng.uniform(-0.2, 0.2, len(poles)))

    def f(x):
        return cst + fp(x)
    with G.Boundary.from_domain(d, adjoint=False, device="cuda") as b:
        fz = b.cauchy_eval(torch.as_tensor(z, device="cuda"), torch.as_tensor(f(d.et), device="cuda"),
                           finf=cst, precision=prec).cpu().numpy()
    idx = rng.choice(z.size, 64, replace=False)
    ref = O.cauchy_formula(d.et, d.etp, d.n, f(d.et), z[idx], False, cst)
    assert np.all(np.abs(fz[idx] - ref) <= 1e-11 * np.maximum(1.0, np.abs(ref)))
    assert np.abs(fz - f(z)).max() < 1e-8


@pytest.mark.gpu
def test_cauchy_eval_edge_cases(G):
    """nz = 0, host arrays, one point per tile edge, a point on a node, bad
    precision and negative nz."""
    d = Dm.three_circles(64)
    f = Dm.f_bounded_ex1
    with G.Boundary.from_domain(d, adjoint=False, device="cuda") as b:
        empty = b.cauchy_eval(torch.empty(0, dtype=torch.complex128, device="cuda"),
                              torch.as_tensor(f(d.et), device="cuda"))
        assert empty.numel() == 0
        z = np.array([0.1 + 0.2j])
        fz = b.cauchy_eval(z, f(d.et))          # host arrays, one point
        assert isinstance(fz, np.ndarray) and abs(fz[0] - f(z)[0]) < 1e-10
        z2 = np.array([0.0 + 0.0j, d.et[5], -0.2 + 0.1j])
        fz2 = b.cauchy_eval(z2, f(d.et))
        assert not np.isfinite(fz2[1]) and np.abs(fz2[[0, 2]] - f(z2[[0, 2]])).max() < 1e-10
        with pytest.raises(G.GnkError):
            b.cauchy_eval(z, f(d.et), precision=G.GNK_PREC_FP32)
        with pytest.raises(G.GnkError):
            G.gnk_cauchy_eval(b.handle, z, f(d.et), np.empty(1, np.complex128), precision=7)
