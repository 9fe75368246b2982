"""Conformal maps onto slit domains by the FBIE route (Sec. 7, Ex. 3 and Ex. 4):
gamma = -Re[e^{i(pi/2 - theta)} log(eta - alpha)], one solve of Eq. (ie), h of
Eq. (h) and A f = gamma + h + i mu;
bounded G:   A = e^{i(pi/2 - theta)} (eta - alpha), w = e^{-h_0} (z - alpha) exp((z - alpha) f(z));
unbounded G: A = e^{i(pi/2 - theta)} (Eq. A), f(inf) = 0, w = (z - alpha) exp(f(z)).

CPU pins of the oracle (independent of its formulas):
  * unit disk: w is the Moebius map (z - alpha)/(1 - conj(alpha) z), on the
    boundary and inside (Cauchy formula), with exponential convergence, and
    w'(alpha) = c = 1/(1 - |alpha|^2);
  * Ex. 2's symmetric five-circle domain, alpha = 0: |w| = 1 on the outer circle,
    |w| constant on every circular-slit boundary and the four radii equal (the
    domain's quarter-turn symmetry); with theta = (pi/2, 0, pi/2, 0, pi/2),
    arg w constant on the radial-slit boundaries;
  * w(alpha) = 0, |w| < 1 inside, and w winds once around 0 along the outer circle;
  * planted mistakes (the sign of gamma, the rotation in A) fail the pins.
Unbounded G (Ex. 4):
  * exterior of the unit circle, alpha outside it: the closed form
    w = -conj(alpha) z (z - alpha)/(1 - conj(alpha) z) (|w| = |alpha| on the
    circle, w(alpha) = 0, w(z) = z + O(1)), i.e. f = -log(1 - 1/(conj(alpha) z)),
    h_0 = log|alpha|, on the boundary and inside, with exponential convergence;
  * a manufactured solution with non-constant theta: gamma = Re[A f],
    mu = Im[A f], h = 0 for an f with poles in the holes and f(inf) = 0;
  * Ex. 4's five circles, alpha = 2.5 on the real axis: |w| constant on every
    circular-slit boundary, the radii of mirror-image circles equal (the
    domain's symmetry under conjugation); with theta = (pi/2, 0, pi/2, 0, pi/2),
    arg w constant on the radial-slit boundaries; w(alpha) = 0 with winding
    number 1 around alpha; w(z)/(z - alpha) -> 1 like 1/|z| at infinity;
  * planted mistakes (the factor (eta - alpha) of the bounded A, the sign of
    gamma) fail these pins.
GPU: gnk_slit_map_data / gnk_slit_map / gnk_slit_map_eval against the oracle,
bounded and unbounded.
"""
import math

import numpy as np
import pytest

from oracle import gnk_dense as O
from paper_1308_5351_gb300 import domains as Dm

HALF = math.pi / 2


def _disk(n, a):
    return Dm.build_domain([Dm.Circle(0j, 1.0, ccw=True)], n, bounded=True, alpha=a)


def test_disk_is_the_moebius_map():
    a = 0.3 + 0.2j
    z = np.array([0.1 + 0.1j, -0.4 + 0.2j, 0.55 - 0.3j])
    errs = []
    for n in (16, 32, 64):
        d = _disk(n, a)
        w, c, hk, wz = O.slit_map(d.et, d.etp, n, a, [HALF], z=z)
        errs.append(max(np.abs(w - (d.et - a) / (1 - np.conj(a) * d.et)).max(),
                        np.abs(wz - (z - a) / (1 - np.conj(a) * z)).max()))
        assert abs(c - 1 / (1 - abs(a) ** 2)) < 1e-12 or n < 64
    assert errs[-1] < 1e-13 and errs[1] < errs[0] / 1e3


def _slit_properties(w, n, m1, theta):
    W = w.reshape(m1, n)
    out = {}
    for k in range(m1):
        if theta[k] == HALF:
            out[k] = ("circ", np.abs(W[k]).mean(), np.ptp(np.abs(W[k])))
        else:
            ang = np.unwrap(np.angle(W[k]))
            out[k] = ("rad", ang.mean(), np.ptp(ang))
    return out


def test_ex2_circular_slits_and_symmetry():
    d = Dm.ex2_circles(0.1, 128)
    th = [HALF] * 5
    w, c, hk, _ = O.slit_map(d.et, d.etp, d.n, 0j, th)
    p = _slit_properties(w, d.n, d.m1, th)
    assert abs(p[0][1] - 1.0) < 1e-12 and p[0][2] < 1e-12
    radii = [p[k][1] for k in range(1, 5)]
    assert max(p[k][2] for k in range(1, 5)) < 1e-9
    assert max(radii) - min(radii) < 1e-12 and max(radii) < 1.0


def test_ex2_radial_slits():
    d = Dm.ex2_circles(0.1, 128)
    th = [HALF, 0.0, HALF, 0.0, HALF]
    w, c, hk, _ = O.slit_map(d.et, d.etp, d.n, 0j, th)
    p = _slit_properties(w, d.n, d.m1, th)
    assert abs(p[0][1] - 1.0) < 1e-12
    assert p[1][2] < 1e-9 and p[3][2] < 1e-9           # arg w constant on the radial slits
    assert p[2][2] < 1e-9 and p[4][2] < 1e-9           # |w| constant on the circular slits
    # the quarter-turn maps radial boundary 1 onto 3 (and circular 2 onto 4)
    assert abs(abs(p[1][1] - p[3][1]) - math.pi) < 1e-9 and abs(p[2][1] - p[4][1]) < 1e-12


def test_interior_and_winding():
    d = Dm.three_circles(128)
    a = 0.05j
    rng = np.random.default_rng(0)
    pts = []
    while len(pts) < 50:
        z = complex(rng.uniform(-0.9, 0.9), rng.uniform(-0.9, 0.9))
        if abs(z) < 0.9 and abs(z - 0.45) > 0.25 and abs(z + 0.45) > 0.25:
            pts.append(z)
    z = np.array(pts + [a])
    w, c, hk, wz = O.slit_map(d.et, d.etp, d.n, a, [HALF] * 3, z=z)
    assert abs(wz[-1]) < 1e-13                          # w(alpha) = 0
    assert np.abs(wz[:-1]).max() < 1.0
    outer = np.unwrap(np.angle(w[:d.n]))
    closing = np.angle(w[0] / w[d.n - 1])
    assert abs((outer[-1] - outer[0] + closing) / (2 * math.pi) - 1.0) < 1e-9


def _pins_pass():
    try:
        test_disk_is_the_moebius_map()
        test_ex2_radial_slits()
    except AssertionError:
        return False
    return True


def test_planted_mistakes_are_caught(monkeypatch):
    orig = O.slit_map_data
    assert _pins_pass()

    def wrong_sign(et, n, alpha, theta, bounded=True):
        A, g = orig(et, n, alpha, theta, bounded)
        return A, -g

    def no_rotation(et, n, alpha, theta, bounded=True):
        _, g = orig(et, n, alpha, theta, bounded)
        return np.asarray(et) - alpha, g

    for fn in (wrong_sign, no_rotation):
        monkeypatch.setattr(O, "slit_map_data", fn)
        assert not _pins_pass(), fn.__name__
        monkeypatch.undo()


# ------------------------------------------------------------------ unbounded G (Ex. 4)
def _exterior_disk(n):
    return Dm.build_domain([Dm.Circle(0j, 1.0, ccw=False)], n, bounded=False)


def test_exterior_disk_closed_form():
    a = 1.7 + 0.9j
    z = np.array([2.0 + 0.5j, -1.5 - 1.2j, 0.3 + 1.4j, 5.0 - 7.0j])

    def phi(x):
        return -np.conj(a) * x * (x - a) / (1 - np.conj(a) * x)
    errs = []
    for n in (32, 64, 128):
        d = _exterior_disk(n)
        w, c, hk, wz = O.slit_map(d.et, d.etp, n, a, [HALF], z=z, bounded=False)
        errs.append(max(np.abs(w - phi(d.et)).max(), np.abs(wz - phi(z)).max(),
                        abs(hk[0] - math.log(abs(a)))))
        assert c == 1.0
    assert errs[-1] < 1e-12 and errs[1] < errs[0] / 1e2


def test_unbounded_manufactured_nonconstant_theta():
    d = Dm.ex4_circles(0.3, 256, theta=[HALF, 0.0, HALF, 0.0, HALF])
    f = Dm.f_poles([cv.centre for cv in d.curves], [1.0, 0.3 - 0.2j, -0.5j, 0.7, 0.2 + 0.4j])
    gam, mu_ex = Dm.manufactured(d, f)
    mu, h, hk = O.fbie(d.et, d.etp, d.A, d.n, gam)
    assert np.abs(mu - mu_ex).max() < 1e-12 and np.abs(h).max() < 1e-12


A_EX4 = 2.5 + 0.0j


def _ex4_pts(d, count, seed=0, box=3.0):
    rng = np.random.default_rng(seed)
    pts = []
    while len(pts) < count:
        z = complex(rng.uniform(-box, box), rng.uniform(-box, box))
        if all(abs(z - cv.centre) > cv.radius + 0.05 for cv in d.curves) and abs(z - A_EX4) > 0.05:
            pts.append(z)
    return np.array(pts)


def test_ex4_circular_slits_and_conjugation_symmetry():
    d = Dm.ex4_circles(0.1, 256)
    th = [HALF] * 5
    w, c, hk, _ = O.slit_map(d.et, d.etp, d.n, A_EX4, th, bounded=False)
    p = _slit_properties(w, d.n, d.m1, th)
    assert max(p[k][2] for k in range(5)) < 1e-9
    # circles (1, 1) <-> (1, -1) and (-1, 1) <-> (-1, -1) are mirror images
    assert abs(hk[1] - hk[4]) < 1e-11 and abs(hk[2] - hk[3]) < 1e-11
    assert np.allclose([p[k][1] for k in range(5)], np.exp(hk), rtol=1e-11, atol=0)


def test_ex4_radial_slits():
    d = Dm.ex4_circles(0.1, 256)
    th = [HALF, 0.0, HALF, 0.0, HALF]
    w, c, hk, _ = O.slit_map(d.et, d.etp, d.n, A_EX4, th, bounded=False)
    p = _slit_properties(w, d.n, d.m1, th)
    assert p[1][2] < 1e-9 and p[3][2] < 1e-9           # arg w constant on the radial slits
    assert p[0][2] < 1e-9 and p[2][2] < 1e-9 and p[4][2] < 1e-9


def test_ex4_interior_zero_and_infinity():
    d = Dm.ex4_circles(0.1, 256)
    th = [HALF] * 5
    # w(alpha) = 0, winding number 1 of w around 0 along a small circle about alpha
    ring = A_EX4 + 0.2 * np.exp(2j * math.pi * np.arange(64) / 64)
    far = np.array([10.0 + 0j, 100.0 + 0j, 1000.0 + 0j])
    z = np.concatenate([[A_EX4], ring, far])
    w, c, hk, wz = O.slit_map(d.et, d.etp, d.n, A_EX4, th, z=z, bounded=False)
    assert abs(wz[0]) < 1e-12
    arg = np.unwrap(np.angle(wz[1:65]))
    turns = (arg[-1] - arg[0] + np.angle(wz[1] / wz[64])) / (2 * math.pi)
    assert abs(turns - 1.0) < 1e-9
    dev = np.abs(wz[65:] / (far - A_EX4) - 1.0)  # |e^{f(z)} - 1| ~ C/|z|
    assert dev[1] < dev[0] / 5 and dev[2] < dev[1] / 5


def _unbounded_pins_pass():
    try:
        test_exterior_disk_closed_form()
        test_ex4_radial_slits()
    except AssertionError:
        return False
    return True


def test_unbounded_planted_mistakes_are_caught(monkeypatch):
    orig = O.slit_map_data
    assert _unbounded_pins_pass()

    def bounded_A(et, n, alpha, theta, bounded=True):
        A, g = orig(et, n, alpha, theta, True)
        return A, g

    def wrong_sign(et, n, alpha, theta, bounded=True):
        A, g = orig(et, n, alpha, theta, bounded)
        return A, -g

    for fn in (bounded_A, wrong_sign):
        monkeypatch.setattr(O, "slit_map_data", fn)
        assert not _unbounded_pins_pass(), fn.__name__
        monkeypatch.undo()


# ------------------------------------------------------------------ GPU
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def G():
    from paper_1308_5351_gb300 import build, gnk
    build.build()
    gnk.load()
    return gnk


CASES = {
    "three_circles_circular": (lambda: Dm.three_circles(256), 0.05j, [HALF] * 3),
    "ex2_mixed": (lambda: Dm.ex2_circles(0.1, 128), 0j, [HALF, 0.0, HALF, 0.0, HALF]),
    "disk": (lambda: _disk(64, 0.3 + 0.2j), 0.3 + 0.2j, [HALF]),
    "ex4_circular": (lambda: Dm.ex4_circles(0.1, 256), A_EX4, [HALF] * 5),
    "ex4_mixed": (lambda: Dm.ex4_circles(0.1, 256), A_EX4, [HALF, 0.0, HALF, 0.0, HALF]),
    "exterior_disk": (lambda: _exterior_disk(64), 1.7 + 0.9j, [HALF]),
}


def _interior_points(d, a):
    if not d.bounded:
        return _ex4_pts(d, 40, seed=4)
    rng = np.random.default_rng(4)
    pts = []
    while len(pts) < 40:
        z = complex(rng.uniform(-0.9, 0.9), rng.uniform(-0.9, 0.9))
        if abs(z) < 0.9 and all(abs(z - cv.centre) > cv.radius + 0.05 for cv in d.curves[1:]):
            pts.append(z)
    return np.array(pts)


@pytest.mark.gpu
@pytest.mark.parametrize("case", list(CASES))
def test_gpu_slit_map_data(G, case):
    mk, a, th = CASES[case]
    d = mk()
    A_ref, g_ref = O.slit_map_data(d.et, d.n, a, th, d.bounded)
    et = torch.as_tensor(d.et, device="cuda")
    A = torch.empty_like(et)
    g = torch.empty(d.N, dtype=torch.float64, device="cuda")
    G.gnk_slit_map_data(d.m1, d.n, et, a, torch.as_tensor(np.asarray(th), device="cuda"), A, g,
                        bounded=d.bounded)
    assert np.abs(A.cpu().numpy() - A_ref).max() <= 1e-15 * np.abs(A_ref).max() * 4
    assert np.abs(g.cpu().numpy() - g_ref).max() <= 1e-13 * max(1.0, np.abs(g_ref).max())


@pytest.mark.gpu
@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", ["fmm", "fp64"])
def test_gpu_slit_map_matches_oracle(G, case, prec):
    """w at the nodes and at interior points within 1e-9 of max(1, |w|): mu and h
    agree with the oracle to 1e-10 relative (solve tolerance 1e-12, condition
    numbers below 100), |mu|, |h| <= 10 here, and w = c (z - alpha) exp(...)
    carries those errors through the exponent."""
    mk, a, th = CASES[case]
    d = mk()
    z = _interior_points(d, a)
    w_ref, c_ref, hk_ref, wz_ref = O.slit_map(d.et, d.etp, d.n, a, th, z=z, bounded=d.bounded)
    p = G.GNK_PREC_FMM if prec == "fmm" else G.GNK_PREC_FP64
    w, hk, wz, res = G.slit_map(d, a, th, z=z, precision=p)
    assert res.status == 0
    sw = max(1.0, np.abs(w_ref).max())
    assert np.abs(w.cpu().numpy() - w_ref).max() <= 1e-9 * sw
    assert np.all(np.abs(wz.cpu().numpy() - wz_ref) <= 1e-9 * np.maximum(1.0, np.abs(wz_ref)))
    assert np.abs(hk.cpu().numpy() - hk_ref).max() <= 1e-10 * max(1.0, np.abs(hk_ref).max())


@pytest.mark.gpu
def test_gpu_slit_map_rejects_bad_arguments(G):
    d = Dm.ex4_circles(0.1, 64)
    with G.Boundary.from_domain(d, adjoint=False, device="cuda") as b:
        z = torch.zeros(4, dtype=torch.complex128, device="cuda")
        x = torch.zeros(d.N, dtype=torch.float64, device="cuda")
        hk = torch.zeros(d.m1, dtype=torch.float64, device="cuda")
        with pytest.raises(G.GnkError):
            G.gnk_slit_map_eval(b.handle, 0j, x, x, x, hk, z, z, precision=G.GNK_PREC_FP32)
