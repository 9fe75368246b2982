"""Conformal maps onto the unit disk with circular and radial slits by the FBIE
route (Sec. 7, Ex. 3): A = e^{i(pi/2 - theta)} (eta - alpha),
gamma = -Re[e^{i(pi/2 - theta)} log(eta - alpha)], one solve of Eq. (ie), h of
Eq. (h), w = e^{-h_0} (z - alpha) exp((z - alpha) f(z)) with A f = gamma + h + i mu.

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
GPU: gnk_slit_map_data / gnk_slit_map / gnk_slit_map_eval against the oracle.
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

    def wrong_sign(et, n, alpha, theta):
        A, g = orig(et, n, alpha, theta)
        return A, -g

    def no_rotation(et, n, alpha, theta):
        _, g = orig(et, n, alpha, theta)
        return np.asarray(et) - alpha, g

    for fn in (wrong_sign, no_rotation):
        monkeypatch.setattr(O, "slit_map_data", fn)
        assert not _pins_pass(), fn.__name__
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
}


@pytest.mark.gpu
@pytest.mark.parametrize("case", list(CASES))
def test_gpu_slit_map_data(G, case):
    mk, a, th = CASES[case]
    d = mk()
    A_ref, g_ref = O.slit_map_data(d.et, d.n, a, th)
    et = torch.as_tensor(d.et, device="cuda")
    A = torch.empty_like(et)
    g = torch.empty(d.N, dtype=torch.float64, device="cuda")
    G.gnk_slit_map_data(d.m1, d.n, et, a, torch.as_tensor(np.asarray(th), device="cuda"), A, g)
    assert np.abs(A.cpu().numpy() - A_ref).max() <= 1e-15 * np.abs(A_ref).max() * 4
    assert np.abs(g.cpu().numpy() - g_ref).max() <= 1e-13 * max(1.0, np.abs(g_ref).max())


@pytest.mark.gpu
@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", ["fmm", "fp64"])
def test_gpu_slit_map_matches_oracle(G, case, prec):
    """w at the nodes and at interior points within 1e-9: mu and h agree with the
    oracle to 1e-10 relative (solve tolerance 1e-12, condition numbers below
    100), |mu|, |h| <= 10 here, and w = c (z - alpha) exp(...) with |w| <= 1
    carries those errors through the exponent."""
    mk, a, th = CASES[case]
    d = mk()
    rng = np.random.default_rng(4)
    pts = []
    while len(pts) < 40:
        z = complex(rng.uniform(-0.9, 0.9), rng.uniform(-0.9, 0.9))
        if abs(z) < 0.9 and all(abs(z - cv.centre) > cv.radius + 0.05 for cv in d.curves[1:]):
            pts.append(z)
    z = np.array(pts)
    w_ref, c_ref, hk_ref, wz_ref = O.slit_map(d.et, d.etp, d.n, a, th, z=z)
    p = G.GNK_PREC_FMM if prec == "fmm" else G.GNK_PREC_FP64
    w, hk, wz, res = G.slit_map(d, a, th, z=z, precision=p)
    assert res.status == 0
    assert np.abs(w.cpu().numpy() - w_ref).max() <= 1e-9
    assert np.abs(wz.cpu().numpy() - wz_ref).max() <= 1e-9
    assert np.abs(hk.cpu().numpy() - hk_ref).max() <= 1e-10 * max(1.0, np.abs(hk_ref).max())


@pytest.mark.gpu
def test_gpu_slit_map_rejects_unbounded(G):
    d = Dm.ex4_circles(0.1, 64)
    with G.Boundary.from_domain(d, adjoint=False, device="cuda") as b:
        x = torch.zeros(d.N, dtype=torch.float64, device="cuda")
        hk = torch.zeros(d.m1, dtype=torch.float64, device="cuda")
        w = torch.empty(d.N, dtype=torch.complex128, device="cuda")
        with pytest.raises(G.GnkError):
            G.gnk_slit_map(b.handle, 0j, x, x, x, hk, w)
