"""Slit maps by the route of the adjoint equation (Sec. 7, Ex. 3 and Ex. 4, the
paper's FBIEad comparison): solves of Eq. (ie*) only, with
A of Eq. (A), A~ = eta'/A (Eq. A*),
  derivative solve:  bounded G   (I + N* + J) psi = e_0,
                     unbounded G (I + N* + J) psi = 2 Im[A~/(eta - alpha)],
  parameter solves:  (I + N* + J) psi_j = e_j, j = 0..m,
psi = th' on a circular-slit boundary and -(log rho)' on a radial one, S its
antiderivative along each boundary (FFT), and the per-boundary constants from
T_j = (1/2pi) int c omega^ psi_j.

CPU pins of the oracle (independent of its formulas):
  * the periodic antiderivative is exact on trigonometric polynomials and
    ignores the n/2 mode at the nodes;
  * unit disk: w is the Moebius map (z - alpha)/(1 - conj(alpha) z), psi its
    boundary-correspondence derivative (1 - |alpha|^2)/|e^{it} - alpha|^2 and
    w'(alpha) = 1/(1 - |alpha|^2), with exponential convergence;
  * exterior of the unit circle (unbounded): w = -conj(alpha) z (z - alpha)/
    (1 - conj(alpha) z), R_0 = |alpha|, psi = Im[eta' w'/w];
  * exterior of a circle onto the plane minus one radial slit (theta = 0): a
    Moebius map composed with Joukowski's, for both routes;
  * Ex. 2 (bounded) and Ex. 4 (unbounded) five circles with constant and mixed
    theta: the same map as the FBIE route (another equation, another solve):
    w on the boundary and inside, w'(alpha) = e^{-h_0}, R_k = e^{h_k - h_0}
    (bounded) or e^{h_k} (unbounded), phi_k = -h_k;
  * the parameter solutions lie in the null space of I + N* (J psi_j = e_j), and
    the derivative solution has the winding numbers of the map;
  * the boundary values are those of a function analytic in G (the exterior
    Cauchy integral vanishes in every hole) with w(alpha) = 0;
  * on a graded square hole (corners) the two routes converge to each other
    like n^-2;
  * planted mistakes (the sign of the antiderivative, c of Eq. (c), the
    rotation of A) fail these pins.
GPU: gnk_slit_map_adjoint / gnk_slit_map_adjoint_eval against the oracle.
"""
import math

import numpy as np
import pytest

from oracle import gnk_dense as O
from paper_1308_5351_gb300 import domains as Dm

HALF = math.pi / 2
MIXED = [HALF, 0.0, HALF, 0.0, HALF]


def test_antiderivative_is_exact_on_trig_polynomials():
    n = 32
    t = np.arange(n) * (2 * math.pi / n)
    p0 = 1.0 + np.cos(3 * t) - 2.0 * np.sin(5 * t) + 0.7 * np.cos(n / 2 * t)
    s0 = t + np.sin(3 * t) / 3 + 2.0 * (np.cos(5 * t) - 1.0) / 5
    p1 = 0.25 * np.sin(t) - 4.0 * np.cos(15 * t)
    s1 = 0.25 * (1.0 - np.cos(t)) - 4.0 * np.sin(15 * t) / 15
    S = O.periodic_antiderivative(np.concatenate([p0, p1]), n)
    assert np.abs(S - np.concatenate([s0, s1])).max() < 5e-14  # |S| up to 2 pi


def test_disk_is_the_moebius_map():
    a = 0.3 + 0.2j
    z = np.array([0.1 + 0.1j, -0.4 + 0.2j, 0.55 - 0.3j])
    errs = []
    for n in (16, 32, 64):
        d = Dm.disk(n, a)
        w, psi, params, scale, omega, wz = O.slit_map_adjoint(d.et, d.etp, d.etpp, n, a, [HALF], z=z)
        t = Dm.nodes(n)
        dth = (1 - abs(a) ** 2) / np.abs(np.exp(1j * t) - a) ** 2
        errs.append(max(np.abs(w - (d.et - a) / (1 - np.conj(a) * d.et)).max(),
                        np.abs(wz - (z - a) / (1 - np.conj(a) * z)).max(),
                        np.abs(psi - dth).max(), abs(scale - 1 / (1 - abs(a) ** 2))))
        assert params[0] == 1.0
    assert errs[-1] < 1e-13 and errs[1] < errs[0] / 1e3


def test_exterior_of_the_unit_circle():
    a = 2.0 + 0.5j
    z = np.array([1.5 + 1.5j, -3.0 + 0.1j])
    errs = []
    for n in (16, 32, 64, 128):
        d = Dm.build_domain([Dm.Circle(0j, 1.0)], n, bounded=False)
        w, psi, params, scale, omega, wz = O.slit_map_adjoint(d.et, d.etp, d.etpp, n, a, [HALF],
                                                              bounded=False, z=z)
        ca = np.conj(a)
        ex = lambda x: -ca * x * (x - a) / (1 - ca * x)
        e = d.et
        dpsi = (d.etp * (1 / e + 1 / (e - a) + ca / (1 - ca * e))).imag
        errs.append(max(np.abs(w - ex(e)).max(), np.abs(wz - ex(z)).max(), np.abs(psi - dpsi).max(),
                        abs(params[0] - abs(a))))
        assert scale == 1.0
    # psi is exact at the nodes here; w converges with the interpolant of psi
    assert errs[-1] < 1e-13 and errs[2] < errs[1] / 1e4 and errs[1] < errs[0] / 1e2


def _radial_exterior_closed_form(c, r, a):
    """Exterior of the circle |z - c| = r onto the plane minus one radial slit,
    w(a) = 0, w = z + O(1): with zeta = (z - c)/r and beta = (a - c)/r, the
    Moebius map u = e^{i arg beta} (1 - conj(beta) zeta)/(zeta - beta) keeps the
    exterior of the unit circle, sends a to infinity and infinity to
    u_inf = -|beta| (real); Joukowski J(u) = u + 1/u maps it onto the plane
    minus [-2, 2], and g = J(u) - J(u_inf) moves the segment along the real
    axis away from 0 with g(inf) = 0, g(a) = inf; w = lambda/g with lambda the
    limit of z g(z)."""
    beta = (a - c) / r
    e = np.exp(1j * np.angle(beta))
    uinf = -abs(beta)
    lam = (1 - 1 / uinf ** 2) * e * (1 - abs(beta) ** 2) * r

    def w(z):
        zeta = (z - c) / r
        u = e * (1 - np.conj(beta) * zeta) / (zeta - beta)
        return lam / (u + 1 / u - (uinf + 1 / uinf))
    return w


def test_exterior_radial_slit_closed_form():
    """theta = 0 on the one boundary of an unbounded domain: both routes against
    the closed form, with exponential convergence; arg w is constant on the
    boundary and w(z)/z -> 1 at infinity."""
    c, r, a = 0.2j, 0.8, 1.5 + 0.7j
    ex = _radial_exterior_closed_form(c, r, a)
    z = np.array([3 + 1j, -2 - 2j, 0.5 - 1.5j])
    assert abs(ex(np.array([1e7 * np.exp(0.3j)]))[0] / (1e7 * np.exp(0.3j)) - 1) < 1e-6
    errs = []
    for n in (32, 64, 128):
        d = Dm.build_domain([Dm.Circle(c, r)], n, bounded=False, theta=[0.0])
        w, psi, params, scale, omega, wz = O.slit_map_adjoint(d.et, d.etp, d.etpp, n, a, [0.0], False, z=z)
        w2, c2, hk, wz2 = O.slit_map(d.et, d.etp, n, a, [0.0], z=z, bounded=False)
        errs.append(max(np.abs(w - ex(d.et)).max(), np.abs(wz - ex(z)).max(),
                        np.abs(w2 - ex(d.et)).max(), np.abs(wz2 - ex(z)).max(),
                        abs(math.remainder(params[0] - np.angle(ex(d.et[:1]))[0], 2 * math.pi))))
    assert errs[-1] < 1e-13 and errs[1] < errs[0] / 1e4, errs


_ROUTE_CASES = {
    "ex2_circular": (lambda n: Dm.ex2_circles(0.1, n), 0j, [HALF] * 5, True),
    "ex2_mixed": (lambda n: Dm.ex2_circles(0.1, n), 0j, MIXED, True),
    "ex4_circular": (lambda n: Dm.ex4_circles(0.1, n), 2.5 + 0j, [HALF] * 5, False),
    "ex4_mixed": (lambda n: Dm.ex4_circles(0.1, n), 2.5 + 0j, MIXED, False),
}
_ZIN = {True: np.array([0.05 + 0.02j, 0.3j, -0.6 + 0.1j]),
        False: np.array([2.5 + 1.0j, -3.0 + 0.2j, 0.1 + 5.0j])}


@pytest.mark.parametrize("case", sorted(_ROUTE_CASES))
def test_same_map_as_the_fbie_route(case):
    mk, a, th, bounded = _ROUTE_CASES[case]
    n = 256
    d = mk(n)
    z = _ZIN[bounded]
    w, psi, params, scale, omega, wz = O.slit_map_adjoint(d.et, d.etp, d.etpp, n, a, th, bounded, z=z)
    w2, c2, hk, wz2 = O.slit_map(d.et, d.etp, n, a, th, z=z, bounded=bounded)
    tol = 1e-9 if case == "ex4_mixed" else 1e-11
    assert np.abs(w - w2).max() < tol
    assert np.abs(wz - wz2).max() < tol
    assert abs(scale - c2) < tol
    h0 = hk[0] if bounded else 0.0
    for k in range(d.m1):
        if th[k] == HALF:
            assert abs(params[k] - math.exp(hk[k] - h0)) < tol
        else:
            assert abs(math.remainder(params[k] + hk[k], 2 * math.pi)) < tol


@pytest.mark.parametrize("bounded", [True, False])
def test_null_space_and_winding(bounded):
    """J psi_j = e_j for the parameter solutions (so (I + N*) psi_j = 0), and the
    derivative solution has mean 1 on the outer boundary of bounded G (the
    boundary winds once around 0) and mean 0 on every slit."""
    n = 128
    d = Dm.ex2_circles(0.1, n) if bounded else Dm.ex4_circles(0.1, n)
    a = 0j if bounded else 2.5 + 0j
    A, _ = O.slit_map_data(d.et, n, a, MIXED, bounded)
    rot = np.repeat(np.exp(1j * (HALF - np.asarray(MIXED))), n)
    Ap = rot * d.etp if bounded else np.zeros_like(d.et)
    Mad = O.matrix_adjoint(d.et, d.etp, d.etpp, A, Ap, n, 1 if bounded else -1)
    comp = np.repeat(np.arange(d.m1), n)
    for j in range(d.m1):
        pj = np.linalg.solve(Mad, (comp == j).astype(float))
        assert np.abs(pj.reshape(d.m1, n).mean(axis=1) - np.eye(d.m1)[j]).max() < 1e-12
    _, psi, _, _, _, _ = O.slit_map_adjoint(d.et, d.etp, d.etpp, n, a, MIXED, bounded)
    means = psi.reshape(d.m1, n).mean(axis=1)
    assert np.abs(means - (np.eye(d.m1)[0] if bounded else 0.0)).max() < 1e-12


@pytest.mark.parametrize("bounded", [True, False])
def test_boundary_values_are_analytic_in_G(bounded):
    n = 512  # gaps of 0.01: 256 nodes leave 1e-8 in the unbounded case
    d = Dm.ex2_circles(0.01, n) if bounded else Dm.ex4_circles(0.01, n)
    a = 0.02 + 0.01j if bounded else 2.5 + 0.3j
    w, psi, params, scale, omega, _ = O.slit_map_adjoint(d.et, d.etp, d.etpp, n, a, MIXED, bounded)
    hole_pts = [cv.centre for cv in d.curves[1 if bounded else 0:]]
    # (1/2 pi i) int f eta' / (eta - z) dt with f analytic in G: 0 in every hole
    f = w if bounded else omega
    for zc in hole_pts:
        v = np.sum(f * d.etp / (d.et - zc)) / (1j * n)
        assert abs(v) < 1e-12 * np.abs(f).max()
    if bounded:
        assert abs(np.sum(w * d.etp / (d.et - a)) / (1j * n)) < 1e-10  # w(alpha) = 0
    # circular slits keep |w| fixed, radial slits arg w fixed
    W = w.reshape(d.m1, n)
    for k, th in enumerate(MIXED):
        if th == HALF:
            assert np.ptp(np.abs(W[k])) < 1e-13 * np.abs(W[k]).max()
        else:
            assert np.ptp(np.unwrap(np.angle(W[k]))) < 1e-13


def test_graded_square_hole_converges_to_the_fbie_route():
    """A square hole with graded corners (p = 3, Sec. 6): psi has a kink at
    each corner (|t - c|^(2p/3 - 1)), so both routes converge algebraically;
    their difference must fall like n^-2 and be below 1e-4 at n = 512."""
    a = -0.3 + 0.5j
    th = [HALF, 0.0, HALF]
    diffs = []
    for n in (128, 256, 512):
        curves = [Dm.Circle(0j, 1.0, ccw=True), Dm.square(0.3 + 0.1j, 0.25, ccw=False),
                  Dm.Circle(-0.4 - 0.2j, 0.2)]
        d = Dm.build_domain(curves, n, bounded=True, alpha=a)
        w = O.slit_map_adjoint(d.et, d.etp, d.etpp, n, a, th, True)[0]
        w2 = O.slit_map(d.et, d.etp, n, a, th)[0]
        diffs.append(np.abs(w - w2).max())
    assert diffs[1] < diffs[0] / 3 and diffs[2] < diffs[1] / 3 and diffs[2] < 1e-4, diffs


def test_planted_mistakes_fail(monkeypatch):
    a = 0.3 + 0.2j
    n = 64
    d = Dm.disk(n, a)
    ref = (d.et - a) / (1 - np.conj(a) * d.et)

    def err():
        w = O.slit_map_adjoint(d.et, d.etp, d.etpp, n, a, [HALF])[0]
        return np.abs(w - ref).max()

    assert err() < 1e-12
    good = O.periodic_antiderivative
    monkeypatch.setattr(O, "periodic_antiderivative", lambda p, n_: -good(p, n_))
    assert err() > 1e-3
    monkeypatch.setattr(O, "periodic_antiderivative", good)
    good_mat = O.matrix_adjoint
    monkeypatch.setattr(O, "matrix_adjoint", lambda et, etp, etpp, A, Ap, n_, c: good_mat(et, etp, etpp, A, Ap, n_, -c))
    assert err() > 1e-3
    monkeypatch.setattr(O, "matrix_adjoint", good_mat)
    # the rotation of A on the radial boundaries (theta ignored)
    d5 = Dm.ex2_circles(0.1, 128)
    w2 = O.slit_map(d5.et, d5.etp, 128, 0j, MIXED)[0]
    good_data = O.slit_map_data
    monkeypatch.setattr(O, "slit_map_data", lambda et, n_, al, th, b=True: good_data(et, n_, al, [HALF] * 5, b))
    w = O.slit_map_adjoint(d5.et, d5.etp, d5.etpp, 128, 0j, MIXED)[0]
    assert np.abs(w - w2).max() > 1e-3


# ---------------------------------------------------------------------------
# GPU: the C-ABI route against the oracle
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def G():
    pytest.importorskip("torch")
    from paper_1308_5351_gb300 import build, gnk
    build.build()
    gnk.load()
    return gnk


_GPU_CASES = {
    "disk": (lambda: Dm.disk(64, 0.3 + 0.2j), 0.3 + 0.2j, [HALF]),
    "ex2_circular": (lambda: Dm.ex2_circles(0.1, 256), 0j, [HALF] * 5),
    "ex2_mixed": (lambda: Dm.ex2_circles(0.1, 256), 0j, MIXED),
    "ex4_circular": (lambda: Dm.ex4_circles(0.1, 256), 2.5 + 0j, [HALF] * 5),
    "ex4_mixed": (lambda: Dm.ex4_circles(0.1, 256), 2.5 + 0j, MIXED),
    # n not a power of two (the direct antiderivative) and an odd number of boundaries
    "three_circles_n100": (lambda: Dm.three_circles(100), 0.05j, [HALF, 0.0, HALF]),
}


def _points_in(d, count=24, seed=7):
    """Points of G at least 0.05 away from every boundary circle."""
    rng = np.random.default_rng(seed)
    pts = []
    while len(pts) < count:
        if d.bounded:
            z = complex(rng.uniform(-0.95, 0.95), rng.uniform(-0.95, 0.95))
            ok = abs(z) < d.curves[0].radius - 0.05 and all(
                abs(z - cv.centre) > cv.radius + 0.05 for cv in d.curves[1:])
        else:
            z = complex(rng.uniform(-4, 4), rng.uniform(-4, 4))
            ok = all(abs(z - cv.centre) > cv.radius + 0.05 for cv in d.curves)
        if ok:
            pts.append(z)
    return np.array(pts)


@pytest.mark.gpu
@pytest.mark.parametrize("case", sorted(_GPU_CASES))
def test_gpu_slit_map_adjoint_data(G, case):
    import torch
    mk, a, th = _GPU_CASES[case]
    d = mk()
    rot = np.repeat(np.exp(1j * (HALF - np.asarray(th))), d.n)
    ref = rot * d.etp if d.bounded else np.zeros_like(d.etp)
    Ap = torch.empty(d.N, dtype=torch.complex128, device="cuda")
    G.gnk_slit_map_adjoint_data(d.m1, d.n, torch.as_tensor(d.etp, device="cuda"),
                                torch.as_tensor(np.asarray(th, dtype=np.float64), device="cuda"), Ap,
                                bounded=d.bounded)
    assert np.abs(Ap.cpu().numpy() - ref).max() <= 4e-16 * max(1.0, np.abs(ref).max())


@pytest.mark.gpu
@pytest.mark.parametrize("case", sorted(_GPU_CASES))
@pytest.mark.parametrize("prec", ["fp64", "fmm"])
def test_gpu_slit_map_adjoint_matches_oracle(G, case, prec):
    """w, omega and psi at the nodes, the parameters and w inside G within 1e-9
    of max(1, |.|): every solve to 1e-12 (condition numbers below 100 here), and
    the constants are sums of omega^ psi_j that carry those errors into the
    exponent."""
    mk, a, th = _GPU_CASES[case]
    d = mk()
    z = _points_in(d)
    w_r, psi_r, par_r, sc_r, om_r, wz_r = O.slit_map_adjoint(d.et, d.etp, d.etpp, d.n, a, th, d.bounded, z=z)
    p = G.GNK_PREC_FMM if prec == "fmm" else G.GNK_PREC_FP64
    w, psi, params, omega, wz, res = G.slit_map_adjoint(d, a, th, z=z, precision=p, restart=40, maxit=20)
    assert res.status == 0 and res.relres <= 1e-12, (res.status, res.relres)
    solves = d.m1 if d.bounded else d.m1 + 1
    assert res.cycles >= solves
    sw = max(1.0, np.abs(w_r).max())
    assert np.abs(w.cpu().numpy() - w_r).max() <= 1e-9 * sw
    assert np.abs(omega.cpu().numpy() - om_r).max() <= 1e-9 * max(1.0, np.abs(om_r).max())
    assert np.abs(psi.cpu().numpy() - psi_r).max() <= 1e-9 * max(1.0, np.abs(psi_r).max())
    par = params.cpu().numpy()
    assert np.abs(par[:-1] - par_r).max() <= 1e-9 * max(1.0, np.abs(par_r).max())
    assert abs(par[-1] - sc_r) <= 1e-9 * sc_r
    assert np.all(np.abs(wz.cpu().numpy() - wz_r) <= 1e-9 * np.maximum(1.0, np.abs(wz_r)))


@pytest.mark.gpu
def test_gpu_slit_map_adjoint_large_n_disk():
    """n = 8192 (beyond the shared-memory FFT: the direct antiderivative) on the
    unit disk against the closed form w = (z - alpha)/(1 - conj(alpha) z), which
    holds at any size."""
    from paper_1308_5351_gb300 import build, gnk as G
    build.build()
    G.load()
    a = 0.3 + 0.2j
    d = Dm.disk(8192, a)
    w, psi, params, omega, wz, res = G.slit_map_adjoint(d, a, [HALF], precision=G.GNK_PREC_FP64)
    assert res.status == 0
    ref = (d.et - a) / (1 - np.conj(a) * d.et)
    assert np.abs(w.cpu().numpy() - ref).max() <= 1e-11
    t = Dm.nodes(8192)
    assert np.abs(psi.cpu().numpy() - (1 - abs(a) ** 2) / np.abs(np.exp(1j * t) - a) ** 2).max() <= 1e-10
    assert abs(params.cpu().numpy()[-1] - 1 / (1 - abs(a) ** 2)) <= 1e-11


@pytest.mark.gpu
def test_gpu_slit_map_adjoint_rejects_bad_arguments(G):
    import torch
    d = Dm.ex2_circles(0.1, 64)
    et = torch.as_tensor(d.et, device="cuda")
    w = torch.empty_like(et)
    with G.Boundary.from_domain(d, adjoint=False, device="cuda") as b:  # no eta''
        with pytest.raises(G.GnkError):
            G.gnk_slit_map_adjoint(b.handle, 0j, np.full(5, HALF), w)
    A, _ = O.slit_map_data(d.et, d.n, 0j, MIXED, True)
    rot = np.repeat(np.exp(1j * (HALF - np.asarray(MIXED))), d.n)
    with G.Boundary(d.m1, d.n, d.et, d.etp, A, d.etpp, rot * d.etp, True) as b:
        for th in ([HALF, 0.3, HALF, 0.0, HALF], [0.0, 0.0, HALF, 0.0, HALF]):
            with pytest.raises(G.GnkError) as e:
                G.gnk_slit_map_adjoint(b.handle, 0j, np.asarray(th), w)
            assert e.value.code == G.GNK_EINVAL
        with pytest.raises(G.GnkError):
            G.gnk_slit_map_adjoint_eval(b.handle, 0j, w, w[:4], w[:4], precision=G.GNK_PREC_FP32)
