"""Pins for the dense CPU oracle: values fixed by the paper and by mathematics,
independent of the oracle's own formulas.

  P1  unit disk, A = eta - alpha, gamma = log|eta - alpha|:
      mu = arg(1 - conj(alpha) eta), h = -log(1 - |alpha|^2)     (Sec. 1, Eqs. ie, h)
  P2  unit circle, A = eta: (I - N) x = x + mean(x); M cos kt = -sin kt,
      M sin kt = cos kt (discrete conjugation is exact below n/2); the adjoint
      matrix is the identity                                        (Sec. 3.3, 4.2)
  P3  manufactured solutions gamma = Re[A f], mu = Im[A f], h = 0, with
      exponential convergence in n                                (Sec. 7, Ex. 1)
  P4  h is piecewise constant                                        (Eq. h, space S)
  P5  adjoint: (I + N* + J) phi = 1 gives J phi = 1 and int gamma phi = 0 (Ex. 1)
  P6  row sums: int N(s,t) dt = -1 (Eq. NM-const) per component; the Neumann
      kernel integrates to c (Eq. Nk-const)
  P7  independent adaptive quadrature of the continuous operators at a node
  V2  spectrum of L: L = (2/n) d/dt on trigonometric polynomials of degree < n/2
  V7  E is antisymmetric
Planted mistakes (a transposed A ratio, a dropped diag(D1), a flipped L, a
wrong identity factor) are injected into the oracle here to show each pin bites.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import gnk_dense as O
from paper_1308_5351_gb300 import domains as Dm


def _fbie(d, gam):
    return O.fbie(d.et, d.etp, d.A, d.n, gam)


# ---------------------------------------------------------------- P1
@pytest.mark.parametrize("alpha", [0.3 + 0.2j, -0.5j, 0.7])
def test_disk_closed_form(alpha):
    errs = []
    for n in (32, 64, 256):
        d = Dm.disk(n, alpha)
        gam = np.log(np.abs(d.et - alpha))
        mu, h, hk = _fbie(d, gam)
        mu_exact = np.angle(1.0 - np.conj(alpha) * d.et)
        errs.append(max(np.abs(mu - mu_exact).max(),
                        np.abs(h + math.log(1.0 - abs(alpha) ** 2)).max()))
    assert errs[-1] < 1e-13
    # exponential convergence (rate |alpha|^n) until round-off
    assert errs[1] < max(errs[0] * abs(alpha) ** 16, 1e-15)


# ---------------------------------------------------------------- P2
def test_unit_circle_operators():
    n = 32
    d = Dm.disk(n, 0j)
    t = Dm.nodes(n)
    IN = O.matrix_IminusN(d.et, d.etp, d.A, n)
    x = np.random.default_rng(0).normal(size=n)
    assert np.abs(IN @ x - (x + x.mean())).max() < 1e-14
    M = O.matrix_M(d.et, d.etp, d.A, n)
    for k in range(1, n // 2):
        assert np.abs(M @ np.cos(k * t) + np.sin(k * t)).max() < 1e-13
        assert np.abs(M @ np.sin(k * t) - np.cos(k * t)).max() < 1e-13
    Ad = O.matrix_adjoint(d.et, d.etp, d.etpp, d.A, d.Ap, n, 1)
    assert np.abs(Ad - np.eye(n)).max() < 1e-14
    # gamma = cos kt => mu = sin kt, h = 0
    mu, h, _ = _fbie(d, np.cos(3 * t))
    assert np.abs(mu - np.sin(3 * t)).max() < 1e-13 and np.abs(h).max() < 1e-13


def test_wittich_circulant_spectrum():
    """L acts as (2/n) d/dt on trigonometric polynomials of degree < n/2 and
    annihilates constants and the alternating (Nyquist) vector."""
    for n in (8, 64, 256):
        L = O.circulant_L(n)
        t = Dm.nodes(n)
        for k in (1, 2, n // 2 - 1):
            assert np.abs(L @ np.sin(k * t) - (2.0 / n) * k * np.cos(k * t)).max() < 1e-12
            assert np.abs(L @ np.cos(k * t) + (2.0 / n) * k * np.sin(k * t)).max() < 1e-12
        assert np.abs(L @ np.ones(n)).max() < 1e-13
        assert np.abs(L @ np.cos(n // 2 * t)).max() < 1e-12
        # circulant first column b_i = (-1)^(i-1) (1/n) cot((i-1) pi/n), b_1 = 0
        lam = np.fft.fft(L[:, 0])
        kk = np.arange(n)
        expect = 1j * 2.0 * np.where(kk < n // 2, kk, kk - n) / n
        expect[n // 2] = 0.0
        assert np.abs(lam - expect).max() < 1e-12


def test_cauchy_matrix_antisymmetric():
    d = Dm.three_circles(32)
    E = O.cauchy_matrix(d.et)
    assert np.all(np.diag(E) == 0)
    assert np.abs(E + E.T).max() == 0.0
    w = np.random.default_rng(1).normal(size=d.N) + 1j
    rows = [0, 5, d.N - 1]
    assert np.allclose(O.cauchy_rows(d.et, w, rows), (E @ w)[rows], rtol=1e-14, atol=1e-13)


# ---------------------------------------------------------------- P3
def _manufactured_error(d, f):
    gam, mu_ex = Dm.manufactured(d, f)
    mu, h, _ = _fbie(d, gam)
    return np.abs(mu - mu_ex).max(), np.abs(h).max()


def test_manufactured_bounded_three_circles():
    errs = []
    for n in (16, 32, 64, 128):
        e_mu, e_h = _manufactured_error(Dm.three_circles(n), Dm.f_bounded_ex1)
        errs.append(max(e_mu, e_h))
    assert errs[-1] < 1e-12
    # exponential convergence: each doubling gains at least 1.5 decades until round-off
    assert errs[1] < errs[0] / 30 and errs[2] < errs[1] / 30


def test_manufactured_unbounded_ex4_paper_f():
    d = Dm.ex4_circles(0.1, 256)
    e_mu, e_h = _manufactured_error(d, Dm.f_unbounded_ex1)
    assert e_mu < 1e-10 and e_h < 1e-10


def test_manufactured_unbounded_ellipses_poles():
    rng = np.random.default_rng(7)
    curves = Dm.random_ellipses(rng, 6, 1.5)
    d = Dm.build_domain(curves, 128, bounded=False)
    f = Dm.f_poles(d.holes, rng.normal(size=d.m1) + 1j * rng.normal(size=d.m1))
    e_mu, e_h = _manufactured_error(d, f)
    assert e_mu < 1e-9 and e_h < 1e-9


def test_manufactured_nonconstant_theta():
    """Ex. 2 domain with theta = (pi/2, 0, pi/2, 0, pi/2) at moderate eps."""
    d = Dm.ex2_circles(0.1, 256, theta=[math.pi / 2, 0, math.pi / 2, 0, math.pi / 2])
    e_mu, e_h = _manufactured_error(d, Dm.f_bounded_ex1)
    assert e_mu < 1e-9 and e_h < 1e-9


def test_manufactured_graded_square_hole():
    """Piecewise-smooth boundary on the graded mesh (Sec. 6): algebraic but fast
    convergence."""
    errs = []
    for n in (64, 128, 256):
        curves = [Dm.Circle(0j, 1.6, ccw=True), Dm.square(0.3 + 0.1j, 0.5, ccw=False)]
        d = Dm.build_domain(curves, n, bounded=True, alpha=-1.2 + 0.3j)
        e_mu, e_h = _manufactured_error(d, Dm.f_bounded_ex1)
        errs.append(e_mu)
    assert errs[-1] < 1e-5 and errs[2] < errs[0] / 100


# ---------------------------------------------------------------- P4
def test_h_piecewise_constant_config1():
    d = Dm.three_circles(256)
    gam = Dm.gamma_log(d, 0.05j)
    mu, h, hk = _fbie(d, gam)
    spread = np.ptp(h.reshape(d.m1, d.n), axis=1)
    assert spread.max() < 1e-12
    # symmetric holes give equal h on both holes
    assert abs(hk[1] - hk[2]) < 1e-12


def test_piecewise_constant_gamma_gives_mu_zero():
    """gamma in S: f = 0 solves the RH problem, so mu = 0 and h = -gamma."""
    d = Dm.three_circles(128)
    gam = np.repeat([0.3, -1.2, 0.7], d.n)
    mu, h, _ = _fbie(d, gam)
    assert np.abs(mu).max() < 1e-12 and np.abs(h + gam).max() < 1e-12


def test_annulus_closed_form():
    """Annulus 0.5 < |z| < 1 with A = eta - alpha (alpha = 0.75 in G) and
    f(z) = 1/z - 0.4i/(z - 0.1 - 0.05i), analytic in G (both poles in the hole):
    the exact solution is mu = Im[A f], h = 0."""
    d = Dm.annulus(256, 0.5, 0.75)
    f = Dm.f_poles([0.0j, 0.1 + 0.05j], [1.0, -0.4j])
    gam, mu_ex = Dm.manufactured(d, f)
    mu, h, _ = _fbie(d, gam)
    assert np.abs(mu - mu_ex).max() < 1e-11 and np.abs(h).max() < 1e-11


# ---------------------------------------------------------------- P5
@pytest.mark.parametrize("bounded", [True, False])
def test_adjoint_invariants(bounded):
    if bounded:
        d = Dm.three_circles(128)
        f = Dm.f_bounded_ex1
    else:
        d = Dm.ex4_circles(0.1, 128)
        f = Dm.f_unbounded_ex1
    phi = O.solve_adjoint_ie(d.et, d.etp, d.etpp, d.A, d.Ap, d.n, d.c, np.ones(d.N))
    means = phi.reshape(d.m1, d.n).mean(axis=1)
    assert np.abs(means - 1.0).max() < 1e-9  # J phi = 1
    gam, _ = Dm.manufactured(d, f)
    En = abs((2 * math.pi / d.n) * np.sum(gam * phi))
    assert En < 1e-9


# ---------------------------------------------------------------- P6
def test_row_sums_eigen_identities():
    """(2pi/n) sum_{j in J_l} N(t_i, t_j) (with the diagonal N(t,t) when l = k)
    tends to -delta_{kl} (Eq. NM-const, per component); the D analogue tends to
    0 for l != k; the Neumann kernel integrates to c (Eq. Nk-const)."""
    for d in (Dm.three_circles(128), Dm.ex4_circles(0.2, 128)):
        B, D = O.matrices_BD(d.et, d.etp, d.A, d.n)
        Nd = (2 * math.pi / d.n) * O.kernel_N_diag(d.etp, d.etpp, d.A, d.Ap)
        comp = d.component_of_node()
        for l in range(d.m1):
            cols = comp == l
            s = B[:, cols].sum(axis=1) + np.where(comp == l, Nd, 0.0)
            target = np.where(comp == l, -1.0, 0.0)
            assert np.abs(s - target).max() < 1e-9
            off = comp != l
            assert np.abs(D[np.ix_(off, cols)].sum(axis=1)).max() < 1e-9
        ones = np.ones(d.N, dtype=np.complex128)
        Kk = O.nystrom_block(d.et, d.etp, ones, d.n, np.arange(d.N), np.arange(d.N)).imag
        Nkd = (2 * math.pi / d.n) * O.kernel_N_diag(d.etp, d.etpp, ones, np.zeros(d.N))
        assert np.abs(Kk.sum(axis=1) + Nkd - d.c).max() < 1e-9


# ---------------------------------------------------------------- P7
def _quad_component(fun, a, b, points=None):
    re = integrate.quad(lambda t: fun(t).real, a, b, points=points, limit=400,
                        epsabs=1e-13, epsrel=1e-13)[0]
    im = integrate.quad(lambda t: fun(t).imag, a, b, points=points, limit=400,
                        epsabs=1e-13, epsrel=1e-13)[0]
    return re + 1j * im


def test_quadrature_of_continuous_operators():
    """phi(s) = int M(s,t)[gamma(t)-gamma(s)] dt (Eq. ie-phi) and
    int N(s,t)[x(t)-x(s)] dt computed by adaptive quadrature of the continuous
    kernels, against the discrete y and (B - diag(B1)) x at n = 128."""
    n = 128
    d = Dm.three_circles(n)
    alpha = d.alpha
    rot = np.exp(1j * (math.pi / 2 - d.theta))

    def geo(k, t):
        z, zp, _ = d.curves[k].eval(np.atleast_1d(np.asarray(t, dtype=float)))
        return z[0], zp[0]

    def A_of(k, t):
        return rot[k] * (geo(k, t)[0] - alpha)

    def gamma_of(k, t):
        return math.log(abs(geo(k, t)[0] - 0.05j))

    def x_of(k, t):
        return math.cos(t + k) + 0.3 * math.sin(2 * t)

    y = O.rhs_y(d.et, d.etp, d.A, n, Dm.gamma_log(d, 0.05j))
    B, _ = O.matrices_BD(d.et, d.etp, d.A, n)
    xv = np.concatenate([[x_of(k, t) for t in Dm.nodes(n)] for k in range(d.m1)])
    Bx = B @ xv - B.sum(axis=1) * xv
    for i in (0, 37, n + 5, 2 * n + 90):
        k, p = divmod(i, n)
        s = Dm.nodes(n)[p]
        zs, _ = geo(k, s)
        As = A_of(k, s)

        def kern(l, t):
            zt, zpt = geo(l, t)
            return As / A_of(l, t) * zpt / (zt - zs) / math.pi

        phi = 0.0
        psi = 0.0
        for l in range(d.m1):
            pts = [s] if (l == k and 0 < s < 2 * math.pi) else None
            phi += _quad_component(lambda t: kern(l, t) * (gamma_of(l, t) - gamma_of(k, s)),
                                   0.0, 2 * math.pi, pts).real
            psi += _quad_component(lambda t: kern(l, t) * (x_of(l, t) - x_of(k, s)),
                                   0.0, 2 * math.pi, pts).imag
        assert abs(y[i] - phi) < 1e-9, (i, y[i], phi)
        assert abs(Bx[i] - psi) < 1e-9, (i, Bx[i], psi)


def test_adjoint_diagonal_against_quadrature():
    """e_i of Eq. (ei): 1 - c + r(t_i) - (2 pi/n) sum_{j != i} N(t_j, t_i) with
    r(s) = int N_g(s, t) dt (Eq. r(s)) by quadrature, against the oracle's e
    (computed through the Neumann-kernel form, Eq. ei2)."""
    n = 128
    d = Dm.ex4_circles(0.2, n)
    e = O.adjoint_e(d.et, d.etp, d.etpp, d.A, d.Ap, n, d.c)
    B, _ = O.matrices_BD(d.et, d.etp, d.A, n)
    rot = np.exp(1j * (math.pi / 2 - d.theta))
    for i in (3, n + 17, 4 * n + 100):
        k, p = divmod(i, n)
        s = Dm.nodes(n)[p]
        zs, zps, _ = d.curves[k].eval(np.array([s]))
        zs, zps = zs[0], zps[0]
        As = rot[k]

        def ng(l, t):
            zt, zpt, _ = d.curves[l].eval(np.array([t]))
            At = rot[l]
            return (As * zpt[0] - At * zps) / (As * (zt[0] - zs)) / math.pi

        r = 0.0
        for l in range(d.m1):
            pts = [s] if (l == k and 0 < s < 2 * math.pi) else None
            r += _quad_component(lambda t: ng(l, t), 0.0, 2 * math.pi, pts).imag
        e_quad = 1 - d.c + r - B[:, i].sum()
        assert abs(e[i] - e_quad) < 1e-9, (i, e[i], e_quad)


# ---------------------------------------------------------------- planted mistakes
def _pins_pass():
    try:
        test_disk_closed_form(0.3 + 0.2j)
        test_manufactured_nonconstant_theta()
        test_h_piecewise_constant_config1()
        test_unit_circle_operators()
        test_wittich_circulant_spectrum()
    except AssertionError:
        return False
    return True


def test_planted_mistakes_are_caught(monkeypatch):
    orig_block = O.nystrom_block
    orig_L = O.circulant_L
    orig_M = O.matrix_M
    orig_MD = O._M_from_D
    orig_KB = O._IminusN_from_B
    assert _pins_pass()

    def transposed(et, etp, A, n, rows, cols):
        rows = np.asarray(rows)
        cols = np.asarray(cols)
        K = orig_block(et, etp, A, n, rows, cols)
        Ar = np.asarray(A)
        return K * (Ar[cols][None, :] / Ar[rows][:, None]) ** 2

    def flipped_L(n):
        return -orig_L(n)

    def no_diag_D1(D, n, m1):
        s = D.sum(axis=1)
        out = orig_MD(D, n, m1)
        idx = np.arange(out.shape[0])
        out[idx, idx] += s
        return out

    def identity_not_two(B):
        K = orig_KB(B)
        idx = np.arange(K.shape[0])
        K[idx, idx] -= 1.0
        return K

    mutants = [("nystrom_block", transposed), ("circulant_L", flipped_L),
               ("_M_from_D", no_diag_D1), ("_IminusN_from_B", identity_not_two)]
    for name, fn in mutants:
        monkeypatch.setattr(O, name, fn)
        assert not _pins_pass(), name
        monkeypatch.undo()
    assert O.nystrom_block is orig_block and O.matrix_M is orig_M
