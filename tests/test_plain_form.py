"""The Nystrom method without singularity subtraction (Sec. 7, Ex. 2
comparison): I - N with N(t,t) of Eq. (N-tt) on the diagonal, M by Wittich's
rule plus the trapezoidal rule for M_1 with M_1(t,t) of Eq. (M1-tt), and
I + N* + J with the same diagonal.

CPU pins of the oracle's plain matrices:
  * N(t,t) and M_1(t,t) are the limits of N(s,t) and M(s,t) + cot((s-t)/2)/(2 pi)
    as t -> s (the defining property of Eqs. N-tt, M1-tt), on an ellipse with a
    non-constant A;
  * unit circle, A = eta: N is constant -1/(2 pi) and M_1 = 0, so I - N = I + 11^T/n
    and M is the discrete conjugation (M cos kt = -sin kt) exactly;
  * Eq. (K-L): the plain M minus diag(M_1(t,t)) equals D + L-hat;
  * disk closed form and manufactured solutions converge exponentially;
  * Ex. 2's finding for constant theta: at separation 1e-2 the subtracted form
    is exact to round-off while the plain form has O(1) errors at n = 128;
  * adjoint: (I + N* + J) phi = 1 gives J phi = 1;
  * planted mistakes in the diagonals or in Wittich's sign make pins fail.
GPU: a handle built with GNK_BUILD_PLAIN reproduces these matrices through every
operator and solver of the C ABI.
"""
import math

import numpy as np
import pytest

from oracle import gnk_dense as O
from paper_1308_5351_gb300 import domains as Dm


def _args(d):
    return d.et, d.etp, d.etpp, d.A, d.Ap, d.n


def _kernels(cv, alpha, s, t):
    """N(s,t), M(s,t) of Eqs. (N), (M) with A = eta - alpha, from the curve itself."""
    zs, _, _ = cv.eval(np.array([s]))
    zt, zpt, _ = cv.eval(np.array([t]))
    k = (zs[0] - alpha) / (zt[0] - alpha) * zpt[0] / (zt[0] - zs[0]) / math.pi
    return k.imag, k.real


def test_diagonal_values_are_the_kernel_limits():
    cv = Dm.Ellipse(0.1 + 0.2j, 1.0, 0.6, 0.3, ccw=True)
    alpha = 0.05 + 0.1j
    dl = 1e-4
    for s in (0.3, 1.7, 4.0):
        z, zp, zpp = cv.eval(np.array([s]))
        A = z - alpha
        Ntt = O.kernel_N_diag(zp, zpp, A, zp)[0]
        M1tt = O.kernel_M1_diag(zp, zpp, A, zp)[0]
        n_lim = 0.5 * (_kernels(cv, alpha, s, s + dl)[0] + _kernels(cv, alpha, s, s - dl)[0])
        m_p = _kernels(cv, alpha, s, s + dl)[1] + 1.0 / math.tan(-dl / 2) / (2 * math.pi)
        m_m = _kernels(cv, alpha, s, s - dl)[1] + 1.0 / math.tan(dl / 2) / (2 * math.pi)
        assert abs(Ntt - n_lim) < 1e-7, (s, Ntt, n_lim)
        assert abs(M1tt - 0.5 * (m_p + m_m)) < 1e-7, (s, M1tt, 0.5 * (m_p + m_m))


def test_unit_circle_plain_matrices():
    n = 32
    d = Dm.disk(n, 0j)
    t = Dm.nodes(n)
    K = O.matrix_IminusN_plain(*_args(d))
    assert np.abs(K - (np.eye(n) + np.full((n, n), 1.0 / n))).max() < 1e-14
    M = O.matrix_M_plain(*_args(d))
    for k in range(1, n // 2):
        assert np.abs(M @ np.cos(k * t) + np.sin(k * t)).max() < 1e-13
    Ad = O.matrix_adjoint_plain(*_args(d))
    assert np.abs(Ad - np.eye(n)).max() < 1e-14


def test_plain_M_splits_as_D_plus_Lhat():
    """Eq. (K-L): -K + (2pi/n) M_1 = L + (2pi/n) M off the diagonal."""
    d = Dm.three_circles(64)
    Mp = O.matrix_M_plain(*_args(d))
    _, D = O.matrices_BD(d.et, d.etp, d.A, d.n)
    M1d = (2 * math.pi / d.n) * O.kernel_M1_diag(d.etp, d.etpp, d.A, d.Ap)
    assert np.abs(Mp - np.diag(M1d) - (D + O.block_L(d.n, d.m1))).max() < 1e-12


def test_plain_disk_closed_form():
    alpha = 0.3 + 0.2j
    errs = []
    for n in (16, 32, 64):
        d = Dm.disk(n, alpha)
        mu, h, _ = O.fbie_plain(*_args(d), np.log(np.abs(d.et - alpha)))
        errs.append(max(np.abs(mu - np.angle(1 - np.conj(alpha) * d.et)).max(),
                        np.abs(h + math.log(1 - abs(alpha) ** 2)).max()))
    assert errs[-1] < 1e-13 and errs[1] < errs[0] / 1e3


def test_plain_manufactured_three_circles():
    errs = []
    for n in (32, 64, 128):
        d = Dm.three_circles(n)
        gam, mu_ex = Dm.manufactured(d, Dm.f_bounded_ex1)
        mu, h, _ = O.fbie_plain(*_args(d), gam)
        errs.append(max(np.abs(mu - mu_ex).max(), np.abs(h).max()))
    assert errs[-1] < 1e-12 and errs[1] < errs[0] / 1e3


def test_ex2_subtraction_matters_for_close_boundaries():
    """Ex. 2, constant theta, separation 1e-2, n = 128: with the subtraction mu is
    exact to round-off; without it the error is O(1)."""
    d = Dm.ex2_circles(1e-2, 128)
    gam, mu_ex = Dm.manufactured(d, Dm.f_bounded_ex1)
    mu_p, _, _ = O.fbie_plain(*_args(d), gam)
    mu_s, _, _ = O.fbie(d.et, d.etp, d.A, d.n, gam)
    assert np.abs(mu_s - mu_ex).max() < 1e-12
    assert np.abs(mu_p - mu_ex).max() > 1e-2


def test_plain_adjoint_invariant():
    d = Dm.three_circles(128)
    phi = O.solve_adjoint_plain(*_args(d), np.ones(d.N))
    assert np.abs(phi.reshape(d.m1, d.n).mean(axis=1) - 1.0).max() < 1e-9


def _plain_pins_pass():
    try:
        test_diagonal_values_are_the_kernel_limits()
        test_unit_circle_plain_matrices()
        test_plain_manufactured_three_circles()
    except AssertionError:
        return False
    return True


def test_planted_mistakes_are_caught(monkeypatch):
    orig_N, orig_M1 = O.kernel_N_diag, O.kernel_M1_diag
    orig_M = O.matrix_M_plain
    assert _plain_pins_pass()

    def n_without_half(etp, etpp, A, Ap):
        return (O._ratio_limit(etpp, etp).imag - O._ratio_limit(Ap, A).imag) / math.pi

    def m1_flipped(etp, etpp, A, Ap):
        return -orig_M1(etp, etpp, A, Ap)

    def wittich_flipped(et, etp, etpp, A, Ap, n):
        out = orig_M(et, etp, etpp, A, Ap, n)
        _, m1 = O._sizes(et, n)
        p = np.arange(n)
        dd = p[:, None] - p[None, :]
        with np.errstate(divide="ignore"):
            K = np.where(dd % 2 != 0, (2.0 / n) / np.tan(dd * math.pi / n), 0.0)
        return out + 2.0 * np.kron(np.eye(m1), K)

    for name, fn in (("kernel_N_diag", n_without_half), ("kernel_M1_diag", m1_flipped),
                     ("matrix_M_plain", wittich_flipped)):
        monkeypatch.setattr(O, name, fn)
        assert not _plain_pins_pass(), name
        monkeypatch.undo()
    assert O.kernel_N_diag is orig_N and O.kernel_M1_diag is orig_M1


# ------------------------------------------------------------------ GPU
torch = pytest.importorskip("torch")
U64 = 2.0 ** -53


@pytest.fixture(scope="module")
def G():
    from paper_1308_5351_gb300 import build, gnk
    build.build()
    gnk.load()
    return gnk


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _host(t):
    return t.detach().cpu().numpy()


def _plain_domains():
    rng = np.random.default_rng(11)
    ell = Dm.random_ellipses(rng, 5, 1.6)
    return {
        "three_circles_n170": Dm.three_circles(170),                  # ragged, direct circulant
        "ellipses5_n512": Dm.build_domain(ell, 512, bounded=False),   # unbounded, odd m+1
        "graded_square_n128": Dm.build_domain([Dm.Circle(0j, 1.6, ccw=True),
                                               Dm.square(0.3 + 0.1j, 0.5, ccw=False)], 128,
                                              bounded=True, alpha=-1.2 + 0.3j),
        "ex2_theta_n64": Dm.ex2_circles(0.1, 64, theta=[math.pi / 2, 0, math.pi / 2, 0, math.pi / 2]),
    }


PDOMS = _plain_domains()


@pytest.mark.gpu
@pytest.mark.parametrize("name", list(PDOMS))
def test_plain_operators_match_oracle(G, name):
    """Tolerance as for the subtracted operators: 4 (64 + N) u max(|A| |x|)."""
    d = PDOMS[name]
    x = np.random.default_rng(5).normal(size=d.N)
    mats = {"IminusN": O.matrix_IminusN_plain(*_args(d)), "M": O.matrix_M_plain(*_args(d)),
            "adjoint": O.matrix_adjoint_plain(*_args(d))}
    with G.Boundary.from_domain(d, device="cuda", plain=True) as b:
        xd = _dev(x)
        got = {"IminusN": _host(b.apply_IminusN(xd)), "M": _host(b.apply_M(xd)),
               "adjoint": _host(b.apply_adjoint(xd))}
    for key, A in mats.items():
        tol = 4 * (64 + d.N) * U64 * (np.abs(A) @ np.abs(x)).max()
        err = np.abs(got[key] - A @ x).max()
        assert err <= tol, (name, key, err, tol)


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["three_circles_n170", "ellipses5_n512", "ex2_theta_n64"])
@pytest.mark.parametrize("prec", [0, 4])
def test_plain_fbie_and_adjoint_match_oracle(G, name, prec):
    """mu within 1e-10 relative of the oracle's LU solution, h within 1e-10 of
    max(1, |h|_inf), in FP64 and in FP32 GMRES with double-float refinement."""
    d = PDOMS[name]
    gam = np.log(np.abs(d.et - (d.holes[0] if d.holes else 0.05j)))
    mu_ref, h_ref, hk_ref = O.fbie_plain(*_args(d), gam)
    phi_ref = O.solve_adjoint_plain(*_args(d), gam)
    bp = G.GNK_PREC_DF32 if prec == 4 else G.GNK_PREC_FP64
    with G.Boundary.from_domain(d, device="cuda", plain=True, precision=bp) as b:
        mu, h, hk, res = b.fbie(_dev(gam), tol=1e-12, precision=prec)
        assert res.status == 0
        mu2, res2 = b.solve_ie(_dev(gam), tol=1e-12, precision=prec)
        assert res2.status == 0
        phi, res3 = b.solve_adjoint_ie(_dev(gam), tol=1e-12, precision=prec)
        assert res3.status == 0
        mu, h, hk, mu2, phi = map(_host, (mu, h, hk, mu2, phi))
    for m in (mu, mu2):
        assert np.abs(m - mu_ref).max() <= 1e-10 * np.abs(mu_ref).max()
    hs = max(1.0, np.abs(h_ref).max())
    assert np.abs(h - h_ref).max() <= 1e-10 * hs and np.abs(hk - hk_ref).max() <= 1e-10 * hs
    assert np.abs(phi - phi_ref).max() <= 1e-10 * np.abs(phi_ref).max()


@pytest.mark.gpu
def test_plain_needs_second_derivative_and_has_no_gradient(G):
    d = Dm.three_circles(64)
    with pytest.raises(G.GnkError):
        G.gnk_build_boundary_ex(d.m1, d.n, d.et, d.etp, d.A, None, None, True,
                                G.GNK_PREC_FP64 | G.GNK_BUILD_PLAIN)
    gam = np.log(np.abs(d.et - 0.05j))
    with G.Boundary.from_domain(d, device="cuda", plain=True) as b:
        mu, h, hk, res = b.fbie(_dev(gam))
        z = torch.zeros(d.N, dtype=torch.float64, device="cuda")
        zc = torch.zeros(d.N, dtype=torch.complex128, device="cuda")
        with pytest.raises(G.GnkError):
            G.gnk_fbie_backward(b.handle, mu, _dev(gam), z, z, zc, zc.clone(), zc.clone(), z.clone(),
                                G.options())
