"""Parity of the CUDA library (through the C ABI) with the dense FP64 oracle.

Tolerances (derived from the arithmetic, u = 2^-53, u32 = 2^-24):
  * Cauchy sums: each FP64 term carries at most ~8 roundings; a sum of N
    terms adds gamma_N ~ N u, so |z - z_ref|_i <= (64 + N) u S_i with
    S_i = sum_j |w_j / (eta_i - eta_j)|.  FP32: the same with u32, plus the
    rounding of the tile-relative positions (relative 2^-24 of |offset|/|d|),
    covered by a factor 8.
  * Operators y = A x: the same bound on |A| |x| with a factor 4 for the
    epilogue (diagonal and circulant terms are FP64).
  * Double-float (df32) Cauchy sums: each term carries ~2^-46 relative error
    from the error-free transformations plus the rounding of the tile-relative
    positions, at most 2^-47 (|o_i| + |delta_j|) / |d_ij| with |o_i| <= |d_ij| +
    |delta_j| and |delta_j| <= D (the largest node-to-reference distance of a
    source tile); hence |dz_i| <= (64 + N) 2^-45 S_i + 2^-45 D sum_j |w_j|/|d_ij|^2.
  * Solves: mu within 1e-10 relative (max norm) of the oracle's LU solution,
    h within 1e-10 per component relative to max(1, |h|_inf); GMRES runs to
    the paper's gmrestol 1e-12 and the test geometries have condition
    numbers below 100.  Mixed precision iterates to the same FP64 residual.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import gnk_dense as O
from paper_1308_5351_gb300 import domains as Dm

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53
U32 = 2.0 ** -24


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


def _domains():
    rng = np.random.default_rng(11)
    ell = Dm.random_ellipses(rng, 5, 1.6)
    ell7 = Dm.random_ellipses(rng, 7, 2.0)
    return {
        "three_circles_n170": Dm.three_circles(170),            # N=510, ragged, direct circulant
        "three_circles_n256": Dm.three_circles(256),            # config 1
        "ellipses5_n512": Dm.build_domain(ell, 512, bounded=False),   # N=2560, odd m1, FFT
        "ellipses7_n300": Dm.build_domain(ell7, 300, bounded=False),  # N=2100, direct circulant
        "graded_square_n128": Dm.build_domain([Dm.Circle(0j, 1.6, ccw=True),
                                               Dm.square(0.3 + 0.1j, 0.5, ccw=False)], 128,
                                              bounded=True, alpha=-1.2 + 0.3j),
        "disk_n8": Dm.disk(8, 0.3 + 0.2j),                      # N < one tile
        "ex2_theta_n64": Dm.ex2_circles(0.1, 64, theta=[math.pi / 2, 0, math.pi / 2, 0, math.pi / 2]),
    }


DOMS = _domains()


def _bnd(G, d):
    return G.Boundary.from_domain(d, adjoint=True, device="cuda")


# ------------------------------------------------------------------ Cauchy sums
PREC = {"fp64": 0, "fp32": 2, "df32": 3}
UDF = 2.0 ** -45


def _tile_span(et, S=256):
    """Largest distance from a node to its source tile's reference node."""
    D = 0.0
    for j0 in range(0, len(et), S):
        blk = et[j0:j0 + S]
        D = max(D, float(np.abs(blk - blk[len(blk) // 2]).max()))
    return D


@pytest.mark.parametrize("name", list(DOMS))
@pytest.mark.parametrize("prec", ["fp64", "fp32", "df32"])
def test_cauchy_sum(G, name, prec):
    d = DOMS[name]
    rng = np.random.default_rng(3)
    w = rng.normal(size=d.N) + 1j * rng.normal(size=d.N)
    E = O.cauchy_matrix(d.et)
    ref = E @ w
    S = np.abs(E) @ np.abs(w)
    with _bnd(G, d) as b:
        z = _host(b.cauchy_sum(_dev(w), precision=PREC[prec]))
    err = np.abs(z - ref)
    if prec == "df32":
        tol = (64 + d.N) * UDF * S + UDF * _tile_span(d.et) * (np.abs(E) ** 2 @ np.abs(w))
    else:
        u = U64 if prec == "fp64" else 8 * U32
        tol = (64 + d.N) * u * S
    assert np.all(err <= tol), (name, prec, float((err / S).max()))


# ------------------------------------------------------------------ operators
@pytest.mark.parametrize("name", list(DOMS))
def test_operators_fp64(G, name):
    d = DOMS[name]
    rng = np.random.default_rng(5)
    x = rng.normal(size=d.N)
    IN = O.matrix_IminusN(d.et, d.etp, d.A, d.n)
    Mm = O.matrix_M(d.et, d.etp, d.A, d.n)
    Ad = O.matrix_adjoint(d.et, d.etp, d.etpp, d.A, d.Ap, d.n, d.c)
    Lh = O.block_L(d.n, d.m1)
    xd = _dev(x)
    with _bnd(G, d) as b:
        got = {
            "IminusN": _host(b.apply_IminusN(xd)),
            "M": _host(b.apply_M(xd)),
            "adjoint": _host(b.apply_adjoint(xd)),
            "circulant": _host(b.apply_circulant(xd)),
        }
    for key, A in (("IminusN", IN), ("M", Mm), ("adjoint", Ad), ("circulant", Lh)):
        ref = A @ x
        scale = np.abs(A) @ np.abs(x)
        tol = 4 * (64 + d.N) * U64 * scale.max()
        assert np.abs(got[key] - ref).max() <= tol, (name, key, np.abs(got[key] - ref).max(), tol)


@pytest.mark.parametrize("name", ["three_circles_n256", "ellipses5_n512", "graded_square_n128"])
def test_operators_fp32(G, name):
    d = DOMS[name]
    rng = np.random.default_rng(6)
    x = rng.normal(size=d.N)
    IN = O.matrix_IminusN(d.et, d.etp, d.A, d.n)
    Ad = O.matrix_adjoint(d.et, d.etp, d.etpp, d.A, d.Ap, d.n, d.c)
    xd = _dev(x)
    with _bnd(G, d) as b:
        y1 = _host(b.apply_IminusN(xd, precision=G.GNK_PREC_FP32))
        y2 = _host(b.apply_adjoint(xd, precision=G.GNK_PREC_FP32))
    for A, y in ((IN, y1), (Ad, y2)):
        scale = (np.abs(A) @ np.abs(x)).max()
        assert np.abs(y - A @ x).max() <= 4 * 8 * (64 + d.N) * U32 * scale


@pytest.mark.parametrize("name", ["three_circles_n256", "ellipses5_n512", "graded_square_n128",
                                  "ellipses7_n300"])
def test_operators_df32(G, name):
    d = DOMS[name]
    rng = np.random.default_rng(8)
    x = rng.normal(size=d.N)
    IN = O.matrix_IminusN(d.et, d.etp, d.A, d.n)
    Mm = O.matrix_M(d.et, d.etp, d.A, d.n)
    Ad = O.matrix_adjoint(d.et, d.etp, d.etpp, d.A, d.Ap, d.n, d.c)
    E = O.cauchy_matrix(d.et)
    xd = _dev(x)
    with _bnd(G, d) as b:
        got = [_host(b.apply_IminusN(xd, precision=G.GNK_PREC_DF32)),
               _host(b.apply_M(xd, precision=G.GNK_PREC_DF32)),
               _host(b.apply_adjoint(xd, precision=G.GNK_PREC_DF32))]
    # the Cauchy-sum bound above, carried through |A| and the (2/n)|q| or |A| factors
    span = _tile_span(d.et)
    for A, y, sc in ((IN, got[0], d.etp / d.A), (Mm, got[1], d.etp / d.A), (Ad, got[2], d.A)):
        w = np.abs(sc * x)
        zb = (64 + d.N) * UDF * (np.abs(E) @ w) + UDF * span * (np.abs(E) ** 2 @ w)
        fac = np.abs(d.A) if A is not Ad else np.abs(d.etp / d.A)
        tol = 4 * ((2.0 / d.n) * fac * zb + (64 + d.N) * U64 * (np.abs(A) @ np.abs(x)))
        assert np.all(np.abs(y - A @ x) <= tol), name


# ------------------------------------------------------------------ solves
def _solve_cases():
    rng = np.random.default_rng(21)
    cases = {}
    d = DOMS["three_circles_n256"]
    cases["config1_log"] = (d, Dm.gamma_log(d, 0.05j))
    d = DOMS["ellipses5_n512"]
    cases["ellipses_log"] = (d, Dm.gamma_log(d, d.holes[0]))
    d = DOMS["graded_square_n128"]
    cases["graded_manufactured"] = (d, Dm.manufactured(d, Dm.f_bounded_ex1)[0])
    d = DOMS["ex2_theta_n64"]
    cases["ex2_theta"] = (d, Dm.manufactured(d, Dm.f_bounded_ex1)[0])
    d = DOMS["ellipses7_n300"]
    cases["ellipses7_random"] = (d, rng.normal(size=d.N))
    return cases


SOLVE = _solve_cases()


SOLVE_PREC = {"fp64": 0, "mixed": 1, "df32": 3, "mixed_df": 4}


@pytest.mark.parametrize("case", list(SOLVE))
@pytest.mark.parametrize("prec", list(SOLVE_PREC))
def test_solve_ie_and_h(G, case, prec):
    d, gam = SOLVE[case]
    mu_ref, h_ref, hk_ref = O.fbie(d.et, d.etp, d.A, d.n, gam)
    p = SOLVE_PREC[prec]
    with _bnd(G, d) as b:
        gd = _dev(gam)
        mu, res = b.solve_ie(gd, tol=1e-12, restart=20, maxit=50, precision=p)
        assert res.status == 0 and res.relres <= 1e-12
        h, hk = b.compute_h(mu, gd)
        mu, h, hk = _host(mu), _host(h), _host(hk)
    assert np.abs(mu - mu_ref).max() <= 1e-10 * np.abs(mu_ref).max()
    hs = max(1.0, np.abs(h_ref).max())
    assert np.abs(h - h_ref).max() <= 1e-10 * hs
    assert np.abs(hk - hk_ref).max() <= 1e-10 * hs
    if prec.startswith("mixed"):
        assert res.matvecs_fp32 > 0 and res.refinements >= 1


@pytest.mark.parametrize("case", list(SOLVE))
@pytest.mark.parametrize("prec", list(SOLVE_PREC))
def test_fbie_fused(G, case, prec):
    """gnk_fbie: mu and h from the fewest Cauchy sums, handle built with the
    matching precision of the precomputed sums."""
    d, gam = SOLVE[case]
    mu_ref, h_ref, hk_ref = O.fbie(d.et, d.etp, d.A, d.n, gam)
    p = SOLVE_PREC[prec]
    bp = G.GNK_PREC_DF32 if prec in ("df32", "mixed_df") else G.GNK_PREC_FP64
    with G.Boundary.from_domain(d, adjoint=False, device="cuda", precision=bp) as b:
        mu, h, hk, res = b.fbie(_dev(gam), tol=1e-12, precision=p)
        assert res.status == 0 and res.relres <= 1e-12
        mu, h, hk = _host(mu), _host(h), _host(hk)
    assert np.abs(mu - mu_ref).max() <= 1e-10 * np.abs(mu_ref).max()
    hs = max(1.0, np.abs(h_ref).max())
    assert np.abs(h - h_ref).max() <= 1e-10 * hs
    assert np.abs(hk - hk_ref).max() <= 1e-10 * hs


@pytest.mark.parametrize("case", ["config1_log", "ellipses_log", "graded_manufactured"])
@pytest.mark.parametrize("prec", list(SOLVE_PREC))
def test_solve_adjoint_ie(G, case, prec):
    d, gam = SOLVE[case]
    ref = O.solve_adjoint_ie(d.et, d.etp, d.etpp, d.A, d.Ap, d.n, d.c, gam)
    p = SOLVE_PREC[prec]
    with _bnd(G, d) as b:
        mu, res = b.solve_adjoint_ie(_dev(gam), tol=1e-12, precision=p)
        assert res.status == 0
        mu = _host(mu)
    assert np.abs(mu - ref).max() <= 1e-10 * np.abs(ref).max()


def test_closed_form_disk(G):
    """Unit disk, A = eta - alpha: mu = arg(1 - conj(alpha) eta), h = -log(1-|alpha|^2)."""
    alpha = 0.3 + 0.2j
    d = Dm.disk(128, alpha)
    gam = np.log(np.abs(d.et - alpha))
    with _bnd(G, d) as b:
        mu, res = b.solve_ie(_dev(gam))
        h, hk = b.compute_h(mu, _dev(gam))
    assert np.abs(_host(mu) - np.angle(1 - np.conj(alpha) * d.et)).max() < 1e-12
    assert np.abs(_host(h) + math.log(1 - abs(alpha) ** 2)).max() < 1e-12


def test_host_buffers_match_device(G):
    """Host (numpy) arrays through the same entry points give identical results."""
    d = DOMS["three_circles_n256"]
    gam = Dm.gamma_log(d, 0.05j)
    b_host = G.Boundary.from_domain(d, adjoint=True)           # host geometry
    b_dev = _bnd(G, d)
    mu_h, _ = b_host.solve_ie(np.ascontiguousarray(gam))
    mu_d, _ = b_dev.solve_ie(_dev(gam))
    assert isinstance(mu_h, np.ndarray)
    assert np.array_equal(mu_h, _host(mu_d))
    h_h, hk_h = b_host.compute_h(mu_h, np.ascontiguousarray(gam))
    h_d, hk_d = b_dev.compute_h(mu_d, _dev(gam))
    assert np.array_equal(h_h, _host(h_d)) and np.array_equal(hk_h, _host(hk_d))
    b_host.close()
    b_dev.close()


def test_deterministic_repeat(G):
    d = DOMS["ellipses5_n512"]
    w = _dev(np.random.default_rng(1).normal(size=d.N) + 1j)
    with _bnd(G, d) as b:
        z1 = _host(b.cauchy_sum(w))
        z2 = _host(b.cauchy_sum(w))
    assert np.array_equal(z1, z2)


# ------------------------------------------------------------------ failure paths (host-made)
def test_nonfinite_input_rejected(G):
    d = Dm.three_circles(32)
    et = d.et.copy()
    et[5] = np.nan
    with pytest.raises(G.GnkError) as e:
        G.Boundary(d.m1, d.n, _dev(et), _dev(d.etp), _dev(d.A), bounded=True)
    assert e.value.code == G.GNK_ENONFINITE


def test_nonconvergence_reports_best_iterate(G):
    d = DOMS["ellipses5_n512"]
    gam = Dm.gamma_log(d, d.holes[0])
    with _bnd(G, d) as b:
        mu, res = b.solve_ie(_dev(gam), restart=2, maxit=1, tol=1e-14)
        assert res.status == G.GNK_ENOTCONV
        assert 0 < res.relres < 1 and np.all(np.isfinite(_host(mu)))


def test_adjoint_needs_second_derivative(G):
    d = Dm.three_circles(32)
    b = G.Boundary(d.m1, d.n, _dev(d.et), _dev(d.etp), _dev(d.A), bounded=True)
    with pytest.raises(G.GnkError) as e:
        b.apply_adjoint(_dev(np.ones(d.N)))
    assert e.value.code == G.GNK_EINVAL
    b.close()


def test_bad_options_rejected(G):
    d = Dm.three_circles(32)
    with _bnd(G, d) as b:
        with pytest.raises(G.GnkError):
            b.solve_ie(_dev(np.ones(d.N)), restart=0)
        with pytest.raises(G.GnkError):
            b.solve_ie(_dev(np.ones(d.N)), precision=7)


@pytest.mark.parametrize("prec", ["fp64", "mixed_df"])
@pytest.mark.parametrize("adjoint", [False, True])
def test_deferred_precompute(G, prec, adjoint):
    """GNK_BUILD_DEFER: Eone and the diagonals are formed by the first call that
    needs them (fused with E(q gamma) inside gnk_fbie when possible); results
    match the immediate build."""
    d, gam = SOLVE["ellipses_log"]
    mu_ref, h_ref, hk_ref = O.fbie(d.et, d.etp, d.A, d.n, gam)
    p = SOLVE_PREC[prec]
    bp = (G.GNK_PREC_DF32 if prec == "mixed_df" else G.GNK_PREC_FP64) | G.GNK_BUILD_DEFER
    with G.Boundary.from_domain(d, adjoint=adjoint, device="cuda", precision=bp) as b:
        mu, h, hk, res = b.fbie(_dev(gam), tol=1e-12, precision=p)
        mu, h, hk = _host(mu), _host(h), _host(hk)
        y = _host(b.apply_IminusN(_dev(gam)))
    assert np.abs(mu - mu_ref).max() <= 1e-10 * np.abs(mu_ref).max()
    assert np.abs(hk - hk_ref).max() <= 1e-10 * max(1.0, np.abs(h_ref).max())
    K = O.matrix_IminusN(d.et, d.etp, d.A, d.n)
    assert np.abs(y - K @ gam).max() <= 1e-11 * (np.abs(K) @ np.abs(gam)).max()
    with G.Boundary.from_domain(d, adjoint=True, device="cuda", precision=bp) as b:
        phi, r2 = b.solve_adjoint_ie(_dev(gam), tol=1e-12)
    ref = O.solve_adjoint_ie(d.et, d.etp, d.etpp, d.A, d.Ap, d.n, d.c, gam)
    assert np.abs(_host(phi) - ref).max() <= 1e-10 * np.abs(ref).max()
