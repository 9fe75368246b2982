"""The Cauchy sum by the fast multipole method (GNK_PREC_FMM; Sec. 2.5, Eqs.
fmm-1, fmm-E: the paper evaluates E w with the FMM of zfmm2dpart at iprec = 4,
tolerance 0.5e-12).

Parity: FMM products against the oracle's direct sums (the plain definition of
E), element by element.  Tolerance: |dz_i| <= 1e-12 S_i + (64 + N) u S_i with
S_i = sum_{j != i} |w_j / (eta_i - eta_j)|, i.e. the paper's FMM tolerance with a
factor 2 of margin plus the FP64 rounding bound of the direct sum.  (At the
expansion order 32 the measured truncation error on these geometries is about
1e-14 S_i.)  Operators, solves and h through the FMM against the dense oracle as
in tests/test_gpu_parity.py; the 65,536-node workload on sampled rows.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import gnk_dense as O
from paper_1308_5351_gb300 import domains as Dm

pytestmark = pytest.mark.gpu

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


def _domains():
    rng = np.random.default_rng(11)
    ell = Dm.random_ellipses(rng, 5, 1.6)
    return {
        "disk_n8": Dm.disk(8, 0.3 + 0.2j),                              # N below one leaf
        "three_circles_n170": Dm.three_circles(170),                    # N = 510
        "ellipses5_n512": Dm.build_domain(ell, 512, bounded=False),     # N = 2560
        "graded_square_n256": Dm.build_domain([Dm.Circle(0j, 1.6, ccw=True),
                                               Dm.square(0.3 + 0.1j, 0.5, ccw=False)], 256,
                                              bounded=True, alpha=-1.2 + 0.3j),  # clustered corners
        "ex4_eps1e-3_n512": Dm.ex4_circles(1e-3, 512),                  # close boundaries
        "ellipses64_n64": Dm.ellipses64(n=64),                          # N = 4096, several levels
    }


DOMS = _domains()


def _S(d, w, rows):
    out = np.empty(len(rows))
    for k, i in enumerate(rows):
        dd = d.et[i] - d.et
        dd[i] = np.inf
        out[k] = np.sum(np.abs(w / dd))
    return out


@pytest.mark.parametrize("name", list(DOMS))
def test_fmm_cauchy_sum_matches_direct(G, name):
    d = DOMS[name]
    rng = np.random.default_rng(3)
    w = rng.normal(size=d.N) + 1j * rng.normal(size=d.N)
    rows = np.arange(d.N)
    ref = O.cauchy_rows(d.et, w, rows)
    S = _S(d, w, rows)
    with G.Boundary.from_domain(d, adjoint=False, device="cuda") as b:
        z = _host(b.cauchy_sum(_dev(w), precision=G.GNK_PREC_FMM))
        z2 = _host(b.cauchy_sum(_dev(w), precision=G.GNK_PREC_FMM))
    err = np.abs(z - ref)
    tol = 1e-12 * S + (64 + d.N) * U64 * S
    assert np.all(err <= tol), (name, (err / S).max())
    assert np.array_equal(z, z2)  # fixed summation order


@pytest.mark.parametrize("name", ["three_circles_n170", "ellipses5_n512", "graded_square_n256"])
def test_fmm_operators(G, name):
    """Operators through the FMM: the Cauchy-sum tolerance carried through |A|, (2/n)|q|."""
    d = DOMS[name]
    x = np.random.default_rng(5).normal(size=d.N)
    E = np.abs(O.cauchy_matrix(d.et))
    mats = {"IminusN": (O.matrix_IminusN(d.et, d.etp, d.A, d.n), d.etp / d.A, np.abs(d.A)),
            "M": (O.matrix_M(d.et, d.etp, d.A, d.n), d.etp / d.A, np.abs(d.A)),
            "adjoint": (O.matrix_adjoint(d.et, d.etp, d.etpp, d.A, d.Ap, d.n, d.c), d.A,
                        np.abs(d.etp / d.A))}
    with G.Boundary.from_domain(d, device="cuda") as b:
        xd = _dev(x)
        got = {"IminusN": _host(b.apply_IminusN(xd, precision=G.GNK_PREC_FMM)),
               "M": _host(b.apply_M(xd, precision=G.GNK_PREC_FMM)),
               "adjoint": _host(b.apply_adjoint(xd, precision=G.GNK_PREC_FMM))}
    for key, (A, sc, fac) in mats.items():
        S = E @ np.abs(sc * x)
        tol = (2.0 / d.n) * fac * (1e-12 + (64 + d.N) * U64) * S * 4 \
            + 4 * (64 + d.N) * U64 * (np.abs(A) @ np.abs(x))
        err = np.abs(got[key] - A @ x)
        assert np.all(err <= tol), (name, key, (err / tol).max())


SOLVE = {
    "config1_log": (Dm.three_circles(256), lambda d: Dm.gamma_log(d, 0.05j)),
    "ellipses_log": (DOMS["ellipses5_n512"], lambda d: Dm.gamma_log(d, d.holes[0])),
    "graded_manufactured": (DOMS["graded_square_n256"], lambda d: Dm.manufactured(d, Dm.f_bounded_ex1)[0]),
}


@pytest.mark.parametrize("case", list(SOLVE))
@pytest.mark.parametrize("prec", ["fmm", "mixed_fmm"])
def test_fmm_fbie_matches_oracle(G, case, prec):
    """mu within 1e-10 relative, h within 1e-10 max(1, |h|_inf), as for the direct sums:
    the FMM error (<= 1e-12 relative to S_i) is far below the solve tolerance."""
    d, gfun = SOLVE[case]
    gam = gfun(d)
    mu_ref, h_ref, hk_ref = O.fbie(d.et, d.etp, d.A, d.n, gam)
    p = G.GNK_PREC_FMM if prec == "fmm" else G.GNK_PREC_MIXED_FMM
    with G.Boundary.from_domain(d, adjoint=False, device="cuda", precision=G.GNK_PREC_FMM) as b:
        mu, h, hk, res = b.fbie(_dev(gam), tol=1e-12, precision=p)
        assert res.status == 0
        mu, h, hk = _host(mu), _host(h), _host(hk)
    assert np.abs(mu - mu_ref).max() <= 1e-10 * np.abs(mu_ref).max()
    hs = max(1.0, np.abs(h_ref).max())
    assert np.abs(h - h_ref).max() <= 1e-10 * hs and np.abs(hk - hk_ref).max() <= 1e-10 * hs


def test_fmm_adjoint_solve(G):
    d = DOMS["ellipses5_n512"]
    gam = Dm.gamma_log(d, d.holes[0])
    ref = O.solve_adjoint_ie(d.et, d.etp, d.etpp, d.A, d.Ap, d.n, d.c, gam)
    with G.Boundary.from_domain(d, device="cuda") as b:
        mu, res = b.solve_adjoint_ie(_dev(gam), tol=1e-12, precision=G.GNK_PREC_MIXED_FMM)
        assert res.status == 0
    assert np.abs(_host(mu) - ref).max() <= 1e-10 * np.abs(ref).max()


def test_fmm_fullsize_ellipses64_sampled_rows(G):
    """64 ellipses, N = 65,536: 256 sampled rows against the oracle's direct sums."""
    d = Dm.ellipses64()
    rng = np.random.default_rng(9)
    w = rng.normal(size=d.N) + 1j * rng.normal(size=d.N)
    rows = np.sort(rng.choice(d.N, 256, replace=False))
    ref = O.cauchy_rows(d.et, w, rows)
    S = _S(d, w, rows)
    with G.Boundary.from_domain(d, adjoint=False, device="cuda") as b:
        z = _host(b.cauchy_sum(_dev(w), precision=G.GNK_PREC_FMM))
    err = np.abs(z[rows] - ref)
    assert np.all(err <= 1e-12 * S + (64 + d.N) * U64 * S), (err / S).max()


def test_profile_mask_records_only_selected_kinds(G):
    """gnk_profile_mask: with only the M2L bit set, an FMM product records the
    M2L launch and nothing else; with all bits set, the near-field, L2P, upward
    pass and L2L kernels too."""
    d = DOMS["ellipses64_n64"]
    w = _dev(np.random.default_rng(2).normal(size=d.N) + 0j)
    with G.Boundary.from_domain(d, adjoint=False, device="cuda") as b:
        b.cauchy_sum(w, precision=G.GNK_PREC_FMM)      # tree and tables built
        torch.cuda.synchronize()
        try:
            G.gnk_profile_mask(1 << G.PROF_FMM)
            G.gnk_profile_enable(True)
            b.cauchy_sum(w, precision=G.GNK_PREC_FMM)
            torch.cuda.synchronize()
            only = {k: G.gnk_profile_query_ex(k) for k in range(12)}
            G.gnk_profile_mask(0xffffffff)
            G.gnk_profile_enable(True)                  # clears the records
            b.cauchy_sum(w, precision=G.GNK_PREC_FMM)
            torch.cuda.synchronize()
            every = {k: G.gnk_profile_query_ex(k) for k in range(12)}
        finally:
            G.gnk_profile_enable(False)
            G.gnk_profile_mask(0xffffffff)
    assert only[G.PROF_FMM][0] >= 1 and only[G.PROF_FMM][3] > 0
    assert all(only[k][0] == 0 for k in range(12) if k != G.PROF_FMM)
    assert every[G.PROF_FMM][0] == only[G.PROF_FMM][0]
    assert every[G.PROF_FMMNEAR][0] >= 1 and every[G.PROF_FMML2P][0] >= 1
    assert every[G.PROF_FMMUP][0] >= 1 and every[G.PROF_FMML2L][0] >= 1


@pytest.mark.parametrize("count,radius,n", [(64, 1e-4, 1024), (16, 1e-5, 1024)])
def test_fmm_deep_tree_clustered_circles(G, count, radius, n):
    """Tiny circles on a coarse grid: the leaf level goes below 11 (14 and 16 here),
    past the device tree builder's lookup grids, so the host builder makes the tree.
    Sampled rows against the oracle's direct sums."""
    side = int(round(count ** 0.5))
    curves = [Dm.Circle(complex(0.1 * i, 0.1 * j), radius, ccw=False) for i in range(side) for j in range(side)]
    d = Dm.build_domain(curves, n, bounded=False)
    rng = np.random.default_rng(17)
    w = rng.normal(size=d.N) + 1j * rng.normal(size=d.N)
    rows = np.sort(rng.choice(d.N, 256, replace=False))
    ref = O.cauchy_rows(d.et, w, rows)
    S = _S(d, w, rows)
    with G.Boundary.from_domain(d, adjoint=False, device="cuda") as b:
        z = _host(b.cauchy_sum(_dev(w), precision=G.GNK_PREC_FMM))
    err = np.abs(z[rows] - ref)
    assert np.all(err <= 1e-12 * S + (64 + d.N) * U64 * S), (err / S).max()
