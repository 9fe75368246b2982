"""Batched FBIE (many domains of uneven connectivity and n, several
right-hand sides each) against the oracle, system by system.

Tolerance: each system is solved to the relative residual 1e-12, so mu agrees
with the oracle's LU solution to 1e-10 relative and h to 1e-10 relative to
max(1, |h|_inf), as for the single-domain solves."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import gnk_dense as O
from paper_1308_5351_gb300 import domains as Dm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_1308_5351_gb300 import build, gnk
    build.build()
    gnk.load()
    return gnk


def _batch_case(seed=4):
    doms = Dm.batch_domains(seed, count=6, conn=(2, 5), ns=(32, 48, 64, 128))
    doms.append(Dm.three_circles(64))                 # bounded, A = eta - alpha
    doms.append(Dm.ex2_circles(0.1, 50, theta=[1.5707963267948966, 0, 1.5707963267948966, 0,
                                                1.5707963267948966]))  # n = 50: direct circulant
    nrhs = [d.m1 for d in doms]
    nrhs[1] = 1
    gams = []
    for d, r in zip(doms, nrhs):
        for k in range(r):
            gams.append(Dm.gamma_log(d, d.holes[k]) if not (d.bounded and k == 0)
                        else Dm.gamma_log(d, d.alpha + 0.01j))
    return doms, nrhs, np.concatenate(gams)


@pytest.mark.parametrize("autotune", [True, False])
def test_batch_matches_oracle(G, autotune):
    doms, nrhs, gam = _batch_case()
    with G.Batch(doms, nrhs, autotune=autotune, device="cuda") as b:
        assert b.L == gam.size
        mu, h, hk, res, rel = b.fbie(torch.as_tensor(gam, device="cuda"), tol=1e-12, restart=20)
        assert res.status == 0 and rel.max() <= 1e-12
        mu, h, hk = mu.cpu().numpy(), h.cpu().numpy(), hk.cpu().numpy()
        tun = b.tuning()
    assert tun["fp32_group"] in (4, 8) and tun["df_group"] in (1, 2, 4)
    off, koff = 0, 0
    for d, r in zip(doms, nrhs):
        for k in range(r):
            g = gam[off:off + d.N]
            mu_r, h_r, hk_r = O.fbie(d.et, d.etp, d.A, d.n, g)
            assert np.abs(mu[off:off + d.N] - mu_r).max() <= 1e-10 * np.abs(mu_r).max()
            hs = max(1.0, np.abs(h_r).max())
            assert np.abs(h[off:off + d.N] - h_r).max() <= 1e-10 * hs
            assert np.abs(hk[koff:koff + d.m1] - hk_r).max() <= 1e-10 * hs
            off += d.N
            koff += d.m1


def test_batch_repeat_and_host_arrays(G):
    """A second solve reuses the captured graph; host arrays give the same result."""
    doms, nrhs, gam = _batch_case(seed=7)
    with G.Batch(doms, nrhs, autotune=False) as b:
        mu1, h1, hk1, r1, _ = b.fbie(np.ascontiguousarray(gam), tol=1e-12)
        mu2, h2, hk2, r2, _ = b.fbie(np.ascontiguousarray(gam), tol=1e-12)
    assert isinstance(mu1, np.ndarray)
    assert np.array_equal(mu1, mu2) and np.array_equal(hk1, hk2)
    assert r1.status == 0 and r2.status == 0


def test_batch_rejects_bad_domains(G):
    d = Dm.three_circles(16)
    with pytest.raises(G.GnkError):
        G.Batch([d], [0])


@pytest.mark.parametrize("prec", [2, 3])
def test_batch_apply_matches_oracle(G, prec):
    """One persistent launch applies (2I + diag(B1) - B) to every system; the
    FP32 bound of the single-domain tests (8 u32 per term, factor 4) and the
    double-float bound scaled by |A||x| cover it."""
    doms, nrhs, _ = _batch_case(seed=9)
    rng = np.random.default_rng(2)
    x = rng.normal(size=sum(d.N * r for d, r in zip(doms, nrhs)))
    with G.Batch(doms, nrhs, autotune=False, device="cuda") as b:
        y = b.apply_IminusN(torch.as_tensor(x, device="cuda"), prec).cpu().numpy()
    off = 0
    for d, r in zip(doms, nrhs):
        K = O.matrix_IminusN(d.et, d.etp, d.A, d.n)
        for k in range(r):
            xs = x[off:off + d.N]
            scale = (np.abs(K) @ np.abs(xs)).max()
            tol = (4 * 8 * (64 + d.N) * 2.0 ** -24 if prec == 2 else 1e-11) * scale
            assert np.abs(y[off:off + d.N] - K @ xs).max() <= tol
            off += d.N


def test_batch_fmm_matches_oracle(G):
    """GNK_PREC_FMM: every domain by the single-domain FBIE path with FMM
    products (the two domains of >= 4096 nodes) or double-float direct sums
    (the small ones), on concurrent worker streams; system by system against
    the oracle to the bounds of the single-domain solves."""
    doms, nrhs, gam = _batch_case(seed=5)
    rng = np.random.default_rng(3)
    for cnt, n in ((5, 1024), (9, 512)):
        d = Dm.build_domain(Dm.random_ellipses(rng, cnt, 2.2), n, bounded=False)
        doms.append(d)
        nrhs.append(2)
        gam = np.concatenate([gam, Dm.gamma_log(d, d.holes[0]), Dm.gamma_log(d, d.holes[1])])
    assert sum(d.N >= 4096 for d in doms) == 2
    with G.Batch(doms, nrhs, autotune=False, device="cuda") as b:
        g = torch.as_tensor(gam, device="cuda")
        mu, h, hk, res, rel = b.fbie(g, tol=1e-12, restart=30, precision=G.GNK_PREC_FMM, timing=1)
        assert res.status == 0 and rel.max() <= 1e-12 and res.solve_ms > 0
        mu2, _, _, res2, _ = b.fbie(g, tol=1e-12, restart=30, precision=G.GNK_PREC_FMM)  # handles reused
        mu, h, hk, mu2 = mu.cpu().numpy(), h.cpu().numpy(), hk.cpu().numpy(), mu2.cpu().numpy()
    assert np.array_equal(mu, mu2)
    off, koff = 0, 0
    for d, r in zip(doms, nrhs):
        for k in range(r):
            g_ = gam[off:off + d.N]
            mu_r, h_r, hk_r = O.fbie(d.et, d.etp, d.A, d.n, g_)
            assert np.abs(mu[off:off + d.N] - mu_r).max() <= 1e-10 * np.abs(mu_r).max()
            hs = max(1.0, np.abs(h_r).max())
            assert np.abs(h[off:off + d.N] - h_r).max() <= 1e-10 * hs
            assert np.abs(hk[koff:koff + d.m1] - hk_r).max() <= 1e-10 * hs
            off += d.N
            koff += d.m1
