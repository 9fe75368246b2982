"""Arnoldi cycles longer than one warp of Givens rotations (Sec. 3.5, Eq.
ie-gmres): with restart 64 on 384 curves of the close-curves domain at
n = 32 (gaps down to 1e-3 r: GMRES needs 44 steps) the previous rotations of
a column are applied by the serial loop instead of the warp scan, in the
FP64 step and in the double-float step.  mu and h must match the dense oracle's
solution to 1e-10 (GMRES to 1e-13), and the solve must really have taken
more than 33 steps in one cycle.
"""
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


@pytest.fixture(scope="module")
def case():
    full = Dm.close_curves(3, 32)
    d = Dm.build_domain(full.curves[:384], 32, bounded=False)  # N = 12,288
    gam = Dm.gamma_log(d, full.holes[0])
    return d, gam, O.fbie(d.et, d.etp, d.A, d.n, gam)


@pytest.mark.parametrize("prec", ["fp64", "fmm"])
def test_long_cycle_matches_oracle(G, case, prec):
    d, gam, (mu_ref, h_ref, hk_ref) = case
    p = {"fp64": G.GNK_PREC_FP64, "fmm": G.GNK_PREC_FMM}[prec]
    with G.Boundary.from_domain(d, adjoint=False, device="cuda", precision=p) as b:
        mu, h, hk, res = b.fbie(torch.as_tensor(gam, device="cuda"), tol=1e-13, precision=p, restart=64, maxit=10)
    assert res.status == 0, res.as_dict()
    assert res.iterations > 33 and res.cycles == 1, res.as_dict()
    mu, h = mu.cpu().numpy(), h.cpu().numpy()
    assert np.abs(mu - mu_ref).max() <= 1e-10 * np.abs(mu_ref).max()
    assert np.abs(h - h_ref).max() <= 1e-10 * max(1.0, np.abs(h_ref).max())


@pytest.fixture(scope="module")
def wide():
    full = Dm.close_curves(3, 32)
    d = Dm.build_domain(full.curves, 32, bounded=False)  # 1024 curves, N = 32,768
    gam = Dm.gamma_log(d, full.holes[0])
    return d, gam, O.fbie(d.et, d.etp, d.A, d.n, gam)


@pytest.mark.parametrize("prec", ["fp64", "fmm"])
def test_partial_sums_read_in_place(G, wide, prec):
    """With 128 Arnoldi blocks (N = 32,768, one block per 256 nodes) the
    blocks' partial sums of a step beyond j = 30 no longer fit the staging
    area (128 (j + 2) > 4096 entries) and are added where they lie: the solve
    must still match the oracle."""
    d, gam, (mu_ref, h_ref, _) = wide
    p = {"fp64": G.GNK_PREC_FP64, "fmm": G.GNK_PREC_FMM}[prec]
    with G.Boundary.from_domain(d, adjoint=False, device="cuda", precision=p) as b:
        mu, h, hk, res = b.fbie(torch.as_tensor(gam, device="cuda"), tol=1e-13, precision=p, restart=64, maxit=10)
    assert res.status == 0, res.as_dict()
    assert res.iterations > 33 and res.cycles == 1, res.as_dict()
    mu, h = mu.cpu().numpy(), h.cpu().numpy()
    assert np.abs(mu - mu_ref).max() <= 1e-10 * np.abs(mu_ref).max()
    assert np.abs(h - h_ref).max() <= 1e-10 * max(1.0, np.abs(h_ref).max())
