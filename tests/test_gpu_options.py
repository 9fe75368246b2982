"""The per-call controls of gnk_options that are not arithmetic: phase times
and tile overrides, read back through the C ABI.

* timing = 1: gnk_fbie reports setup, right-hand side, GMRES and h phase
  times (CUDA events); each is positive and their sum is at most the call's
  wall time.  gnk_solve_ie reports its three phases; gnk_batch_fbie the
  whole call as its solve time.
* tile_chunks (direct pair kernels) and tile_variant (batched kernels) change
  how the sums are split, not what they are: mu and h match the dense
  oracle for each override (FP64, double-float and mixed precision), and the
  batch reports the overridden shape while the call runs with it.
* Out-of-range overrides are rejected before any launch.
"""
import time

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
    rng = np.random.default_rng(31)
    d = Dm.build_domain(Dm.random_ellipses(rng, 6, 1.8), 512, bounded=False)  # N = 3072
    gam = Dm.gamma_log(d, d.holes[0])
    return d, gam, O.fbie(d.et, d.etp, d.A, d.n, gam)


def _close(mu, h, ref):
    mu_ref, h_ref, _ = ref
    return (np.abs(mu - mu_ref).max() <= 1e-10 * np.abs(mu_ref).max()
            and np.abs(h - h_ref).max() <= 1e-10 * max(1.0, np.abs(h_ref).max()))


@pytest.mark.parametrize("prec", ["fp64", "fmm"])
def test_fbie_phase_times(G, case, prec):
    d, gam, ref = case
    p = {"fp64": G.GNK_PREC_FP64, "fmm": G.GNK_PREC_FMM}[prec]
    g = torch.as_tensor(gam, device="cuda")
    with G.Boundary.from_domain(d, adjoint=False, device="cuda", precision=p | G.GNK_BUILD_DEFER) as b:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mu, h, hk, res = b.fbie(g, tol=1e-12, precision=p, timing=1)
        wall_ms = 1e3 * (time.perf_counter() - t0)
        assert res.status == 0
        phases = [res.setup_ms, res.rhs_ms, res.solve_ms, res.h_ms]
        assert all(t > 0.0 for t in phases), res.as_dict()
        assert sum(phases) <= wall_ms * 1.05 + 0.05
        assert res.solve_ms >= max(res.setup_ms, res.rhs_ms, res.h_ms)
        assert _close(mu.cpu().numpy(), h.cpu().numpy(), ref)
        mu2, res2 = b.solve_ie(g, tol=1e-12, precision=p, timing=1)
        assert res2.rhs_ms > 0.0 and res2.solve_ms > 0.0 and res2.h_ms == 0.0
        mu3, h3, hk3, res3 = b.fbie(g, tol=1e-12, precision=p)  # timing off
        assert res3.setup_ms == res3.rhs_ms == res3.solve_ms == res3.h_ms == 0.0


@pytest.mark.parametrize("prec,bprec", [(0, 0), (4, 3), (1, 0)], ids=["fp64", "mixed_df", "mixed"])
@pytest.mark.parametrize("chunks", [1, 3, 64])
def test_tile_chunks_override(G, case, prec, bprec, chunks):
    d, gam, ref = case
    g = torch.as_tensor(gam, device="cuda")
    with G.Boundary.from_domain(d, adjoint=False, device="cuda", precision=bprec) as b:
        mu, h, hk, res = b.fbie(g, tol=1e-12, precision=prec, tile_chunks=chunks)
        assert res.status == 0
        assert _close(mu.cpu().numpy(), h.cpu().numpy(), ref)


def test_bad_overrides_rejected(G, case):
    d, gam, _ = case
    g = torch.as_tensor(gam, device="cuda")
    with G.Boundary.from_domain(d, adjoint=False, device="cuda") as b:
        for kw in ({"tile_chunks": 65}, {"tile_chunks": -1}, {"tile_variant": 8}):
            with pytest.raises(G.GnkError) as e:
                b.fbie(g, **kw)
            assert e.value.code == G.GNK_EINVAL


def test_batch_tile_variant_override(G):
    rng = np.random.default_rng(8)
    doms = [Dm.build_domain(Dm.random_ellipses(rng, m, 1.5), n, bounded=False)
            for m, n in ((2, 128), (3, 64), (4, 96))]
    nrhs = [d.m1 for d in doms]
    gam = np.concatenate([Dm.gamma_log(d, d.holes[k]) for d in doms for k in range(d.m1)])
    refs = []
    for d in doms:
        G_ = np.stack([Dm.gamma_log(d, d.holes[k]) for k in range(d.m1)], axis=1)
        refs.append(O.fbie(d.et, d.etp, d.A, d.n, G_)[0])
    with G.Batch(doms, nrhs, autotune=False, device="cuda") as b:
        tuned = b.tuning()
        shapes32 = [(1, 8), (2, 4), (2, 8), (4, 4)]
        shapesdf = [(1, 2), (1, 4), (2, 2)]
        for v in range(0, 8):
            mu, h, hk, res, rel = b.fbie(torch.as_tensor(gam, device="cuda"), tol=1e-10, tile_variant=v,
                                         timing=1)
            assert res.status == 0 and res.solve_ms > 0.0
            t = b.tuning()
            if 1 <= v <= 4:
                assert (t["fp32_targets"], t["fp32_group"]) == shapes32[v - 1]
            elif v >= 5:
                assert (t["df_targets"], t["df_group"]) == shapesdf[v - 5]
            else:
                assert t["fp32_targets"] == tuned["fp32_targets"] and t["df_group"] == tuned["df_group"]
            mu = mu.cpu().numpy()
            off = 0
            for d, r, mo in zip(doms, nrhs, refs):
                got = mu[off:off + d.N * r].reshape(r, d.N).T
                assert np.abs(got - mo).max() <= 1e-9 * np.abs(mo).max(), v
                off += d.N * r
