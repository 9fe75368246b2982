"""Device memory of handles, solves and temporaries comes from a stream-ordered
pool that keeps freed memory: building, solving with and freeing a handle every
step must not grow the device's memory use after the first step, and work
ordered across streams (a handle built on one stream and used on another after
the caller synchronises) must give the same result as on one stream."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1308_5351_gb300 import domains as Dm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_1308_5351_gb300 import build, gnk
    build.build()
    gnk.load()
    return gnk


def _fbie_step(G, d, gam, stream_build, stream_solve, precision):
    et, etp, A = (torch.as_tensor(a, device="cuda") for a in (d.et, d.etp, d.A))
    mu = torch.empty_like(gam)
    h = torch.empty_like(gam)
    hk = torch.empty(d.m1, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    hnd = G.gnk_build_boundary_ex(d.m1, d.n, et, etp, A, None, None, d.bounded,
                                  precision | G.GNK_BUILD_DEFER, stream_build)
    stream_build.synchronize()
    opts = G.options(tol=1e-12, restart=20, maxit=50, precision=precision)
    res = G.gnk_fbie(hnd, gam, mu, h, hk, opts, stream_solve)
    stream_solve.synchronize()
    G.gnk_free_boundary(hnd)
    return mu.cpu().numpy(), hk.cpu().numpy(), res


@pytest.mark.parametrize("precision", ["fmm", "fp64"])
def test_repeated_steps_do_not_grow_memory(G, precision):
    p = G.GNK_PREC_FMM if precision == "fmm" else G.GNK_PREC_FP64
    d = Dm.ellipses64(n=128)  # N = 8192
    gam = torch.as_tensor(Dm.gamma_log(d, d.holes[0]), device="cuda")
    s = torch.cuda.current_stream()
    free = []
    for _ in range(6):
        _, _, res = _fbie_step(G, d, gam, s, s, p)
        assert res.status == 0
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
    # after the first steps the pool serves every allocation from memory it keeps
    assert max(free[2:]) - min(free[2:]) <= 64 << 20, [f >> 20 for f in free]


def test_build_and_solve_on_different_streams(G):
    d = Dm.ellipses64(n=128)
    gam = torch.as_tensor(Dm.gamma_log(d, d.holes[0]), device="cuda")
    s0 = torch.cuda.current_stream()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    mu_a, hk_a, ra = _fbie_step(G, d, gam, s0, s0, G.GNK_PREC_FMM)
    mu_b, hk_b, rb = _fbie_step(G, d, gam, s1, s2, G.GNK_PREC_FMM)
    assert ra.status == 0 and rb.status == 0
    assert np.array_equal(mu_a, mu_b) and np.array_equal(hk_a, hk_b)  # fixed summation order
