"""Failure paths and hand-written arithmetic that can be tested on the GPU
without a fault.

* The bounded grid-barrier waits of the cooperative Arnoldi step (Sec. 3.5):
  with the test hook one block never arrives, the other blocks' waits run out
  after a short limit, and the solve returns GNK_ECUDA with the timed-out
  message, in FP64 and in the mixed-precision refinement (whose inner FP32
  solve carries the failure).  The device stays usable: the next solve with
  the hook cleared matches the oracle.
* The FP64 reciprocal of the pair kernels, rcp.approx seed refined by the
  series y0 (1 + e + e^2) with e = 1 - x y0, against CUDA's IEEE division
  1.0 / x over the range of |d|^2 the kernels meet (1e-14 at graded corners
  to 1e4) and beyond: at most 1 ulp apart, and the distribution of the
  differences is recorded in the test's output.
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
def dom():
    rng = np.random.default_rng(21)
    return Dm.build_domain(Dm.random_ellipses(rng, 5, 1.6), 512, bounded=False)  # N = 2560: 10 blocks


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_arnoldi_barrier_timeout_is_reported(G, dom, prec):
    d = dom
    p = {"fp64": G.GNK_PREC_FP64, "mixed": G.GNK_PREC_MIXED}[prec]
    gam = Dm.gamma_log(d, d.holes[0])
    mu_ref, _, _ = O.fbie(d.et, d.etp, d.A, d.n, gam)
    g = torch.as_tensor(gam, device="cuda")
    with G.Boundary.from_domain(d, adjoint=False, device="cuda") as b:
        try:
            G.gnk_debug_barrier_fault(1, 4096)
            with pytest.raises(G.GnkError) as e:
                b.solve_ie(g, tol=1e-12, precision=p)
            assert e.value.code == G.GNK_ECUDA
            assert "timed out" in str(e.value)
        finally:
            G.gnk_debug_barrier_fault(-1, 0)
        torch.cuda.synchronize()  # the context is intact
        mu, res = b.solve_ie(g, tol=1e-12, precision=p)
        assert res.status == 0
        mu = mu.cpu().numpy()
    assert np.abs(mu - mu_ref).max() <= 1e-10 * np.abs(mu_ref).max()


def test_barrier_hook_rejects_bad_arguments(G):
    with pytest.raises(G.GnkError):
        G.gnk_debug_barrier_fault(-2, 0)
    with pytest.raises(G.GnkError):
        G.gnk_debug_barrier_fault(0, -1)
    G.gnk_debug_barrier_fault(-1, 0)


def _ulps(a, b):
    """Distance in units in the last place between two arrays of positive doubles."""
    ia = a.view(np.int64)
    ib = b.view(np.int64)
    return np.abs(ia - ib)


def test_recip_f64_against_cuda_division(G):
    rng = np.random.default_rng(5)
    # |d|^2 of the pair kernels: from ~1e-14 (graded corners) to ~1e4, and wider
    lo, hi = -20.0, 20.0
    x = 10.0 ** rng.uniform(lo, hi, size=1 << 20)
    x = np.concatenate([x, 2.0 ** np.arange(-60, 61, dtype=np.float64),
                        np.nextafter(2.0 ** np.arange(-60, 61, dtype=np.float64), 0.0)])
    xd = torch.as_tensor(x, device="cuda")
    y_lib = torch.empty_like(xd)
    y_div = torch.empty_like(xd)
    G.gnk_debug_recip_f64(xd, y_lib, y_div)
    torch.cuda.synchronize()
    y_lib, y_div = y_lib.cpu().numpy(), y_div.cpu().numpy()
    assert np.array_equal(y_div, 1.0 / x)  # CUDA's division is correctly rounded, like the host's
    u = _ulps(y_lib, y_div)
    counts = {int(k): int((u == k).sum()) for k in np.unique(u)}
    print(f"recip_f64 vs 1.0/x over 1e{lo:.0f}..1e{hi:.0f}: ulp distance counts {counts}")
    assert u.max() <= 1
    rel = np.abs(y_lib * x - 1.0)
    assert rel.max() <= 2.0 ** -51


def _trunc24(x):
    """x truncated toward zero to 24 significant bits (clears the low 29 bits
    of the binary64 significand): the definition of the split's high part."""
    b = x.view(np.uint64) & ~np.uint64((1 << 29) - 1)
    return b.view(np.float64)


def test_split_f64_bit_level_against_definition(G):
    """The FMM kernels' double-float split from the bits of x: in its range
    (2^-80 <= |x| < 2^101) hi is x truncated to 24 significant bits (exact as a
    float) and |x - (hi + lo)| < 2^-46 |x|; elsewhere (0, tiny, huge, Inf, NaN)
    it is the conversion split (float(x), float(x - float(x)))."""
    rng = np.random.default_rng(9)
    x = np.concatenate([
        rng.choice([-1.0, 1.0], 1 << 18) * 10.0 ** rng.uniform(-24, 30, 1 << 18),
        np.array([0.0, -0.0, 2.0 ** -80, -(2.0 ** -80), np.nextafter(2.0 ** -80, 0.0), 2.0 ** 101,
                  np.nextafter(2.0 ** 101, 0.0), 1e-300, -1e300, 5e-324, np.inf, -np.inf, np.nan, 1.0, -1.0,
                  1.0 + 2.0 ** -52, 3.0 - 2.0 ** -51]),
    ])
    xd = torch.as_tensor(x, device="cuda")
    hi = torch.empty(x.size, dtype=torch.float32, device="cuda")
    lo = torch.empty_like(hi)
    G.gnk_debug_split_f64(xd, hi, lo)
    torch.cuda.synchronize()
    hi, lo = hi.cpu().numpy().astype(np.float64), lo.cpu().numpy().astype(np.float64)
    ax = np.abs(x)
    fast = (ax >= 2.0 ** -80) & (ax < 2.0 ** 101)
    assert np.array_equal(hi[fast], _trunc24(x[fast]))
    err = np.abs(x[fast] - (hi[fast] + lo[fast]))  # exact: hi + lo spans < 53 bits
    assert (err <= 2.0 ** -46 * ax[fast]).all(), err.max()
    assert (np.sign(lo[fast]) * np.sign(x[fast]) >= 0).all()
    slow = ~fast & np.isfinite(x)
    f = x[slow].astype(np.float32).astype(np.float64)
    assert np.array_equal(hi[slow], f)
    assert np.array_equal(lo[slow], (x[slow] - f).astype(np.float32).astype(np.float64))
    nonfin = ~np.isfinite(x)
    assert np.array_equal(np.isnan(hi[nonfin]), np.isnan(x[nonfin]))
