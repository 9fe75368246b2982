"""gnk_cauchy_sum_noalloc: the Cauchy sum for callers that cannot allocate
device memory (plugins inside a host application that owns all device
memory, real-time loops that cannot accept an allocation's implicit
synchronisation or its possible failure).  It keeps its partial sums in a
fixed array of the library's device image, shared by every call.

On two calls in a row (the second reads a scratch array that still holds the
first call's contents) its output must match
  * the oracle's dense Cauchy matrix times w, element by element, and
  * gnk_cauchy_sum, the entry point that allocates,
within the bound the parity tests use for FP64 Cauchy sums:
|z - z_ref|_i <= (64 + N) u S_i, S_i = sum_j |w_j / (eta_i - eta_j)|.
The device's free memory must not change across the second call.
This file is collected last so that a failure here comes after every other
test has run."""
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


def _case(seed, count, n):
    rng = np.random.default_rng(seed)
    d = Dm.build_domain(Dm.random_ellipses(rng, count, 2.0), n, bounded=False)
    w = rng.normal(size=d.N) + 1j * rng.normal(size=d.N)
    return d, w


@pytest.mark.parametrize("seed,count,n", [(1, 5, 512), (2, 3, 170), (3, 1, 8)])
def test_noalloc_matches_oracle_and_cauchy_sum_twice(G, seed, count, n):
    d, w = _case(seed, count, n)
    z_oracle = O.cauchy_matrix(d.et) @ w
    S = np.array([np.sum(np.abs(w) / np.where(np.arange(d.N) == i, np.inf,
                                                np.abs(d.et[i] - d.et))) for i in range(d.N)])
    tol = (64 + d.N) * U64 * S
    et = torch.as_tensor(d.et, device="cuda")
    wd = torch.as_tensor(w, device="cuda")
    with G.Boundary.from_domain(d, adjoint=False, device="cuda") as b:
        z_lib = b.cauchy_sum(wd).cpu().numpy()
    assert np.all(np.abs(z_lib - z_oracle) <= tol)
    outs = [torch.full_like(wd, complex("nan")) for _ in range(2)]
    torch.cuda.synchronize()
    G.gnk_cauchy_sum_noalloc(d.N, et, wd, outs[0])
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    G.gnk_cauchy_sum_noalloc(d.N, et, wd, outs[1])  # scratch still holds call 1's sums
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before
    for z in outs:
        got = z.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.all(np.abs(got - z_oracle) <= tol)
        assert np.all(np.abs(got - z_lib) <= tol)


def test_noalloc_rejects_oversize_short_and_host_arrays(G):
    big = 65537
    et = torch.zeros(big, dtype=torch.complex128, device="cuda")
    with pytest.raises(G.GnkError) as e:
        G.gnk_cauchy_sum_noalloc(big, et, et, et)
    assert e.value.code == G.GNK_EINVAL and "65536" in str(e.value)
    short = torch.zeros(15, dtype=torch.complex128, device="cuda")
    with pytest.raises(G.GnkError) as e:
        G.gnk_cauchy_sum_noalloc(16, et, short, et)
    assert e.value.code == G.GNK_EINVAL and "fewer than N" in str(e.value)
    h = np.zeros(16, dtype=np.complex128)
    with pytest.raises(G.GnkError) as e:
        G.gnk_cauchy_sum_noalloc(16, h, h, h)
    assert e.value.code == G.GNK_EINVAL
