"""gnk_cauchy_sum_noalloc: the Cauchy sum for callers that cannot allocate
device memory (graph capture, host frameworks that own the memory pool,
latency-critical loops).  Its output must match gnk_cauchy_sum's on two calls
in a row, within the tolerance the parity tests use for FP64 Cauchy sums:
|z - z_ref|_i <= (64 + N) u S_i, S_i = sum_j |w_j / (eta_i - eta_j)|.
This file is collected last so that a failure here comes after every other
test has run."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

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
def test_noalloc_matches_cauchy_sum_twice(G, seed, count, n):
    d, w = _case(seed, count, n)
    et = torch.as_tensor(d.et, device="cuda")
    wd = torch.as_tensor(w, device="cuda")
    with G.Boundary.from_domain(d, adjoint=False, device="cuda") as b:
        z_ref = b.cauchy_sum(wd).cpu().numpy()
    S = np.array([np.sum(np.abs(w) / np.where(np.arange(d.N) == i, np.inf,
                                                np.abs(d.et[i] - d.et))) for i in range(d.N)])
    tol = (64 + d.N) * U64 * S
    for _ in range(2):  # the shared scratch keeps the previous call's contents
        z = torch.full_like(wd, complex("nan"))
        G.gnk_cauchy_sum_noalloc(d.N, et, wd, z)
        torch.cuda.synchronize()
        got = z.cpu().numpy()
        assert np.all(np.abs(got - z_ref) <= tol)


def test_noalloc_rejects_oversize_and_host_arrays(G):
    big = 65537
    et = torch.zeros(big, dtype=torch.complex128, device="cuda")
    with pytest.raises(G.GnkError) as e:
        G.gnk_cauchy_sum_noalloc(big, et, et, et)
    assert e.value.code == G.GNK_EINVAL and "65536" in str(e.value)
    h = np.zeros(16, dtype=np.complex128)
    with pytest.raises(G.GnkError) as e:
        G.gnk_cauchy_sum_noalloc(16, h, h, h)
    assert e.value.code == G.GNK_EINVAL
