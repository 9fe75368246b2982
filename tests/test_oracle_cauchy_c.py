"""Pins for the oracle's all-core C Cauchy sum (oracle/cauchy_omp.c), which
the benchmark times for the host's pair-evaluation rate (Sec. 2.5, Eq. fmm-E):

  * roots of unity: for eta_j = exp(2 pi i j / n) and w = 1,
    sum_{j != i} 1 / (eta_i - eta_j) = (n - 1) / (2 eta_i)  (closed form);
  * the same nodes with w_j = eta_j, through the identity
    eta_j / (eta_i - eta_j) = eta_i / (eta_i - eta_j) - 1;
  * brute force: the dense Cauchy matrix of gnk_dense times w on ellipses,
    within (64 + N) u S_i;
  * the result does not depend on the thread count (each row summed in order).
"""
import numpy as np
import pytest

from oracle import cauchy_cpu as C
from oracle import gnk_dense as O
from paper_1308_5351_gb300 import domains as Dm

U = 2.0 ** -53


def test_roots_of_unity_closed_form():
    for n in (2, 7, 64, 1000):
        eta = np.exp(2j * np.pi * np.arange(n) / n)
        z = C.cauchy_sum(eta, np.ones(n, dtype=np.complex128), threads=2)
        assert np.abs(z - (n - 1) / (2 * eta)).max() <= 1e-12 * n


def test_weights_eta_identity():
    n = 96
    eta = np.exp(2j * np.pi * np.arange(n) / n)
    z1 = C.cauchy_sum(eta, np.ones(n, dtype=np.complex128))
    z = C.cauchy_sum(eta, eta)
    # sum_{j != i} eta_j/(eta_i - eta_j) = eta_i sum_{j != i} 1/(eta_i - eta_j) - (n - 1)
    assert np.abs(z - (eta * z1 - (n - 1))).max() <= 1e-11


@pytest.mark.parametrize("threads", [1, 3])
def test_against_dense_cauchy_matrix(threads):
    rng = np.random.default_rng(12)
    d = Dm.build_domain(Dm.random_ellipses(rng, 4, 1.5), 150, bounded=False)
    w = rng.normal(size=d.N) + 1j * rng.normal(size=d.N)
    ref = O.cauchy_matrix(d.et) @ w
    S = np.array([np.sum(np.abs(w) / np.where(np.arange(d.N) == i, np.inf, np.abs(d.et[i] - d.et)))
                  for i in range(d.N)])
    z = C.cauchy_sum(d.et, w, threads=threads)
    assert np.all(np.abs(z - ref) <= (64 + d.N) * U * S)


def test_thread_count_does_not_change_the_result():
    rng = np.random.default_rng(3)
    et = rng.normal(size=777) + 1j * rng.normal(size=777)
    w = rng.normal(size=777) + 1j * rng.normal(size=777)
    assert np.array_equal(C.cauchy_sum(et, w, threads=1), C.cauchy_sum(et, w, threads=5))
