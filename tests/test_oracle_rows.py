"""Pins for the oracle's row-wise forms, which check the full-size GPU solves
one sampled row at a time (Sec. 3, Eqs. sys and y; Sec. 4, Eq. sys*).

  * rows_IminusN, rows_M and rows_adjoint against the dense matrices
    (2I + diag(B1) - B), (D - diag(D1) + L-hat) and (diag(e) + B^T + P-hat)
    times x, which are pinned by closed forms and quadrature in
    test_oracle_pins: rows in the first, a middle and the last component
    (and both ends of each), on a bounded domain with non-constant A and on an
    unbounded one, to 1e-13 of |matrix| |x|;
  * the same row forms directly against the unit circle's closed forms with
    A = eta (Sec. 3.3, 4.2): (I - N) x = x + mean(x), M cos kt = -sin kt,
    M sin kt = cos kt for k < n/2, the adjoint matrix is the identity;
  * planted mistakes in the row forms (the component of a row taken modulo
    the number of components, a dropped row-sum term, B in place of B^T in
    the adjoint, the component mean taken over the wrong block) make the pins
    fail.
"""
import math

import numpy as np
import pytest

from oracle import gnk_dense as O
from paper_1308_5351_gb300 import domains as Dm


def _bounded():
    # non-constant A (theta differs per boundary) and curves of unequal shape
    return Dm.ex2_circles(0.1, 24, theta=[math.pi / 2, 0, math.pi / 2, 0, math.pi / 2])


def _unbounded():
    rng = np.random.default_rng(7)
    return Dm.build_domain(Dm.random_ellipses(rng, 4, 1.5), 20, bounded=False)


def _rows(d):
    n, m1 = d.n, d.m1
    mid = m1 // 2
    rows = [0, 1, n - 1, mid * n, mid * n + n // 2, mid * n + n - 1, (m1 - 1) * n, d.N - 1]
    rng = np.random.default_rng(d.N)
    rows += list(rng.choice(d.N, size=6, replace=False))
    return np.array(sorted(set(int(r) for r in rows)))


def _x(d, seed=3):
    return np.random.default_rng(seed).normal(size=d.N)


def _close(got, dense, x, rows, tol=1e-13):
    scale = (np.abs(dense) @ np.abs(x))[rows]
    return bool(np.all(np.abs(got - (dense @ x)[rows]) <= tol * scale))


# ------------------------------------------------------------------ checks (return bool)
def _check_dense(d):
    x = _x(d)
    rows = _rows(d)
    K, M = O.matrices_K_M(d.et, d.etp, d.A, d.n)
    Ad = O.matrix_adjoint(d.et, d.etp, d.etpp, d.A, d.Ap, d.n, d.c)
    return (_close(O.rows_IminusN(d.et, d.etp, d.A, d.n, x, rows), K, x, rows),
            _close(O.rows_M(d.et, d.etp, d.A, d.n, x, rows), M, x, rows),
            _close(O.rows_adjoint(d.et, d.etp, d.etpp, d.A, d.Ap, d.n, d.c, x, rows), Ad, x, rows))


def _check_unit_circle():
    n = 32
    d = Dm.disk(n, 0j)
    t = Dm.nodes(n)
    rows = np.arange(n)
    x = _x(d)
    ok = [np.abs(O.rows_IminusN(d.et, d.etp, d.A, n, x, rows) - (x + x.mean())).max() < 1e-14]
    for k in (1, 5, n // 2 - 1):
        ok.append(np.abs(O.rows_M(d.et, d.etp, d.A, n, np.cos(k * t), rows) + np.sin(k * t)).max() < 1e-13)
        ok.append(np.abs(O.rows_M(d.et, d.etp, d.A, n, np.sin(k * t), rows) - np.cos(k * t)).max() < 1e-13)
    ok.append(np.abs(O.rows_adjoint(d.et, d.etp, d.etpp, d.A, d.Ap, n, 1, x, rows) - x).max() < 1e-14)
    return all(ok)


def _all_pass():
    return (all(_check_dense(_bounded())) and all(_check_dense(_unbounded()))
            and _check_unit_circle())


# ------------------------------------------------------------------ tests
@pytest.mark.parametrize("make", [_bounded, _unbounded], ids=["bounded_theta", "unbounded"])
def test_rows_match_dense_matrices(make):
    d = make()
    assert d.m1 >= 3
    ok_in, ok_m, ok_adj = _check_dense(d)
    assert ok_in, "rows_IminusN"
    assert ok_m, "rows_M"
    assert ok_adj, "rows_adjoint"


def test_rows_unit_circle_closed_forms():
    assert _check_unit_circle()


# ------------------------------------------------------------------ planted mistakes
def _rows_M_wrong_component(et, etp, A, n, x, rows):
    """rows_M with the component of row i taken as i mod (m+1)."""
    N, m1 = O._sizes(et, n)
    rows = np.asarray(rows)
    D = O.nystrom_block(et, etp, A, n, rows, np.arange(N)).real
    x = np.asarray(x, dtype=np.float64)
    L = O.circulant_L(n)
    out = D @ x - D.sum(axis=1) * x[rows]
    for k, i in enumerate(rows):
        comp, p = int(i) % m1, int(i) % n
        out[k] += L[p] @ x[comp * n:(comp + 1) * n]
    return out


def _rows_M_no_rowsum(et, etp, A, n, x, rows):
    """rows_M without the diag(D1) term."""
    N, _ = O._sizes(et, n)
    rows = np.asarray(rows)
    D = O.nystrom_block(et, etp, A, n, rows, np.arange(N)).real
    x = np.asarray(x, dtype=np.float64)
    L = O.circulant_L(n)
    out = D @ x
    for k, i in enumerate(rows):
        comp, p = divmod(int(i), n)
        out[k] += L[p] @ x[comp * n:(comp + 1) * n]
    return out


def _rows_IminusN_no_rowsum(et, etp, A, n, x, rows):
    """rows_IminusN without the diag(B1) term."""
    N, _ = O._sizes(et, n)
    rows = np.asarray(rows)
    B = O.nystrom_block(et, etp, A, n, rows, np.arange(N)).imag
    x = np.asarray(x, dtype=np.float64)
    return 2.0 * x[rows] - B @ x


def _rows_adjoint_not_transposed(et, etp, etpp, A, Ap, n, c, x, rows):
    """rows_adjoint with the rows of B in place of the rows of B^T."""
    N, _ = O._sizes(et, n)
    rows = np.asarray(rows)
    x = np.asarray(x, dtype=np.float64)
    allr = np.arange(N)
    B = O.nystrom_block(et, etp, A, n, rows, allr).imag
    ones = np.ones(N, dtype=np.complex128)
    Kk = O.nystrom_block(et, etp, ones, n, rows, allr).imag
    ng = (2.0 / n) * (O._ratio_limit(np.asarray(etpp)[rows], np.asarray(etp)[rows])
                      - O._ratio_limit(np.asarray(Ap)[rows], np.asarray(A)[rows])).imag
    e = 1.0 - c + Kk.sum(axis=1) + ng
    means = x.reshape(-1, n).mean(axis=1)
    return e * x[rows] + B @ x + means[rows // n]


def _rows_adjoint_mean_of_block0(et, etp, etpp, A, Ap, n, c, x, rows):
    """rows_adjoint with P-hat x taken as the mean of the first component."""
    good = ORIG["rows_adjoint"](et, etp, etpp, A, Ap, n, c, x, rows)
    x = np.asarray(x, dtype=np.float64)
    means = x.reshape(-1, n).mean(axis=1)
    return good - means[np.asarray(rows) // n] + means[0]


ORIG = {"rows_adjoint": O.rows_adjoint}


@pytest.mark.parametrize("name,mutant", [
    ("rows_M", _rows_M_wrong_component),
    ("rows_M", _rows_M_no_rowsum),
    ("rows_IminusN", _rows_IminusN_no_rowsum),
    ("rows_adjoint", _rows_adjoint_not_transposed),
    ("rows_adjoint", _rows_adjoint_mean_of_block0),
], ids=["M_component_mod", "M_no_rowsum", "IminusN_no_rowsum", "adjoint_B_not_BT", "adjoint_mean_block0"])
def test_planted_mistakes_in_row_forms_are_caught(monkeypatch, name, mutant):
    assert _all_pass()
    monkeypatch.setattr(O, name, mutant)
    assert not _all_pass(), name
    monkeypatch.undo()
    assert _all_pass()
