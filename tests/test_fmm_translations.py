"""CPU pins of the translation algebra the FMM kernels use (Sec. 2.5; the
complex-analytic 2-D FMM with expansions scaled by the box width r):

  multipole  phi(z) = sum_k a_k r^k / (z - c)^(k+1),  a_k = sum_j w_j ((s_j - c)/r)^k
  local      phi(z) = sum_l b_l ((z - c)/r)^l

The kernels do not tabulate a P x P matrix per relative box position:
  * M2M and L2L between a box and a child in quadrant q = 2 qa + qb (child
    centre c1 = c0 + delta r0, delta = g/4, g = (2 qa - 1) + i (2 qb - 1)) are
    the real Pascal sums C(m,k) (M2M: P - 1 passes of one neighbour addition
    per lane) and C(l,m) (L2L: a table [l][m], zero outside the triangle,
    summed by lane m) between scalings by powers of g and conj(g);
  * M2L is the fixed Pascal matrix C(k+l, l) between two complex scalings.
These tests emulate those steps in numpy (FP64) and compare them with the
matrix forms and with expansions formed directly from point sources, so a
wrong sign, index, quadrant or scaling in the factorisation fails here.
"""
import math

import numpy as np
import pytest

P = 32


def _g(q):
    qa, qb = q >> 1, q & 1
    return complex(2 * qa - 1, 2 * qb - 1)


def _gauss_angle(q):
    # the kernels' table: angle of g in units of pi/4
    return {3: 1, 1: 3, 0: 5, 2: 7}[q]


def _gpow(ang, e, s):
    """g^e 2^s for g = sqrt(2) e^{i pi ang / 4}: 2^floor(e/2) (c + i d), c, d in {0, +-1}."""
    a8 = (ang * e) & 7
    m = math.ldexp(1.0, (e >> 1) + s)
    gr = m if a8 in (0, 1, 7) else (-m if a8 in (3, 4, 5) else 0.0)
    gi = m if a8 in (1, 2, 3) else (-m if a8 in (5, 6, 7) else 0.0)
    return complex(gr, gi)


def _table_up():
    """The kernels' L2L Pascal table: BU[l][m] = C(l, m) for l >= m, zero elsewhere."""
    return np.array([[math.comb(l, m) if l >= m else 0 for m in range(P)] for l in range(P)], dtype=float)


def _binom_lower(v):
    """lane m: sum_{k<=m} C(m,k) v_k, by the M2M passes (pass i adds the left
    neighbour's pre-pass value on lanes m >= i)."""
    v = np.array(v, dtype=complex)
    for i in range(1, P):
        u = np.concatenate([[0], v[:-1]])
        lanes = np.arange(P) >= i
        v = np.where(lanes, v + u, v)
    return v


def _binom_upper(v):
    """lane m: sum_l BU[l][m] v_l, the L2L Pascal-table sum over a staged vector."""
    T = _table_up()
    v = np.asarray(v, dtype=complex)
    return np.array([sum(T[l, m] * v[l] for l in range(P)) for m in range(P)])


def _m2m_binom(a1, q):
    ang = _gauss_angle(q)
    c = np.array([a1[k] * _gpow(8 - ang, k, 0) for k in range(P)])
    S = _binom_lower(c)
    return np.array([S[m] * _gpow(ang, m, -2 * m) for m in range(P)])


def _l2l_binom(b0, q):
    ang = _gauss_angle(q)
    e = np.array([b0[l] * _gpow(ang, l, -2 * l) for l in range(P)])
    T = _binom_upper(e)
    return np.array([T[m] * _gpow(8 - ang, m, 0) for m in range(P)])


def test_gaussian_powers_are_exact():
    for q in range(4):
        g = _g(q)
        for e in range(P + 1):
            assert _gpow(_gauss_angle(q), e, 0) == g ** e
            assert _gpow(8 - _gauss_angle(q), e, 0) == np.conj(g) ** e
            assert _gpow(_gauss_angle(q), e, -2 * e) == (g / 4) ** e


def test_pascal_table_is_exact_and_triangular():
    BU = _table_up()
    assert BU.max() < 2.0 ** 29  # C(31, 15): exact as a double-float pair
    assert np.array_equal(np.tril(BU), BU)


def test_passes_and_table_are_pascal_sums():
    rng = np.random.default_rng(0)
    v = rng.normal(size=P) + 1j * rng.normal(size=P)
    lo = np.array([sum(math.comb(m, k) * v[k] for k in range(m + 1)) for m in range(P)])
    up = np.array([sum(math.comb(l, m) * v[l] for l in range(m, P)) for m in range(P)])
    assert np.allclose(_binom_lower(v), lo, rtol=1e-13, atol=0)
    assert np.allclose(_binom_upper(v), up, rtol=1e-13, atol=0)


@pytest.mark.parametrize("q", range(4))
def test_m2m_pascal_matches_matrix_form_and_direct_multipole(q):
    """M2M of a child's multipole equals the parent multipole formed directly from
    the child's sources (r0 = width of the parent, r1 = r0/2)."""
    rng = np.random.default_rng(10 + q)
    c0, r0 = 0.3 - 0.2j, 0.8
    c1, r1 = c0 + _g(q) / 4 * r0, r0 / 2
    s = c1 + (rng.uniform(-0.5, 0.5, 40) + 1j * rng.uniform(-0.5, 0.5, 40)) * r1
    w = rng.normal(size=40) + 1j * rng.normal(size=40)
    a1 = np.array([np.sum(w * ((s - c1) / r1) ** k) for k in range(P)])
    a0 = np.array([np.sum(w * ((s - c0) / r0) ** k) for k in range(P)])
    d = (c1 - c0) / r0
    mat = np.array([sum(math.comb(m, k) * 2.0 ** -k * d ** (m - k) * a1[k] for k in range(m + 1))
                    for m in range(P)])
    got = _m2m_binom(a1, q)
    scale = np.abs(a0).max()
    assert np.abs(mat - a0).max() <= 1e-13 * scale
    assert np.abs(got - a0).max() <= 1e-13 * scale


@pytest.mark.parametrize("q", range(4))
def test_l2l_pascal_matches_matrix_form_and_direct_local(q):
    """L2L of a parent's local expansion (of far sources) equals the child's local
    expansion formed directly from those sources."""
    rng = np.random.default_rng(20 + q)
    c0, r0 = -0.1 + 0.4j, 0.5
    c1, r1 = c0 + _g(q) / 4 * r0, r0 / 2
    s = c0 + (2.0 + rng.uniform(0, 1, 30)) * r0 * np.exp(2j * np.pi * rng.uniform(size=30))
    w = rng.normal(size=30) + 1j * rng.normal(size=30)

    def local(c, r):  # phi(z) = sum_j w_j/(z - s_j) = sum_l b_l ((z - c)/r)^l
        return np.array([np.sum(-w * r ** l / (s - c) ** (l + 1)) for l in range(P)])

    b0, b1 = local(c0, r0), local(c1, r1)
    d = (c1 - c0) / r0
    mat = np.array([sum(math.comb(l, m) * 2.0 ** -m * d ** (l - m) * b0[l] for l in range(m, P))
                    for m in range(P)])
    got = _l2l_binom(b0, q)
    # the truncation at P terms is the only difference from the direct local expansion
    scale = np.abs(b1).max()
    assert np.abs(got - mat).max() <= 1e-13 * scale
    assert np.abs(got - b1).max() <= 1e-9 * scale


@pytest.mark.parametrize("off", [(2, 0), (3, -2), (-3, 3), (0, -2), (-2, -3), (3, 3)])
def test_m2l_pascal_factorisation(off):
    """b_l = (1/r) delta^-l sum_k C(k+l, l) [(-1)^(k+1) delta^-(k+1) a_k], delta the
    source box centre minus the target box centre in box widths, against the
    matrix form and against the local expansion of the sources themselves."""
    rng = np.random.default_rng(100 + 7 * off[0] + off[1])
    r = 0.25
    cs, ct = 0.1 + 0.1j, 0.1 + 0.1j + complex(*off) * r  # source and target box centres
    s = cs + (rng.uniform(-0.5, 0.5, 50) + 1j * rng.uniform(-0.5, 0.5, 50)) * r
    w = rng.normal(size=50) + 1j * rng.normal(size=50)
    a = np.array([np.sum(w * ((s - cs) / r) ** k) for k in range(P)])
    d = (cs - ct) / r  # the offset code (dx, dy) is the source box's position relative to the target
    mat = np.array([sum((-1) ** (k + 1) * math.comb(k + l, l) * d ** (-(k + l + 1)) * a[k] for k in range(P))
                    for l in range(P)]) / r
    pre = np.array([(-1) ** (k + 1) * d ** (-(k + 1)) for k in range(P)])
    H = np.array([[math.comb(k + l, l) for k in range(P)] for l in range(P)], dtype=float)
    got = (d ** -np.arange(P)) * (H @ (pre * a)) / r
    direct = np.array([np.sum(-w * r ** l / (s - ct) ** (l + 1)) for l in range(P)])
    scale = np.abs(direct).max()
    assert np.abs(got - mat).max() <= 1e-13 * np.abs(mat).max()
    assert np.abs(got - direct).max() <= 1e-6 * scale  # truncation of the multipole at P terms


def test_planted_mistakes_fail():
    """A swapped quadrant, the unconjugated pre-scaling and a sign slip in M2L all fail."""
    rng = np.random.default_rng(7)
    a1 = rng.normal(size=P) + 1j * rng.normal(size=P)
    d = _g(3) / 4
    mat = np.array([sum(math.comb(m, k) * 2.0 ** -k * d ** (m - k) * a1[k] for k in range(m + 1))
                    for m in range(P)])
    assert np.abs(_m2m_binom(a1, 3) - mat).max() <= 1e-13 * np.abs(mat).max()
    assert np.abs(_m2m_binom(a1, 0) - mat).max() > 1e-3 * np.abs(mat).max()
    ang = _gauss_angle(3)
    c = np.array([a1[k] * _gpow(ang, k, 0) for k in range(P)])  # g^k instead of conj(g)^k
    wrong = np.array([_binom_lower(c)[m] * _gpow(ang, m, -2 * m) for m in range(P)])
    assert np.abs(wrong - mat).max() > 1e-3 * np.abs(mat).max()
    # the L2L table in place of the M2M table (a transposed Pascal matrix)
    c = np.array([a1[k] * _gpow(8 - ang, k, 0) for k in range(P)])
    wrong = np.array([_binom_upper(c)[m] * _gpow(ang, m, -2 * m) for m in range(P)])
    assert np.abs(wrong - mat).max() > 1e-3 * np.abs(mat).max()
    dd = 2.0 + 1.0j
    pre_wrong = np.array([(-1) ** k * dd ** (-(k + 1)) for k in range(P)])
    pre = -pre_wrong
    H = np.array([[math.comb(k + l, l) for k in range(P)] for l in range(P)], dtype=float)
    good = (dd ** -np.arange(P)) * (H @ (pre * a1))
    bad = (dd ** -np.arange(P)) * (H @ (pre_wrong * a1))
    assert np.abs(good - bad).max() > 1e-3 * np.abs(good).max()
