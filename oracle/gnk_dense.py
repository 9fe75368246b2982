"""Dense FP64 CPU oracle for the Nystrom discretisation of the boundary integral
equations with the generalized Neumann kernel.

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously correct
reference that the CUDA library is checked against.  Only the test-suite, the
package smoke check and the benchmark's CPU-baseline leg may import it; the
library itself never does.  It shares no code with the CUDA path: every matrix
is assembled entry by entry from the paper's definitions and every linear
system is solved by LU (numpy/LAPACK gesv).

Paper sections followed (Nasser, "Fast solution of boundary integral equations
with the generalized Neumann kernel"):
  * kernels N, M, N(t,t), M1(t,t)          Sec. 2.2, Eqs. (N), (M), (N-tt), (M1-tt)
  * Cauchy matrix E                        Sec. 2.5, Eq. (fmm-E)
  * Nystrom matrix B, system               Sec. 3.2, Eqs. (B), (sys)
  * D, Wittich-derived circulant L, y      Sec. 3.3, Eqs. (phi-kp2), (y)
  * h                                      Sec. 3.6, Eq. (bh)
  * adjoint: e, B^T, P-hat, system         Sec. 4, Eqs. (ei2), (bve), (sys*)
  * Neumann kernel N_k and N_g(t,t)        Sec. 4.1, Eqs. (Nk), (Ng-tt)
  * variant without singularity subtraction Sec. 7 (Ex. 2), Eqs. (ie-sys), (phi-kp),
                                           (N-tt), (M1-tt)
  * Cauchy integral formula                Sec. 5, Eqs. (cauchy4), (cauchy6)
  * slit maps by the FBIE route            Sec. 7, Ex. 3 (map formulas of the
                                           method the paper cites; see slit_map)
  * slit maps by the adjoint route         Sec. 7, Ex. 3 and Ex. 4 (solves of
                                           Eq. (ie*) only; the steps are derived
                                           before slit_map_adjoint)

Readings of the paper taken here (each is listed with its reason in the design
notes of the repository):
  * The row-sum diagonal of the second-kind system is (2I + diag(B 1) - B), Eq. (sys).
  * At a corner node of a graded mesh eta'(t) = 0; the diagonal term
    Im(eta''/eta' - A'/A) takes its one-sided limit, which is 0 for a polygon
    (eta''/eta' is real along a straight edge and A'/A -> 0).
  * h is returned as the full node vector of Eq. (bh); h_k is its mean on
    component k.
  * Without singularity subtraction, M keeps Wittich's rule for its cotangent
    part (the method of Eq. (phi-kp) applied to gamma itself), and at a corner
    node both parts of eta''/eta' take the value 0, as in the diagonal above.

Parity: every function here is pinned by tests/test_oracle_pins.py against
closed forms (disk, unit circle), manufactured analytic solutions, the
eigen-identities of Eq. (NM-const), and adaptive quadrature of the continuous
operators; the slit maps by tests/test_slit_map.py and
tests/test_slit_map_adjoint.py (closed forms, the two routes against each
other, analyticity of the boundary values).
"""
from __future__ import annotations

import math

import numpy as np

_ROW_BLOCK = 1024


def _sizes(et, n):
    N = int(np.asarray(et).shape[0])
    if n <= 0 or n % 2 or N % n:
        raise ValueError("need n even and len(eta) a multiple of n")
    return N, N // n


# ---------------------------------------------------------------------------
# Sec. 2.5: the Cauchy matrix E, (E)_ij = 1/(eta_i - eta_j), i != j; 0 on i == j
# ---------------------------------------------------------------------------

def cauchy_matrix(et):
    """Dense E of Eq. (fmm-E)."""
    et = np.asarray(et, dtype=np.complex128)
    N = et.shape[0]
    E = np.zeros((N, N), dtype=np.complex128)
    for r0 in range(0, N, _ROW_BLOCK):
        r1 = min(N, r0 + _ROW_BLOCK)
        d = et[r0:r1, None] - et[None, :]
        idx = np.arange(r0, r1)
        d[idx - r0, idx] = 1.0
        blk = 1.0 / d
        blk[idx - r0, idx] = 0.0
        E[r0:r1] = blk
    return E


def cauchy_rows(et, x, rows):
    """(E x)_i = sum_{j != i} x_j / (eta_i - eta_j) for the listed rows, one row at
    a time (used to check sampled outputs at sizes where E does not fit)."""
    et = np.asarray(et, dtype=np.complex128)
    x = np.asarray(x, dtype=np.complex128)
    out = np.empty(len(rows), dtype=np.complex128)
    for k, i in enumerate(rows):
        d = et[i] - et
        d[i] = 1.0
        terms = x / d
        terms[i] = 0.0
        out[k] = terms.sum()
    return out


# ---------------------------------------------------------------------------
# Sec. 2.2 / 3.2 / 3.3: the Nystrom blocks of N and M
# ---------------------------------------------------------------------------

def nystrom_block(et, etp, A, n, rows, cols):
    """K_ij = (2 pi / n) [M(t_i, t_j) + i N(t_i, t_j)] for i in rows, j in cols, i.e.

        K_ij = (2/n) * A(t_i)/A(t_j) * eta'(t_j) / (eta(t_j) - eta(t_i)),

    with K_ij = 0 where i == j.  Then B = Im K (Eq. B) and D = Re K
    (the matrix D of Sec. 3.3), since (2 pi/n)(1/pi) = 2/n.
    """
    et = np.asarray(et, dtype=np.complex128)
    etp = np.asarray(etp, dtype=np.complex128)
    A = np.asarray(A, dtype=np.complex128)
    rows = np.asarray(rows)
    cols = np.asarray(cols)
    S = et[rows][:, None]
    T = et[cols][None, :]
    same = rows[:, None] == cols[None, :]
    diff = np.where(same, 1.0, T - S)
    K = (A[rows][:, None] / A[cols][None, :]) * etp[cols][None, :] / diff
    K = np.where(same, 0.0, K) * (2.0 / n)
    return K


def matrices_BD(et, etp, A, n):
    """Dense B (Eq. B) and D (Sec. 3.3)."""
    N, _ = _sizes(et, n)
    B = np.empty((N, N))
    D = np.empty((N, N))
    allc = np.arange(N)
    for r0 in range(0, N, _ROW_BLOCK):
        r1 = min(N, r0 + _ROW_BLOCK)
        K = nystrom_block(et, etp, A, n, np.arange(r0, r1), allc)
        B[r0:r1] = K.imag
        D[r0:r1] = K.real
    return B, D


def circulant_L(n):
    """L of Sec. 3.3: L_pq = (-1)^(p-q) (1/n) cot((p-q) pi / n), p != q; 0 on p == q."""
    if n % 2:
        raise ValueError("n must be even")
    p = np.arange(n)
    d = p[:, None] - p[None, :]
    with np.errstate(divide="ignore"):
        L = np.where(d == 0, 0.0,
                     np.where(d % 2 == 0, 1.0, -1.0) / n / np.tan(d * math.pi / n))
    L[d == 0] = 0.0
    return L


def block_L(n, m1):
    """L-hat = diag(L, ..., L) with m+1 blocks (Sec. 3.3)."""
    return np.kron(np.eye(m1), circulant_L(n))


def _IminusN_from_B(B):
    """2I + diag(B 1) - B formed in the storage of B (entries as written:
    -B_ij off the diagonal, 2 + sum_j B_ij on it, since B_ii = 0)."""
    s = B.sum(axis=1)
    K = np.negative(B, out=B)
    idx = np.arange(K.shape[0])
    K[idx, idx] += 2.0 + s
    return K


def _M_from_D(D, n, m1):
    """D - diag(D 1) + L-hat formed in the storage of D: L is added on each
    diagonal block (L-hat is block diagonal), then D 1 is taken off the
    diagonal (D_ii = L_pp = 0)."""
    s = D.sum(axis=1)
    L = circulant_L(n)
    for k in range(m1):
        blk = slice(k * n, (k + 1) * n)
        D[blk, blk] += L
    idx = np.arange(D.shape[0])
    D[idx, idx] -= s
    return D


def matrix_IminusN(et, etp, A, n):
    """2I + diag(B 1) - B: the discretisation of I - N with singularity
    subtraction (Eqs. ie-sys2, sys)."""
    B, _ = matrices_BD(et, etp, A, n)
    return _IminusN_from_B(B)


def matrix_M(et, etp, A, n):
    """D - diag(D 1) + L-hat: the discretisation of M (Eq. y, using L-hat 1 = 0)."""
    N, m1 = _sizes(et, n)
    _, D = matrices_BD(et, etp, A, n)
    return _M_from_D(D, n, m1)


def matrices_K_M(et, etp, A, n):
    """(2I + diag(B1) - B, D - diag(D1) + L-hat) from one assembly of B and D."""
    N, m1 = _sizes(et, n)
    B, D = matrices_BD(et, etp, A, n)
    return _IminusN_from_B(B), _M_from_D(D, n, m1)


def rhs_y(et, etp, A, n, gam):
    """y = phi(t) = D gamma - diag(D 1) gamma + L-hat gamma (Eq. y)."""
    return matrix_M(et, etp, A, n) @ np.asarray(gam, dtype=np.float64)


def solve_ie(et, etp, A, n, gam):
    """mu solving (2I + diag(B1) - B) mu = -y (Eq. sys), by LU."""
    K, Mm = matrices_K_M(et, etp, A, n)
    y = Mm @ np.asarray(gam, dtype=np.float64)
    return np.linalg.solve(K, -y)


def compute_h(et, etp, A, n, mu, gam):
    """h(t) = ([D - diag(D1) + L-hat] mu - [2I + diag(B1) - B] gamma) / 2 (Eq. bh).

    Returns (h at the nodes, h_k = mean of h over component k)."""
    N, m1 = _sizes(et, n)
    K, Mm = matrices_K_M(et, etp, A, n)
    h = (Mm @ mu - K @ gam) / 2.0
    return h, h.reshape(m1, n).mean(axis=1)


def fbie(et, etp, A, n, gam):
    """The triple (mu, h, h_k) of Sec. 3 computed densely, with one assembly
    of the two matrices and one LU.  gam is one right-hand side (N) or
    several as the columns of an N x R array; mu and h then have the same
    shape and h_k is m1 x R."""
    N, m1 = _sizes(et, n)
    K, Mm = matrices_K_M(et, etp, A, n)
    gam = np.asarray(gam, dtype=np.float64)
    mu = np.linalg.solve(K, -(Mm @ gam))
    h = (Mm @ mu - K @ gam) / 2.0
    return mu, h, h.reshape((m1, n) + h.shape[1:]).mean(axis=1)


# ---------------------------------------------------------------------------
# Sec. 2.2: diagonal limits of the kernels (used by the pins and by the
# variant without singularity subtraction)
# ---------------------------------------------------------------------------

def _ratio_limit(num, den):
    """num/den with the corner convention 0/0 := 0 (graded-mesh corner nodes)."""
    num = np.asarray(num, dtype=np.complex128)
    den = np.asarray(den, dtype=np.complex128)
    out = np.zeros_like(num)
    nz = den != 0
    out[nz] = num[nz] / den[nz]
    return out


def kernel_N_diag(etp, etpp, A, Ap):
    """N(t,t) = (1/pi) (1/2 Im eta''/eta' - Im A'/A)  (Eq. N-tt)."""
    return (0.5 * _ratio_limit(etpp, etp).imag - _ratio_limit(Ap, A).imag) / math.pi


def kernel_M1_diag(etp, etpp, A, Ap):
    """M1(t,t) = (1/pi) (1/2 Re eta''/eta' - Re A'/A)  (Eq. M1-tt)."""
    return (0.5 * _ratio_limit(etpp, etp).real - _ratio_limit(Ap, A).real) / math.pi


# ---------------------------------------------------------------------------
# Sec. 4: the adjoint equation (I + N* + J) mu = gamma
# ---------------------------------------------------------------------------

def adjoint_e(et, etp, etpp, A, Ap, n, c):
    """e_i = 1 - c + (2 pi/n) sum_{j != i} N_k(t_i, t_j) + (2 pi/n) N_g(t_i, t_i)
    (Eq. ei2) with the Neumann kernel N_k(s,t) = (1/pi) Im[eta'(t)/(eta(t)-eta(s))]
    (Eq. Nk) and N_g(t,t) = (1/pi) Im[eta''/eta' - A'/A] (Eq. Ng-tt)."""
    N, _ = _sizes(et, n)
    ones = np.ones(N, dtype=np.complex128)
    allc = np.arange(N)
    rowsum = np.empty(N)
    for r0 in range(0, N, _ROW_BLOCK):
        r1 = min(N, r0 + _ROW_BLOCK)
        # nystrom_block with A == 1 is (2/n) eta'_j/(eta_j - eta_i): (2pi/n) pi N_k / pi
        K = nystrom_block(et, etp, ones, n, np.arange(r0, r1), allc)
        rowsum[r0:r1] = K.imag.sum(axis=1)
    ng = (2.0 / n) * (_ratio_limit(etpp, etp) - _ratio_limit(Ap, A)).imag
    return 1.0 - c + rowsum + ng


def matrix_adjoint(et, etp, etpp, A, Ap, n, c):
    """diag(e) + B^T + P-hat (Eq. sys*), P-hat = diag(P,...,P), P = (1/n) 1 1^T,
    formed in one N x N array: B^T, then 1/n on each diagonal block (P-hat
    is block diagonal), then e on the diagonal (B_ii = 0)."""
    N, m1 = _sizes(et, n)
    B, _ = matrices_BD(et, etp, A, n)
    e = adjoint_e(et, etp, etpp, A, Ap, n, c)
    Ad = np.ascontiguousarray(B.T)
    del B
    for k in range(m1):
        blk = slice(k * n, (k + 1) * n)
        Ad[blk, blk] += 1.0 / n
    idx = np.arange(N)
    Ad[idx, idx] += e
    return Ad


def solve_adjoint_ie(et, etp, etpp, A, Ap, n, c, gam):
    """mu solving (diag(e) + B^T + P-hat) mu = gamma (Eq. sys*), by LU."""
    return np.linalg.solve(matrix_adjoint(et, etp, etpp, A, Ap, n, c),
                           np.asarray(gam, dtype=np.float64))


# ---------------------------------------------------------------------------
# Sec. 7, Ex. 2 comparison: the same Nystrom method without singularity
# subtraction.  The kernels keep their diagonal values (Eqs. N-tt, M1-tt)
# instead of the row-sum terms of Eqs. (ie-m), (ie-phi).
# ---------------------------------------------------------------------------

def matrix_IminusN_plain(et, etp, etpp, A, Ap, n):
    """I - N by the trapezoidal rule with N(t_i, t_i) of Eq. (N-tt) on the
    diagonal: (I - N)_ij = delta_ij - (2 pi/n) N(t_i, t_j)."""
    B, _ = matrices_BD(et, etp, A, n)
    Nd = (2.0 * math.pi / n) * kernel_N_diag(etp, etpp, A, Ap)
    return np.eye(B.shape[0]) - B - np.diag(Nd)


def matrix_M_plain(et, etp, etpp, A, Ap, n):
    """M discretised term by term as in Eq. (phi-kp) but applied to gamma itself
    (no gamma(s) subtracted): on the block of a component, Wittich's matrix -K
    for the cotangent part plus the trapezoidal rule for M_1 of Eq. (M-M1),
    with M_1(t, t) of Eq. (M1-tt) on the diagonal; off the block the
    trapezoidal rule for M."""
    N, m1 = _sizes(et, n)
    _, D = matrices_BD(et, etp, A, n)      # D_ij = (2 pi/n) M(t_i, t_j), i != j
    p = np.arange(n)
    d = p[:, None] - p[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        cot = np.where(d == 0, 0.0, 1.0 / np.tan(d * math.pi / n))
    wittich = np.where(d % 2 != 0, (2.0 / n) * cot, 0.0)        # K_pq
    M1d = (2.0 * math.pi / n) * kernel_M1_diag(etp, etpp, A, Ap)
    out = D.copy()
    for k in range(m1):
        blk = slice(k * n, (k + 1) * n)
        # (2 pi/n) M1(s_p, s_q) = (2 pi/n) M(s_p, s_q) + (1/n) cot((p - q) pi / n), p != q
        m1_blk = D[blk, blk] + cot / n
        out[blk, blk] = -wittich + m1_blk + np.diag(M1d[blk])
    return out


def fbie_plain(et, etp, etpp, A, Ap, n, gam):
    """mu of (I - N) mu = -M gamma and h = (M mu - (I - N) gamma)/2 with the
    plain matrices above, by LU.  Returns (mu, h, h_k)."""
    N, m1 = _sizes(et, n)
    K = matrix_IminusN_plain(et, etp, etpp, A, Ap, n)
    M = matrix_M_plain(et, etp, etpp, A, Ap, n)
    gam = np.asarray(gam, dtype=np.float64)
    mu = np.linalg.solve(K, -(M @ gam))
    h = (M @ mu - K @ gam) / 2.0
    return mu, h, h.reshape(m1, n).mean(axis=1)


def matrix_adjoint_plain(et, etp, etpp, A, Ap, n):
    """I + N* + J by the trapezoidal rule: N*(s, t) = N(t, s) (Eq. Nt-N*), so the
    off-diagonal part is B^T and the diagonal is N(t, t) (Eq. N-tt); J gives
    P-hat."""
    N, m1 = _sizes(et, n)
    B, _ = matrices_BD(et, etp, A, n)
    Nd = (2.0 * math.pi / n) * kernel_N_diag(etp, etpp, A, Ap)
    P = np.kron(np.eye(m1), np.full((n, n), 1.0 / n))
    return np.eye(N) + np.diag(Nd) + B.T + P


def solve_adjoint_plain(et, etp, etpp, A, Ap, n, gam):
    """mu solving (I + N* + J) mu = gamma with the plain matrix, by LU."""
    return np.linalg.solve(matrix_adjoint_plain(et, etp, etpp, A, Ap, n),
                           np.asarray(gam, dtype=np.float64))


# ---------------------------------------------------------------------------
# Row-wise forms for sampled checks at sizes where dense matrices do not fit
# ---------------------------------------------------------------------------

def rows_IminusN(et, etp, A, n, x, rows):
    """Rows of (2I + diag(B1) - B) x (Eq. sys), one block of rows at a time."""
    N, _ = _sizes(et, n)
    rows = np.asarray(rows)
    K = nystrom_block(et, etp, A, n, rows, np.arange(N))
    B = K.imag
    x = np.asarray(x, dtype=np.float64)
    return 2.0 * x[rows] + B.sum(axis=1) * x[rows] - B @ x


def rows_M(et, etp, A, n, x, rows):
    """Rows of (D - diag(D1) + L-hat) x (Eq. y)."""
    N, _ = _sizes(et, n)
    rows = np.asarray(rows)
    K = nystrom_block(et, etp, A, n, rows, np.arange(N))
    D = K.real
    x = np.asarray(x, dtype=np.float64)
    L = circulant_L(n)
    out = D @ x - D.sum(axis=1) * x[rows]
    for k, i in enumerate(rows):
        comp, p = divmod(int(i), n)
        out[k] += L[p] @ x[comp * n:(comp + 1) * n]
    return out


def rows_adjoint(et, etp, etpp, A, Ap, n, c, x, rows):
    """Rows of (diag(e) + B^T + P-hat) x (Eq. sys*)."""
    N, _ = _sizes(et, n)
    rows = np.asarray(rows)
    x = np.asarray(x, dtype=np.float64)
    allr = np.arange(N)
    # (B^T)_{ij} = B_{ji}: the columns `rows` of B
    BT = nystrom_block(et, etp, A, n, allr, rows).imag.T
    ones = np.ones(N, dtype=np.complex128)
    Kk = nystrom_block(et, etp, ones, n, rows, allr).imag
    ng = (2.0 / n) * (_ratio_limit(np.asarray(etpp)[rows], np.asarray(etp)[rows])
                      - _ratio_limit(np.asarray(Ap)[rows], np.asarray(A)[rows])).imag
    e = 1.0 - c + Kk.sum(axis=1) + ng
    comp = rows // n
    means = x.reshape(-1, n).mean(axis=1)
    return e * x[rows] + BT @ x + means[comp]


# ---------------------------------------------------------------------------
# Gradient of a loss L(mu, h) of the FBIE outputs (dense adjoint)
# ---------------------------------------------------------------------------

def fbie_gradient(et, etp, A, n, gam, g_mu, g_h):
    """dL/d(eta, eta', A, gamma) for a loss with dL/dmu = g_mu and dL/dh = g_h,
    where mu solves K mu = -M gamma and h = (M mu - K gamma)/2 with
    K = 2I + diag(B1) - B, M = D - diag(D1) + L-hat (Eqs. sys, y, bh).

    Dense adjoint: lambda = K^-T (g_mu + M^T g_h / 2) by LU; the geometry enters
    through Z_ij = A_i eta'_j / (A_j (eta_j - eta_i)) (i != j), B = (2/n) Im Z,
    D = (2/n) Re Z, and the loss varies with the geometry as
      S = sum_{i != j} WB_ij B_ij + WD_ij D_ij,
      WB_ij = -g_h,i (gam_i - gam_j)/2 - lambda_i (mu_i - mu_j),
      WD_ij =  g_h,i (mu_j - mu_i)/2 - lambda_i (gam_j - gam_i),
    differentiated entry by entry.  Complex gradients are packed as
    dL/dRe + i dL/dIm.  Returns (g_et, g_etp, g_A, g_gam, mu, h)."""
    et = np.asarray(et, dtype=np.complex128)
    etp = np.asarray(etp, dtype=np.complex128)
    A = np.asarray(A, dtype=np.complex128)
    gam = np.asarray(gam, dtype=np.float64)
    g_mu = np.asarray(g_mu, dtype=np.float64)
    g_h = np.asarray(g_h, dtype=np.float64)
    N, m1 = _sizes(et, n)
    K = matrix_IminusN(et, etp, A, n)
    M = matrix_M(et, etp, A, n)
    mu = np.linalg.solve(K, -(M @ gam))
    h = (M @ mu - K @ gam) / 2.0
    lam = np.linalg.solve(K.T, g_mu + 0.5 * (M.T @ g_h))
    # entries and their holomorphic derivatives
    diff = et[None, :] - et[:, None]            # eta_j - eta_i
    off = ~np.eye(N, dtype=bool)
    dsafe = np.where(off, diff, 1.0)
    Z = np.where(off, (A[:, None] / A[None, :]) * etp[None, :] / dsafe, 0.0)
    Y = np.where(off, (A[:, None] / A[None, :]) / dsafe, 0.0)          # dZ_ij / d eta'_j
    WB = -0.5 * g_h[:, None] * (gam[:, None] - gam[None, :]) - lam[:, None] * (mu[:, None] - mu[None, :])
    WD = 0.5 * g_h[:, None] * (mu[None, :] - mu[:, None]) - lam[:, None] * (gam[None, :] - gam[:, None])
    C = np.where(off, (2.0 / n) * (WD - 1j * WB), 0.0)                # S = Re sum C_ij Z_ij
    R = C * Z / dsafe                                                # d/d eta_i of C_ij Z_ij
    d_et = R.sum(axis=1) - R.sum(axis=0)
    d_etp = (C * Y).sum(axis=0)
    CZ = C * Z
    d_A = (CZ.sum(axis=1) - CZ.sum(axis=0)) / A
    g_gam = -0.5 * (K.T @ g_h) - M.T @ lam
    return np.conj(d_et), np.conj(d_etp), np.conj(d_A), g_gam, mu, h


# ---------------------------------------------------------------------------
# Sec. 5: the Cauchy integral formula with singularity subtraction
# ---------------------------------------------------------------------------

def cauchy_formula(et, etp, n, f_nodes, z, bounded, finf=0.0):
    """f(z) from its boundary values by the ratio forms of Eq. (cauchy4):
    bounded G:   f(z) = sum_j f_j eta'_j/(eta_j - z) / sum_j eta'_j/(eta_j - z),
    unbounded G: f(z) = (f_inf + (1/(n i)) sum_j f_j eta'_j/(eta_j - z))
                        / (1 + (1/(n i)) sum_j eta'_j/(eta_j - z)).
    Direct sums over all nodes for each point z (z off the boundary)."""
    et = np.asarray(et, dtype=np.complex128)
    etp = np.asarray(etp, dtype=np.complex128)
    f_nodes = np.asarray(f_nodes, dtype=np.complex128)
    z = np.atleast_1d(np.asarray(z, dtype=np.complex128))
    out = np.empty(z.shape, dtype=np.complex128)
    for k, zk in enumerate(z):
        c = etp / (et - zk)
        s1 = np.sum(f_nodes * c)
        s2 = np.sum(c)
        if bounded:
            out[k] = s1 / s2
        else:
            out[k] = (finf + s1 / (n * 1j)) / (1.0 + s2 / (n * 1j))
    return out


# ---------------------------------------------------------------------------
# Sec. 7, Ex. 3 and Ex. 4: conformal maps onto slit domains by the FBIE route:
# one solve of Eq. (ie) and h of Eq. (h), with theta = pi/2 on a boundary that
# becomes a circular slit and theta = 0 on one that becomes a radial slit.
# The map formulas are the method the paper cites for these examples (its
# references, not restated in the paper); with gamma =
# -Re[e^{i(pi/2 - theta)} log(eta - alpha)] (arg continuous along each
# boundary) and the analytic f with boundary values A f = gamma + h + i mu:
#   bounded G (Ex. 3), A = e^{i(pi/2 - theta)} (eta - alpha), alpha in G:
#     w(z) = e^{-h_0} (z - alpha) exp((z - alpha) f(z))
#     onto the unit disk (|w| = 1 on the outer boundary) with circular slits
#     |w| = e^{h_j - h_0} and radial slits, w(alpha) = 0, w'(alpha) > 0;
#   unbounded G (Ex. 4), A = e^{i(pi/2 - theta)} (Eq. A), f(inf) = 0, alpha in G:
#     w(z) = (z - alpha) exp(f(z))
#     onto the plane with circular slits |w| = e^{h_j} and radial slits
#     arg w = -h_j, w(alpha) = 0 and w(z) = z + O(1) at infinity.
# ---------------------------------------------------------------------------

def slit_map_data(et, n, alpha, theta, bounded=True):
    """A and gamma of the slit map for theta given per boundary component."""
    et = np.asarray(et, dtype=np.complex128)
    N, m1 = _sizes(et, n)
    th = np.repeat(np.asarray(theta, dtype=np.float64), n)
    rot = np.exp(1j * (math.pi / 2 - th))
    lg = np.empty(N, dtype=np.complex128)
    for k in range(m1):
        d = et[k * n:(k + 1) * n] - alpha
        lg[k * n:(k + 1) * n] = np.log(np.abs(d)) + 1j * np.unwrap(np.angle(d))
    A = rot * (et - alpha) if bounded else rot.astype(np.complex128)
    gam = -(rot * lg).real
    return A, gam


def slit_map(et, etp, n, alpha, theta, z=None, bounded=True):
    """Boundary values w(eta) of the slit map, the constant c (e^{-h_0} for
    bounded G, 1 for unbounded G), the per-component h_k, and (if z is given)
    w at the points z of G by the Cauchy formula of Eq. (cauchy4) applied to f
    (with f(inf) = 0 for unbounded G)."""
    et = np.asarray(et, dtype=np.complex128)
    N, m1 = _sizes(et, n)
    A, gam = slit_map_data(et, n, alpha, theta, bounded)
    mu, h, hk = fbie(et, etp, A, n, gam)
    fb = (gam + h + 1j * mu) / A
    wz = None
    if bounded:
        c = math.exp(-hk[0])
        w = c * (et - alpha) * np.exp((et - alpha) * fb)
    else:
        c = 1.0
        w = (et - alpha) * np.exp(fb)
    if z is not None:
        z = np.asarray(z, dtype=np.complex128)
        fz = cauchy_formula(et, etp, n, fb, z, bounded)
        wz = c * (z - alpha) * np.exp((z - alpha) * fz) if bounded else (z - alpha) * np.exp(fz)
    return w, c, hk, wz


# ---------------------------------------------------------------------------
# Sec. 7, Ex. 3 and Ex. 4: the same slit maps by the route of the adjoint
# equation (the paper's FBIEad comparison): only solves of Eq. (ie*), then the
# boundary correspondence integrated per boundary by the FFT.  The paper gives
# the route's cost and count of solves but not its formulas (they are in its
# references); the steps below are derived here from the kernel identities of
# Sec. 2.2 and Cauchy's theorem:
#
# With A of Eq. (A) for the slit map and A~ = eta'/A (Eq. A*), the kernel
# formed with A~ is -N* (Eq. Nt-N*).  For g analytic in G (bounded G; for
# unbounded G with g(inf) = 0) write A~ g = a + i b on the boundary; Plemelj's
# formula gives (I - N~) b = -M~ a, i.e. (I + N*) b = M* a.  For a function q
# analytic in the holes and vanishing at infinity the sign of N~ flips:
# (I + N~) b_q = M~ a_q.
#
# Write the map as w(z) = (z - alpha) exp(omega(z)), omega analytic in G
# (omega(inf) = 0 for unbounded G).  On a circular-slit boundary (theta = pi/2)
# w(eta(t)) = R_k exp(i th_k(t)), so eta' w'/w = i th_k'(t); on a radial-slit
# boundary (theta = 0) w(eta(t)) = rho_k(t) exp(i phi_k), so eta' w'/w = (log
# rho_k)'(t).  Hence, with psi = th' (circular) and psi = -(log rho)' (radial),
#   bounded G:   H = (z - alpha) w'/w is analytic, H(alpha) = 1 and A~ H = i psi,
#                so (I + N*) psi = 0; the winding of w along the boundaries
#                gives J psi = (1, 0, ..., 0), so (I + N* + J) psi = e_0;
#   unbounded G: w'/w = 1/(z - alpha) + omega' splits into a part analytic in
#                G with value 0 at infinity and one analytic in the holes, and
#                the two identities above give (I + N*) psi =
#                2 Im[A~/(eta - alpha)]; every boundary is a slit, J psi = 0.
# This is the one solve for the derivative of the boundary correspondence.
# Its antiderivative along each boundary (zero at t = 0) is S(t): th_k =
# th_k(0) + S and log rho_k = c_k - S.
#
# The parameters: the solutions psi_j of (I + N* + J) psi_j = e_j (j = 0..m)
# lie in the null space of I + N* (J psi_j = e_j) and belong to analytic g_j
# with A~ g_j = i psi_j; eta' g_j/(eta - alpha) (bounded) or eta' g_j
# (unbounded) is i psi_j on a circular boundary and -psi_j on a radial one.
# Cauchy's theorem for omega times that function gives, with
#   T_j = (1/(2 pi)) int_Gamma c(t) omega^(t) psi_j(t) dt,   c = i (circular),
#         c = -1 (radial), omega^ = omega without its per-boundary constants
#         (circular: -log|eta - alpha| + i (S - arg(eta - alpha));
#          radial:   -S - log|eta - alpha| - i arg(eta - alpha)),
# and rho = log w'(alpha) = Im T_0 for bounded G (w'(alpha) > 0, R_0 = 1),
# rho = 0 for unbounded G:
#   circular k:  log R_k = rho - Im T_k,   th_k(0) = Re T_k;
#   radial k:    c_k = rho + Re T_k,       phi_k = Im T_k.
# (The residue of g_j/(z - alpha) at alpha is 1 for a circular j and i for a
# radial j, which gives these two forms.)  Bounded G needs m + 1 solves
# (psi_0 is also the derivative), unbounded G m + 2.
# ---------------------------------------------------------------------------

def periodic_antiderivative(psi, n):
    """S(t_p) = int_0^{t_p} psi(t) dt on each boundary component for the
    trigonometric interpolant of psi at the n nodes: the mean times t plus the
    periodic part whose DFT coefficients are those of psi divided by i k
    (k = 0 and the n/2 mode, whose antiderivative vanishes at the nodes,
    dropped), shifted so that S(0) = 0."""
    P = np.asarray(psi, dtype=np.float64).reshape(-1, n)
    t = np.arange(n) * (2.0 * math.pi / n)
    C = np.fft.fft(P, axis=1)
    k = np.fft.fftfreq(n, d=1.0 / n)
    mean = C[:, 0].real / n
    div = np.where(k == 0, 1.0, 1j * k)
    Q = C / div
    Q[:, 0] = 0.0
    Q[:, n // 2] = 0.0
    per = np.fft.ifft(Q, axis=1).real
    return (mean[:, None] * t[None, :] + per - per[:, :1]).ravel()


def slit_map_adjoint(et, etp, etpp, n, alpha, theta, bounded=True, z=None):
    """The slit map of slit_map by solves of Eq. (ie*) only (the derivation
    above).  Returns (w at the nodes, psi, params, scale, omega at the nodes,
    w at z or None): psi is th' on circular and -(log rho)' on radial
    boundaries; params[k] is R_k (circular) or phi_k (radial); scale is
    w'(alpha) for bounded G and 1 for unbounded G."""
    et = np.asarray(et, dtype=np.complex128)
    etp = np.asarray(etp, dtype=np.complex128)
    N, m1 = _sizes(et, n)
    theta = np.asarray(theta, dtype=np.float64)
    circ_k = theta == math.pi / 2
    if not np.all(circ_k | (theta == 0.0)) or (bounded and not circ_k[0]):
        raise ValueError("theta must be pi/2 or 0 per boundary (pi/2 on the outer one of bounded G)")
    A, _ = slit_map_data(et, n, alpha, theta, bounded)
    rot = np.repeat(np.exp(1j * (math.pi / 2 - theta)), n)
    Ap = rot * etp if bounded else np.zeros(N, dtype=np.complex128)
    c = 1 if bounded else -1
    Mad = matrix_adjoint(et, etp, etpp, A, Ap, n, c)
    comp = np.repeat(np.arange(m1), n)
    # psi_j: (I + N* + J) psi_j = e_j (Eq. sys*), j = 0..m
    psis = [np.linalg.solve(Mad, (comp == j).astype(np.float64)) for j in range(m1)]
    if bounded:
        psi = psis[0]
    else:
        At = etp / A
        psi = np.linalg.solve(Mad, 2.0 * (At / (et - alpha)).imag)
    S = periodic_antiderivative(psi, n)
    # log(eta - alpha) with arg continuous along each boundary
    lg = np.empty(N, dtype=np.complex128)
    for k in range(m1):
        d = et[k * n:(k + 1) * n] - alpha
        lg[k * n:(k + 1) * n] = np.log(np.abs(d)) + 1j * np.unwrap(np.angle(d))
    circ = np.repeat(circ_k, n)
    om_hat = np.where(circ, -lg.real + 1j * (S - lg.imag), -S - lg.real - 1j * lg.imag)
    cw = np.where(circ, 1j, -1.0)
    T = np.array([np.sum(cw * om_hat * p) / n for p in psis])  # (1/2pi)(2pi/n) sum
    rho = T[0].imag if bounded else 0.0
    params = np.empty(m1)
    kappa = np.empty(m1, dtype=np.complex128)
    w = np.empty(N, dtype=np.complex128)
    for k in range(m1):
        s = slice(k * n, (k + 1) * n)
        if circ_k[k]:
            logR, th0 = rho - T[k].imag, T[k].real
            params[k] = math.exp(logR)
            kappa[k] = logR + 1j * th0
            w[s] = params[k] * np.exp(1j * (th0 + S[s]))
        else:
            ck, phik = rho + T[k].real, T[k].imag
            params[k] = phik
            kappa[k] = ck + 1j * phik
            w[s] = np.exp(ck - S[s]) * np.exp(1j * phik)
    omega = om_hat + np.repeat(kappa, n)
    wz = None
    if z is not None:
        z = np.asarray(z, dtype=np.complex128)
        oz = cauchy_formula(et, etp, n, omega, z, bounded)
        wz = (z - alpha) * np.exp(oz)
    return w, psi, params, (math.exp(rho) if bounded else 1.0), omega, wz
