"""Differentiation of the FBIE computation.

CPU: the oracle's dense adjoint gradient against central finite differences
of the oracle's forward (every input kind: eta, eta', A, gamma; bounded and
unbounded; a graded polygon).
GPU: gnk_fbie_backward against the oracle gradient, the transposed solve
against the oracle, and torch.autograd through Fourier coefficients of star
curves against central finite differences of the GPU forward.
Tolerances: finite differences with step 1e-6 carry ~1e-9 truncation and
rounding error on O(1) gradients; the GPU backward solves to 1e-12 and is
compared at 1e-8 relative to the largest gradient entry.
"""
import math

import numpy as np
import pytest

from oracle import gnk_dense as O
from paper_1308_5351_gb300 import domains as Dm


def _fd_check(d, gam, rng, entries, eps=1e-6):
    cm = rng.normal(size=d.N)
    ch = rng.normal(size=d.N)
    ge, gp, gA, gg, mu, h = O.fbie_gradient(d.et, d.etp, d.A, d.n, gam, cm, ch)

    def loss(et, etp, A, g):
        mu, h, _ = O.fbie(et, etp, A, d.n, g)
        return cm @ mu + ch @ h

    grads = {"et": ge, "etp": gp, "A": gA}
    scale = max(np.abs(ge).max(), np.abs(gp).max(), np.abs(gA).max(), np.abs(gg).max())
    for name in ("et", "etp", "A"):
        for m in entries:
            for dz in (1.0, 1j):
                args = {"et": d.et.copy(), "etp": d.etp.copy(), "A": d.A.copy()}
                args[name][m] += eps * dz
                Lp = loss(args["et"], args["etp"], args["A"], gam)
                args[name][m] -= 2 * eps * dz
                Lm = loss(args["et"], args["etp"], args["A"], gam)
                fd = (Lp - Lm) / (2 * eps)
                an = grads[name][m].real if dz == 1.0 else grads[name][m].imag
                assert abs(fd - an) <= 1e-7 * scale, (name, m, dz, fd, an)
    for m in entries:
        g = gam.copy()
        g[m] += eps
        Lp = loss(d.et, d.etp, d.A, g)
        g[m] -= 2 * eps
        Lm = loss(d.et, d.etp, d.A, g)
        assert abs((Lp - Lm) / (2 * eps) - gg[m]) <= 1e-7 * scale


def test_oracle_gradient_bounded_fd():
    d = Dm.three_circles(16)
    _fd_check(d, Dm.gamma_log(d, 0.05j), np.random.default_rng(0), [0, 7, 20, 40])


def test_oracle_gradient_unbounded_theta_fd():
    d = Dm.ex4_circles(0.2, 12, theta=[0.3, 1.1, -0.4, 2.0, 0.9])
    _fd_check(d, Dm.gamma_log(d, 0.0), np.random.default_rng(1), [1, 13, 30, 59])


def test_oracle_gradient_graded_fd():
    curves = [Dm.Circle(0j, 1.6, ccw=True), Dm.square(0.3 + 0.1j, 0.5, ccw=False)]
    d = Dm.build_domain(curves, 16, bounded=True, alpha=-1.2 + 0.3j)
    _fd_check(d, Dm.manufactured(d, Dm.f_bounded_ex1)[0], np.random.default_rng(2), [2, 16, 19, 27])


# ------------------------------------------------------------------ GPU
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def G():
    from paper_1308_5351_gb300 import build, gnk
    build.build()
    gnk.load()
    return gnk


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


@pytest.mark.gpu
@pytest.mark.parametrize("which", ["bounded", "unbounded_theta", "graded"])
@pytest.mark.parametrize("prec", [0, 1, 4, 5, 6])
def test_backward_matches_oracle(G, which, prec):
    rng = np.random.default_rng(5)
    if which == "bounded":
        d = Dm.three_circles(128)
        gam = Dm.gamma_log(d, 0.05j)
    elif which == "unbounded_theta":
        d = Dm.ex4_circles(0.2, 96, theta=[0.3, 1.1, -0.4, 2.0, 0.9])
        gam = Dm.gamma_log(d, 0.0)
    else:
        curves = [Dm.Circle(0j, 1.6, ccw=True), Dm.square(0.3 + 0.1j, 0.5, ccw=False)]
        d = Dm.build_domain(curves, 128, bounded=True, alpha=-1.2 + 0.3j)
        gam = Dm.manufactured(d, Dm.f_bounded_ex1)[0]
    cm = rng.normal(size=d.N)
    ch = rng.normal(size=d.N)
    ref = O.fbie_gradient(d.et, d.etp, d.A, d.n, gam, cm, ch)
    bprec = G.GNK_PREC_DF32 if prec == 4 else G.GNK_PREC_FP64
    if prec in (5, 6):  # the six Cauchy and six 1/d^2 sums by three FMM passes
        bprec = G.GNK_PREC_FMM
    with G.Boundary.from_domain(d, adjoint=False, device="cuda", precision=bprec) as b:
        mu, h, hk, res = b.fbie(_dev(gam), tol=1e-13, precision=prec)
        out = [torch.empty(d.N, dtype=torch.complex128, device="cuda") for _ in range(3)]
        g_gam = torch.empty(d.N, dtype=torch.float64, device="cuda")
        G.gnk_fbie_backward(b.handle, mu, _dev(gam), _dev(cm), _dev(ch), out[0], out[1], out[2], g_gam,
                            G.options(tol=1e-13, precision=prec))
    got = [o.cpu().numpy() for o in out] + [g_gam.cpu().numpy()]
    scale = max(np.abs(r).max() for r in ref[:4])
    for k in range(4):
        assert np.abs(got[k] - ref[k]).max() <= 1e-8 * scale, (which, prec, k)


@pytest.mark.gpu
def test_transpose_solve_matches_oracle(G):
    d = Dm.three_circles(128)
    rhs = np.random.default_rng(9).normal(size=d.N)
    K = O.matrix_IminusN(d.et, d.etp, d.A, d.n)
    ref = np.linalg.solve(K.T, rhs)
    with G.Boundary.from_domain(d, adjoint=False, device="cuda") as b:
        x = torch.empty(d.N, dtype=torch.float64, device="cuda")
        res = G.gnk_solve_ie_transpose(b.handle, _dev(rhs), x, G.options(tol=1e-13))
    assert res.status == 0
    assert np.abs(x.cpu().numpy() - ref).max() <= 1e-10 * np.abs(ref).max()


def _star_domain(coeffs, n, centres, r0, polygons):
    from paper_1308_5351_gb300 import autograd as AG
    ets, etps = [], []
    for c, (ak, bk) in zip(centres, coeffs):
        z, zp = AG.star_boundary(c, r0, ak, bk, n)
        ets.append(z)
        etps.append(zp)
    t = Dm.nodes(n)
    for poly in polygons:
        z, zp, _ = poly.eval(t)
        ets.append(torch.as_tensor(z, device="cuda"))
        etps.append(torch.as_tensor(zp, device="cuda"))
    return torch.cat(ets), torch.cat(etps)


@pytest.mark.gpu
def test_autograd_fourier_coefficients_vs_fd(G):
    """d(h_1 - h_0)/d(a_k, b_k) through torch.autograd (one transposed solve)
    against central differences of the GPU forward."""
    from paper_1308_5351_gb300 import autograd as AG
    rng = np.random.default_rng(4)
    kmax, n, r0 = 8, 128, 0.3
    centres = [0j, 1.0 + 0j, 0.5 + 0.9j]
    polygons = [Dm.square(-0.9 + 0.2j, 0.24, ccw=False)]
    base = [(rng.normal(0, 0.05 / np.arange(1, kmax + 1)), rng.normal(0, 0.05 / np.arange(1, kmax + 1)))
            for _ in centres]
    m1 = len(centres) + len(polygons)

    def J(coeffs, need_grad):
        et, etp = _star_domain(coeffs, n, centres, r0, polygons)
        A = torch.ones_like(et)
        gam = torch.log(torch.abs(et - centres[0]))
        mu, h, hk = AG.fbie(et, etp, A, gam, m1, n, bounded=False, tol=1e-13)
        return hk[1] - hk[0]

    params = [(torch.tensor(a, device="cuda", requires_grad=True), torch.tensor(b, device="cuda", requires_grad=True))
              for a, b in base]
    val = J(params, True)
    val.backward()
    eps = 1e-6
    for s in range(len(centres)):
        for which in (0, 1):
            for k in (0, 3, kmax - 1):
                def shifted(delta):
                    cs = []
                    for t, (a, b) in enumerate(base):
                        a2, b2 = a.copy(), b.copy()
                        if t == s:
                            (a2 if which == 0 else b2)[k] += delta
                        cs.append((torch.tensor(a2, device="cuda"), torch.tensor(b2, device="cuda")))
                    with torch.no_grad():
                        return float(J(cs, False))
                fd = (shifted(eps) - shifted(-eps)) / (2 * eps)
                an = float(params[s][which].grad[k])
                assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (s, which, k, fd, an)


@pytest.mark.gpu
def test_autograd_hk_output_and_second_backward(G):
    """h_k returned by the library's forward pass equals the component means of
    h; a loss through h_k and the same loss through the means of h give the
    same gradient; a second backward with retain_graph reuses the handle."""
    from paper_1308_5351_gb300 import autograd as AG
    d = Dm.three_circles(64)
    gam = Dm.gamma_log(d, 0.05j)
    et = torch.as_tensor(d.et, device="cuda").requires_grad_(True)
    etp = torch.as_tensor(d.etp, device="cuda")
    A = torch.as_tensor(d.A, device="cuda")
    g = torch.as_tensor(gam, device="cuda").requires_grad_(True)
    w = torch.tensor([0.3, -1.0, 2.0], dtype=torch.float64, device="cuda")
    mu, h, hk = AG.fbie(et, etp, A, g, d.m1, d.n, bounded=True, tol=1e-13)
    assert torch.allclose(hk, h.detach().view(d.m1, d.n).mean(dim=1), rtol=0, atol=1e-13)
    (w * hk).sum().backward(retain_graph=True)
    ga, gg = et.grad.clone(), g.grad.clone()
    et.grad = None
    g.grad = None
    (w * h.view(d.m1, d.n).mean(dim=1)).sum().backward()
    assert torch.allclose(et.grad, ga, rtol=0, atol=1e-9 * float(ga.abs().max()))
    assert torch.allclose(g.grad, gg, rtol=0, atol=1e-9 * float(gg.abs().max()))
