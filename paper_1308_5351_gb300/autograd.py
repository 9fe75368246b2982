"""torch.autograd wrapper of the FBIE computation (gnk_fbie forward,
gnk_fbie_backward backward), and differentiable boundary parametrisations.

`fbie(et, etp, A, gam, m1, n, bounded)` returns (mu, h, h_k) as torch tensors
that carry gradients to et, etp, A (complex) and gam (real): the forward pass
is one gnk_fbie call (h_k, the mean of h over each component, comes from the
library), the backward pass one gnk_fbie_backward call (a transposed GMRES
solve plus one pass of Cauchy and derivative-kernel sums; no Krylov basis is
stored between the passes).  The arithmetic of both passes follows
`precision` (GNK_PREC_* of the library).

`star_boundary` builds eta, eta' of star-shaped curves
r(th) = r0 (1 + sum_k a_k cos k th + b_k sin k th) with torch operations, so a
loss of (mu, h, h_k) differentiates down to the Fourier coefficients.
"""
from __future__ import annotations

import math

import torch

from . import gnk as G


class _FBIE(torch.autograd.Function):
    """The boundary handle of the forward pass stays open until this node is
    released, so a second backward (retain_graph=True) can reuse it."""

    @staticmethod
    def forward(ctx, et, etp, A, gam, m1, n, bounded, precision, tol, restart):
        bprec = G.GNK_PREC_DF32 if precision in (G.GNK_PREC_DF32, G.GNK_PREC_MIXED_DF) else G.GNK_PREC_FP64
        if precision in (G.GNK_PREC_FMM, G.GNK_PREC_MIXED_FMM):
            bprec = G.GNK_PREC_FMM
        b = G.Boundary(m1, n, et.detach().contiguous(), etp.detach().contiguous(),
                       A.detach().contiguous(), None, None, bounded, precision=bprec)
        g = gam.detach().contiguous()
        mu, h, hk, res = b.fbie(g, tol=tol, precision=precision, restart=restart)
        if res.status != 0:
            b.close()
            raise G.GnkError(res.status, "forward solve did not converge")
        ctx.b = b
        ctx.opts = dict(tol=tol, precision=precision, restart=restart)
        ctx.save_for_backward(mu, g)
        return mu, h, hk

    @staticmethod
    def backward(ctx, g_mu, g_h, g_hk):
        if ctx.b is None or ctx.b.handle is None:
            raise RuntimeError("the boundary handle of this FBIE forward pass has been released")
        mu, gam = ctx.saved_tensors
        N = mu.numel()
        g_mu = torch.zeros_like(mu) if g_mu is None else g_mu.contiguous().to(torch.float64)
        g_h = torch.zeros_like(mu) if g_h is None else g_h.contiguous().to(torch.float64)
        g_hk = None if g_hk is None else g_hk.contiguous().to(torch.float64)
        g_et = torch.empty(N, dtype=torch.complex128, device=mu.device)
        g_etp = torch.empty_like(g_et)
        g_A = torch.empty_like(g_et)
        g_gam = torch.empty_like(mu)
        G.gnk_fbie_backward(ctx.b.handle, mu, gam, g_mu, g_h, g_et, g_etp, g_A, g_gam,
                            G.options(**ctx.opts), grad_hk=g_hk)
        need = ctx.needs_input_grad
        return (g_et if need[0] else None, g_etp if need[1] else None, g_A if need[2] else None,
                g_gam if need[3] else None, None, None, None, None, None, None)


def fbie(et, etp, A, gam, m1, n, bounded=True, precision=G.GNK_PREC_FP64, tol=1e-12, restart=20):
    """(mu, h, h_k) of the FBIE computation, differentiable in et, etp, A, gam."""
    return _FBIE.apply(et, etp, A, gam, int(m1), int(n), bool(bounded), int(precision), float(tol),
                       int(restart))


def star_boundary(centre, r0, ak, bk, n, ccw=False):
    """eta, eta' at t_p = 2 pi p / n of centre + r(th) e^{i th}, th = +-t, with
    r(th) = r0 (1 + sum_k ak_k cos k th + bk_k sin k th); differentiable in
    ak, bk (real tensors of equal length)."""
    dev = ak.device
    s = 1.0 if ccw else -1.0
    t = torch.arange(n, dtype=torch.float64, device=dev) * (2 * math.pi / n)
    th = s * t
    k = torch.arange(1, ak.numel() + 1, dtype=torch.float64, device=dev)[:, None]
    c = torch.cos(k * th[None, :])
    sn = torch.sin(k * th[None, :])
    r = r0 * (1.0 + (ak[:, None] * c + bk[:, None] * sn).sum(0))
    dr = r0 * (k * (-ak[:, None] * sn + bk[:, None] * c)).sum(0)
    e = torch.exp(1j * th.to(torch.complex128))
    z = complex(centre) + r.to(torch.complex128) * e
    zp = s * (dr.to(torch.complex128) + 1j * r.to(torch.complex128)) * e
    return z, zp
