"""torch.autograd.Function wrappers of the library's operators (marshalling only).

``DwFunction``: y = gamma5 D_w(mu; U) x (Sec. 1, Eq. 1.2) with gradients with
respect to the links U, the chemical potential mu and the source x, from the
library's adjoint kernels (``ovl_dw_grad``, and the stencil with mu -> -mu for
A^dag).
``SignFunction``: y = sgn(gamma5 D_w(mu; U)) b by k steps of two-sided Lanczos
(Sec. 4), with gradients with respect to U, mu and b from the library's
resolvent-form derivative (``ovl_sign_grad``: one two-sided process started
from b and the upstream gradient).
Complex gradients follow PyTorch's convention (g_z = dl/dRe z + i dl/dIm z).
"""
from __future__ import annotations

import torch

from . import ovl as _ovl


class DwFunction(torch.autograd.Function):
    """y = A(U, mu) x; call as DwFunction.apply(U, mu, x, ctx, kappa)."""

    @staticmethod
    def forward(ctx, U, mu, x, lat, kappa):
        mu_f = float(mu)
        lat.set_gauge(U.detach().contiguous())
        y = lat.apply_Dw(mu_f, kappa, x.detach().contiguous(), flags=_ovl.GAMMA5)
        ctx.save_for_backward(U, x)
        ctx.lat, ctx.mu, ctx.kappa = lat, mu_f, kappa
        ctx.mu_is_tensor = isinstance(mu, torch.Tensor)
        return y

    @staticmethod
    def backward(ctx, g):
        U, x = ctx.saved_tensors
        lat, mu, kappa = ctx.lat, ctx.mu, ctx.kappa
        g = g.contiguous()
        lat.set_gauge(U.detach().contiguous())
        grad_x = lat.apply_Dw(mu, kappa, g, flags=_ovl.DAGGER) if ctx.needs_input_grad[2] else None
        grad_U = torch.empty_like(U) if ctx.needs_input_grad[0] else None
        grad_mu = None
        if ctx.needs_input_grad[0] or ctx.needs_input_grad[1]:
            _, gm = lat.dw_grad(mu, kappa, x.detach().contiguous(), g, grad_U)
            if ctx.needs_input_grad[1] and ctx.mu_is_tensor:
                grad_mu = torch.tensor(gm, dtype=torch.float64, device=g.device)
        return grad_U, grad_mu, grad_x, None, None


class SignFunction(torch.autograd.Function):
    """y = sgn(A(U, mu)) b; call as SignFunction.apply(U, mu, b, ctx, kappa, k)."""

    @staticmethod
    def forward(ctx, U, mu, b, lat, kappa, k):
        mu_f = float(mu)
        lat.set_gauge(U.detach().contiguous())
        b_ = b.detach().contiguous()
        y, _ = lat.sign_krylov(_ovl.LANCZOS2, int(k), mu_f, kappa, b_)
        ctx.save_for_backward(U, b_)
        ctx.lat, ctx.mu, ctx.kappa, ctx.k = lat, mu_f, kappa, int(k)
        ctx.mu_is_tensor = isinstance(mu, torch.Tensor)
        return y

    @staticmethod
    def backward(ctx, g):
        U, b = ctx.saved_tensors
        lat = ctx.lat
        lat.set_gauge(U.detach().contiguous())
        grad_U = torch.empty_like(U) if ctx.needs_input_grad[0] else None
        grad_b = torch.empty_like(b) if ctx.needs_input_grad[2] else None
        gm, _ = lat.sign_grad(ctx.k, ctx.mu, ctx.kappa, b, g.contiguous(), grad_U=grad_U, grad_b=grad_b)
        grad_mu = None
        if ctx.needs_input_grad[1] and ctx.mu_is_tensor:
            grad_mu = torch.tensor(gm, dtype=torch.float64, device=g.device)
        return grad_U, grad_mu, grad_b, None, None, None


def sign_A(U, mu, b, lat, kappa, k):
    return SignFunction.apply(U, mu, b, lat, kappa, k)


def apply_A(U, mu, x, lat, kappa):
    return DwFunction.apply(U, mu, x, lat, kappa)
