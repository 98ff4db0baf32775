"""torch.autograd.Function wrappers: gradients of the corrected images (Eq. 1) and of the
objective J (Eq. 4) with respect to the two input images, the field b and the weights alpha and
beta, at fixed b.  Forward and backward run in the library's CUDA kernels (hysco_correct /
hysco_correct_adjoint, hysco_eval / hysco_image_grad); this module only marshals tensors.

SolvedField differentiates through the Gauss-Newton solve itself: its output is the solved
field b*, and its backward applies the implicit function theorem at b* (one adjoint PCG solve with
the Gauss-Newton Hessian, hysco_solve_adjoint), exact when b* is a stationary point of J.
"""
from __future__ import annotations

import torch


class CorrectedImages(torch.autograd.Function):
    """(Ip, Im, b) -> (Tp, Tm) = (I+(x + b)(1 + d_v b), I-(x - b)(1 - d_v b)) on handle h."""

    @staticmethod
    def forward(ctx, h, Ip, Im, b):
        Tp, Tm = h.correct(Ip, Im, b)
        ctx.h = h
        ctx.save_for_backward(Ip, Im, b)
        return Tp, Tm

    @staticmethod
    def backward(ctx, gTp, gTm):
        Ip, Im, b = ctx.saved_tensors
        need = ctx.needs_input_grad
        if not any(need[1:4]):
            return None, None, None, None
        gTp = None if gTp is None else gTp.float().contiguous()
        gTm = None if gTm is None else gTm.float().contiguous()
        dIp, dIm, db = ctx.h.correct_adjoint(Ip, Im, b, gTp, gTm, want=need[1:4])
        return (None, None if dIp is None else dIp.to(Ip.dtype),
                None if dIm is None else dIm.to(Im.dtype), db)


class CorrectedImage(torch.autograd.Function):
    """(Ip, Im, b) -> T = 1/2 (Tp + Tm), the corrected image, on handle h."""

    @staticmethod
    def forward(ctx, h, Ip, Im, b):
        T = h.correct_mean(Ip, Im, b)
        ctx.h = h
        ctx.save_for_backward(Ip, Im, b)
        return T

    @staticmethod
    def backward(ctx, gT):
        Ip, Im, b = ctx.saved_tensors
        need = ctx.needs_input_grad
        if not any(need[1:4]):
            return None, None, None, None
        dIp, dIm, db = ctx.h.correct_mean_adjoint(Ip, Im, b, gT.float().contiguous(),
                                                  want=need[1:4])
        return (None, None if dIp is None else dIp.to(Ip.dtype),
                None if dIm is None else dIm.to(Im.dtype), db)


class Objective(torch.autograd.Function):
    """(Ip, Im, b, alpha, beta) -> J (float64 scalar) = D + alpha S + beta P on handle h, whose
    weights alpha and beta the arguments must equal (dJ/dalpha = S, dJ/dbeta = P)."""

    @staticmethod
    def forward(ctx, h, Ip, Im, b, alpha, beta):
        a = float(alpha) if not isinstance(alpha, torch.Tensor) else float(alpha.item())
        be = float(beta) if not isinstance(beta, torch.Tensor) else float(beta.item())
        if a != h.alpha or be != h.beta:
            raise ValueError(f"alpha, beta = {a}, {be} differ from the handle's "
                             f"{h.alpha}, {h.beta}")
        terms, grad = h.eval(Ip, Im, b, grad=True)
        ctx.h = h
        ctx.save_for_backward(Ip, Im, b, grad, terms)
        ctx.weight_like = (alpha if isinstance(alpha, torch.Tensor) else None,
                           beta if isinstance(beta, torch.Tensor) else None)
        return terms[0].clone()

    @staticmethod
    def backward(ctx, gJ):
        Ip, Im, b, grad, terms = ctx.saved_tensors
        need = ctx.needs_input_grad
        g = float(gJ.item())
        dIp = dIm = None
        if need[1] or need[2]:
            dIp, dIm = ctx.h.image_grad(Ip, Im, b, g, want=(need[1], need[2]))
            dIp = None if dIp is None else dIp.to(Ip.dtype)
            dIm = None if dIm is None else dIm.to(Im.dtype)
        db = grad * g if need[3] else None
        wa, wb = ctx.weight_like
        da = (g * terms[2]).to(wa.dtype).reshape(wa.shape) if need[4] else None
        dbe = (g * terms[3]).to(wb.dtype).reshape(wb.shape) if need[5] else None
        return None, dIp, dIm, db, da, dbe


def corrected_images(h, Ip, Im, b):
    """Differentiable (Tp, Tm)."""
    return CorrectedImages.apply(h, Ip, Im, b)


def corrected_image(h, Ip, Im, b):
    """Differentiable 1/2 (Tp + Tm), the corrected image."""
    return CorrectedImage.apply(h, Ip, Im, b)


def objective(h, Ip, Im, b, alpha=None, beta=None):
    """Differentiable J; alpha / beta default to the handle's weights (as float64 tensors)."""
    dev = b.device
    alpha = torch.tensor(h.alpha, dtype=torch.float64, device=dev) if alpha is None else alpha
    beta = torch.tensor(h.beta, dtype=torch.float64, device=dev) if beta is None else beta
    return Objective.apply(h, Ip, Im, b, alpha, beta)


class SolvedField(torch.autograd.Function):
    """(Ip, Im, alpha, beta) -> b*: the GN-PCG solve on handle h (whose alpha and beta the arguments
    must equal).  Backward by implicit differentiation at b*: with H v = dL/db*,
    dL/dI+- = -d(v^T g)/dI+-, dL/dalpha = -v^T grad S, dL/dbeta = -v^T grad P."""

    @staticmethod
    def forward(ctx, h, Ip, Im, alpha, beta, solve_kwargs, adjoint_iters, adjoint_rtol):
        a = float(alpha) if not isinstance(alpha, torch.Tensor) else float(alpha.item())
        be = float(beta) if not isinstance(beta, torch.Tensor) else float(beta.item())
        if a != h.alpha or be != h.beta:
            raise ValueError(f"alpha, beta = {a}, {be} differ from the handle's "
                             f"{h.alpha}, {h.beta}")
        b, _ = h.solve(Ip, Im, stats=False, **solve_kwargs)
        ctx.h = h
        ctx.adjoint = (adjoint_iters, adjoint_rtol)
        ctx.weight_like = (alpha if isinstance(alpha, torch.Tensor) else None,
                           beta if isinstance(beta, torch.Tensor) else None)
        ctx.save_for_backward(Ip, Im, b)
        return b

    @staticmethod
    def backward(ctx, gb):
        Ip, Im, b = ctx.saved_tensors
        need = ctx.needs_input_grad
        it, rtol = ctx.adjoint
        _, dIp, dIm, dth = ctx.h.solve_adjoint(Ip, Im, b, gb.float().contiguous(), max_iters=it,
                                               rtol=rtol)
        wa, wb = ctx.weight_like
        return (None, dIp.to(Ip.dtype) if need[1] else None,
                dIm.to(Im.dtype) if need[2] else None,
                dth[0].to(wa.dtype).reshape(wa.shape) if need[3] else None,
                dth[1].to(wb.dtype).reshape(wb.shape) if need[4] else None, None, None, None)


def solved_field(h, Ip, Im, alpha=None, beta=None, adjoint_iters=200, adjoint_rtol=1e-6,
                 **solve_kwargs):
    """Differentiable b* = solve(Ip, Im) (OT start, the handle's weights); keyword arguments go to
    Hysco.solve (gn_iters, pcg_max_iters, ...)."""
    dev = Ip.device
    alpha = torch.tensor(h.alpha, dtype=torch.float64, device=dev) if alpha is None else alpha
    beta = torch.tensor(h.beta, dtype=torch.float64, device=dev) if beta is None else beta
    return SolvedField.apply(h, Ip, Im, alpha, beta, solve_kwargs, adjoint_iters, adjoint_rtol)
