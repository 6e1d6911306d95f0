"""torch.autograd access to the ranking solve (Eq. 6) and to the Laplacian quadratic
form of Eq. 4, with the w-gradients computed by the library's kernels.

* ``solve(g, w, Y, lam)`` -> F = M(w)^-1 lam Y, M = (1 + lam) I - Theta(w).  Its
  backward to w is the adjoint method (``hgl_adjoint_grad``): one batched CG solve of
  M Z = dL/dF with the same operator (M is symmetric), then the bilinear form of the
  Eq. 4 gradient, d/dw_e tr(Z^T Theta F).  Only F is kept from the forward solve; the
  adjoint CG runs its own recurrences.  Y is data: no gradient flows to it.
* ``laplacian_quadratic(g, w, F)`` -> tr(F^T Delta(w) F), Delta = I - Theta, by
  ``hgl_laplacian_quadratic`` (the trace is summed in the library).  Backward:
  to w by ``hgl_weight_grad`` (mu = 0, dv(w) included), to F as 2 Delta F by
  ``hgl_apply_theta`` (a = 2, b = -2); both scaled by the incoming scalar gradient.

The regularised loss of the adaptive method, tr(F^T Delta F) + lam ||F - Y||^2 +
mu ||w||^2 at F = F(w), is then

    F = solve(g, w, Y, lam)
    L = laplacian_quadratic(g, w, F) + lam * ((F - Y) ** 2).sum() + mu * (w ** 2).sum()

and ``L.backward()`` gives dL/dw.  All panels are FP64 on the graph's device.
"""
from __future__ import annotations

import torch

from . import hgl


def _as_panel(t: torch.Tensor) -> torch.Tensor:
    """The library's panel layout (row-major, rows padded to 16 bytes), copying if needed."""
    t = t.detach()
    if t.dtype == torch.float64 and t.stride(1) == 1 and (t.stride(0) * 8) % 16 == 0 and t.data_ptr() % 16 == 0:
        return t
    P = hgl.padded_panel(t.shape[0], t.shape[1], torch.float64, t.device)
    P.copy_(t)
    return P


class _Solve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, w, Y, g, lam, tol, dtype, precond):
        F, _, _, _ = hgl.cg_solve(g, w.detach(), lam, _as_panel(Y), tol=tol, dtype=dtype, precond=precond)
        ctx.save_for_backward(w, F)
        ctx.cfg = (g, lam, tol, dtype, precond)
        return F

    @staticmethod
    def backward(ctx, dF):
        w, F = ctx.saved_tensors
        g, lam, tol, dtype, precond = ctx.cfg
        grad_w = None
        if ctx.needs_input_grad[0]:
            grad_w, _, _ = hgl.adjoint_grad(g, w.detach(), lam, _as_panel(F), _as_panel(dF), tol=tol, dtype=dtype,
                                            precond=precond)
        return grad_w, None, None, None, None, None, None


class _LaplacianQuadratic(torch.autograd.Function):
    @staticmethod
    def forward(ctx, w, F, g):
        Fp = _as_panel(F)
        value, DF = hgl.laplacian_quadratic(g, w.detach(), Fp)  # tr(F^T Delta F), Delta F
        ctx.save_for_backward(w, Fp, DF)
        ctx.g = g
        return torch.tensor(value, dtype=torch.float64, device=Fp.device)

    @staticmethod
    def backward(ctx, go):
        w, Fp, DF = ctx.saved_tensors
        g = ctx.g
        grad_w = grad_F = None
        if ctx.needs_input_grad[0]:
            grad_w = hgl.weight_grad(g, w.detach(), Fp, 0.0) * go
        if ctx.needs_input_grad[1]:
            s = float(go)
            grad_F = hgl.apply_theta(g, w.detach(), Fp, 2.0 * s, -2.0 * s)
        return grad_w, grad_F, None


def solve(g: hgl.Graph, w: torch.Tensor, Y: torch.Tensor, lam: float, tol: float = 1e-10,
          dtype: int = hgl.HGL_FP64, precond: hgl.Precond | None = None) -> torch.Tensor:
    """F = M(w)^-1 lam Y (Eq. 6), differentiable in w by the adjoint method."""
    return _Solve.apply(w, Y, g, lam, tol, dtype, precond)


def laplacian_quadratic(g: hgl.Graph, w: torch.Tensor, F: torch.Tensor) -> torch.Tensor:
    """tr(F^T Delta(w) F) (Eq. 4's first term), differentiable in w and F."""
    return _LaplacianQuadratic.apply(w, F, g)
