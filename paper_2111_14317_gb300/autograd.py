"""Differentiation through the solutions: torch.autograd.Function over libhpt.

Forward tracks start points to t = 1 and polishes them (hpt_track); backward
is the implicit-function adjoint (hpt_adjoint): at a solution x of
F(x; c) = 0 with J = F_x, the coefficient gradient of a real loss L is
-sum_solutions lambda_k conj(x^{a_{k,i}}) with J^H lambda = dL/dx, in
PyTorch's convention dL/dRe z + i dL/dIm z for complex tensors.  Paths that
did not converge carry no gradient.
"""
from __future__ import annotations

import torch

from . import hpt


class HptSolve(torch.autograd.Function):
    """x, status = HptSolve.apply(coeffs, spec, y0, params)

    coeffs: (M,) complex128 tensor (the differentiable input);
    spec:   dict(n, m, exponents, lifting, cell[, precision]) describing the
            supports, lifting and cell (see include/hpt.h);
    y0:     (p, n) complex128 CUDA tensor of start points for the cell;
    params: hpt.Params or None.
    Returns x (p, n) complex128 and the per-path status (int32).
    """

    @staticmethod
    def forward(ctx, coeffs, spec, y0, params=None):
        sysh = hpt.System(spec["n"], spec["m"], spec["exponents"], coeffs.detach().cpu().numpy(),
                          spec["lifting"], spec["cell"], spec.get("precision", hpt.HPT_FP64))
        x, status, _ = sysh.track(y0.contiguous(), params)
        ctx.sysh = sysh
        ctx.coeff_device = coeffs.device
        ctx.save_for_backward(x, status)
        ctx.mark_non_differentiable(status)
        return x, status

    @staticmethod
    def backward(ctx, gx, _gstatus):
        x, status = ctx.saved_tensors
        if gx is None:
            return None, None, None, None
        keep = torch.nonzero(status == hpt.CONVERGED).squeeze(1)
        gc = ctx.sysh.adjoint(x.index_select(0, keep).contiguous(),
                              gx.to(torch.complex128).index_select(0, keep).contiguous())
        return gc.to(ctx.coeff_device), None, None, None


def solve(coeffs, spec, y0, params=None):
    """Differentiable solutions of the target system (see HptSolve)."""
    return HptSolve.apply(coeffs, spec, y0, params)
