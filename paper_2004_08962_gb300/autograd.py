"""Differentiable HICU convolutions: torch.autograd.Function wrappers over libhicu.

  ConvNull         R = H(x) f                       forward: hicu_conv_null
  ConvNullAdjoint  g = (1 - M) o H^H(R f) on S      forward: hicu_conv_null_adjoint
  NullObjective    F = ||H(x) f||_F^2               forward: hicu_conv_null (objective only)

x is multi-coil k-space [C][Nz][Ny][Nx] and f a bank of p annihilating filters [p][n]
(n = C kz ky kx), both complex64 on the GPU.  Every convolution, adjoint, filter gradient
and projection runs in the library's kernels; this module only chains them (besides
zero-filling output arrays and scaling p x n filter banks by the upstream scalar
gradient).  Gradients follow PyTorch's
convention for complex tensors (for a real loss L the gradient of z is 2 dL/d(conj z)),
which makes each vector-Jacobian product the adjoint of the linear map:

  ConvNull:        x_bar = H^H(R_bar f)  (adjoint, no mask)    f_bar = H(x)^H R_bar
  ConvNullAdjoint: R_bar = H(P g_bar) f  (conv of the masked upstream gradient)
                   f_bar = H(P g_bar)^H R   (g is conjugate-linear in f)
  NullObjective:   x_bar = 2 H^H(R f),  f_bar = 2 H(x)^H R,  with R = H(x) f

where P is the projection onto unobserved entries of S.  NullObjective keeps no
convolution output between forward and backward: the forward only reduces ||R||^2 and
the backward recomputes R, which is what keeps 3D problems (R of hundreds of MB) in memory.
"""
from __future__ import annotations

from typing import Optional, Sequence

import torch

from . import hicu


class HicuConv:
    """Geometry, region, precision and handle shared by the differentiable operators."""

    def __init__(self, handle: hicu.Handle, dims: Sequence[int], ncoil: int, kernel: Sequence[int],
                 region=None, circular=(0, 0, 0), mask_per_coil: bool = False, prec: int = hicu.HICU_FP32):
        self.h = handle
        self.geom = hicu.make_geom(dims, ncoil, kernel, circular, mask_per_coil=mask_per_coil)
        off, ext = region if region is not None else ((0, 0, 0), tuple(dims))
        self.region = hicu.make_region(off, ext)
        self.prec = prec
        self.shape = (ncoil, dims[2], dims[1], dims[0])

    def conv_null(self, x: torch.Tensor, f: torch.Tensor) -> torch.Tensor:
        return ConvNull.apply(x, f, self)

    def conv_null_adjoint(self, R: torch.Tensor, f: torch.Tensor, mask: Optional[torch.Tensor] = None):
        return ConvNullAdjoint.apply(R, f, mask, self)

    def null_objective(self, x: torch.Tensor, f: torch.Tensor) -> torch.Tensor:
        return NullObjective.apply(x, f, self)

    # ---- raw library calls (no autograd)
    def _conv(self, x, f, want_R=True):
        if want_R:
            return hicu.hicu_conv_null(self.h, self.geom, self.region, x.contiguous(), f.contiguous(),
                                       prec=self.prec)
        _, obj = hicu.hicu_conv_null(self.h, self.geom, self.region, x.contiguous(), f.contiguous(),
                                     prec=self.prec, want_objective=True, store_R=False)
        return obj

    def _adjoint(self, R, f, mask=None):
        g = torch.zeros(self.shape, dtype=torch.complex64, device=R.device)
        return hicu.hicu_conv_null_adjoint(self.h, self.geom, self.region, R.contiguous(), f.contiguous(),
                                           mask=mask, g=g, prec=self.prec)

    def _fgrad(self, x, Rbar):
        return hicu.hicu_conv_null_filter_grad(self.h, self.geom, self.region, x.contiguous(),
                                               Rbar.contiguous())

    def _project(self, x, mask):
        return hicu.hicu_project_unobserved(self.h, self.geom, self.region, x.contiguous(), mask)


class ConvNull(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, f, op: HicuConv):
        ctx.op = op
        ctx.save_for_backward(x, f)
        return op._conv(x, f)

    @staticmethod
    def backward(ctx, gR):
        x, f = ctx.saved_tensors
        op = ctx.op
        gR = gR.contiguous()
        gx = op._adjoint(gR, f) if ctx.needs_input_grad[0] else None
        gf = op._fgrad(x, gR) if ctx.needs_input_grad[1] else None
        return gx, gf, None


class ConvNullAdjoint(torch.autograd.Function):
    @staticmethod
    def forward(ctx, R, f, mask, op: HicuConv):
        ctx.op = op
        ctx.mask = mask
        ctx.save_for_backward(R, f)
        return op._adjoint(R, f, mask)

    @staticmethod
    def backward(ctx, gg):
        R, f = ctx.saved_tensors
        op = ctx.op
        gp = op._project(gg.contiguous(), ctx.mask)
        gR = op._conv(gp, f) if ctx.needs_input_grad[0] else None
        gf = op._fgrad(gp, R) if ctx.needs_input_grad[1] else None
        return gR, gf, None, None


class NullObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, f, op: HicuConv):
        ctx.op = op
        ctx.save_for_backward(x, f)   # R = H(x) f is not kept: the backward recomputes it
        return op._conv(x, f, want_R=False).reshape(())

    @staticmethod
    def backward(ctx, go):
        x, f = ctx.saved_tensors
        op = ctx.op
        R = op._conv(x, f)
        # both maps are real-linear in R and g is real-linear in f, so the real factor 2 go
        # is applied to the small p x n banks instead of the large arrays; it stays a device
        # scalar (no host read, so the backward pass never waits for the stream)
        s = (2.0 * go.detach()).to(f.dtype)
        gx = op._adjoint(R, f * s) if ctx.needs_input_grad[0] else None
        gf = op._fgrad(x, R) * s if ctx.needs_input_grad[1] else None
        return gx, gf, None
