"""torch.autograd.Function around create / solve / energy / grad of libesmp2.

forward returns E2 (a float64 scalar tensor on the inputs' device); backward returns
dE2/dF and dE2/d(ia|jb) from the library's adjoint (esmp2_grad), scaled by the incoming
gradient.  Gradients with respect to ooov, ovvv and C are not provided (None)."""
from __future__ import annotations

import numpy as np
import torch

from .esmp2 import FP64, Handle


class ESMP2Energy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, F, ovov, ooov, ovvv, C, tol: float = 1e-10, precision: int = FP64, maxit: int = 3000):
        dev = F.device
        h = Handle(F.detach(), ovov.detach(), ooov.detach(), ovvv.detach(), C.detach())
        h.solve(tol=tol, maxit=maxit, precision=precision)
        e = h.energy()["E2"]
        ctx.h = h
        ctx.dev = dev
        return torch.tensor(e, dtype=torch.float64, device=dev)

    @staticmethod
    def backward(ctx, g):
        dF, dov, _ = ctx.h.grad()
        ctx.h.close()
        dev = ctx.dev
        gF = torch.from_numpy(np.ascontiguousarray(dF)).to(dev) * g
        gov = torch.from_numpy(np.ascontiguousarray(dov)).to(dev) * g
        return gF, gov, None, None, None, None, None, None


def esmp2_energy(F, ovov, ooov, ovvv, C, tol: float = 1e-10, precision: int = FP64, maxit: int = 3000):
    """Differentiable E2 (with respect to F and (ia|jb))."""
    return ESMP2Energy.apply(F, ovov, ooov, ovvv, C, tol, precision, maxit)
