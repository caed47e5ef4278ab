"""C_eff as a differentiable function of the per-voxel moduli.

forward: ce_solve of the six unit load cases + ce_ceff (C = S E^-1).
backward: ce_grad with w = dL/dC: the discrete operator is symmetric, so the
adjoint fields of J = sum w_mn C_mn are the converged forward fields; no
second solve is run and no iterate is stored (the library keeps the
converged fields of the forward solve as the checkpoint).  Inverse problems
are the paper's future item 5 (Sec. 5.3).
"""
from __future__ import annotations

import numpy as np
import torch

from . import ce


class CEff(torch.autograd.Function):
    @staticmethod
    def forward(ctx, K, G, tol=1e-6, max_iter=1_000_000, prec="fp32", St=None, n_check=0, keep=True):
        if not (K.is_cuda and G.is_cuda):
            raise ce.CeError(ce.CE_EINVAL, "CEff needs CUDA tensors")
        c = ce.Context(K, G, prec=prec, St=St, n_check=n_check)
        try:
            c.solve(None, tol=tol, max_iter=max_iter)
            C = torch.from_numpy(c.ceff()).to(K.device)
        except Exception:
            c.close()
            raise
        # the converged fields are the checkpoint of the backward pass; when
        # no gradient will be asked for (keep is False: no input requires one,
        # or autograd was off at the call) the context and its device state
        # are released at once
        if keep and (ctx.needs_input_grad[0] or ctx.needs_input_grad[1]):
            ctx.ce = c
        else:
            c.close()
            ctx.ce = None
        ctx.shape = K.shape
        return C

    @staticmethod
    def backward(ctx, gC):
        c = ctx.ce
        if c is None:
            return None, None, None, None, None, None, None, None
        w = gC.detach().to("cpu", torch.float64).numpy()
        dK = torch.empty(ctx.shape, dtype=torch.float32, device=gC.device)
        dG = torch.empty(ctx.shape, dtype=torch.float32, device=gC.device)
        c.grad(w, dK, dG)
        torch.cuda.current_stream().synchronize()
        c.close()
        return dK, dG, None, None, None, None, None, None


def ceff(K, G, **kw):
    """C_eff (6x6 float64 tensor on K's device); differentiable in K and G."""
    keep = torch.is_grad_enabled() and (K.requires_grad or G.requires_grad)
    return CEff.apply(K, G, kw.get("tol", 1e-6), kw.get("max_iter", 1_000_000), kw.get("prec", "fp32"),
                      kw.get("St"), kw.get("n_check", 0), keep)
