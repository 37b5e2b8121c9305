"""torch.autograd.Function over gp_logml_and_grad.

Forward runs the whole training pass in libgp (Eq. ll and its gradient by
the stochastic trace estimator of Sec. 3.2); backward returns the saved
gradient scaled by the upstream gradient.  Hyperparameters are CPU float64
tensors (natural parameters); X and y stay on the device.
"""
from __future__ import annotations

import numpy as np
import torch

from .api import Theta, gp_logml_and_grad


class MarginalLikelihood(torch.autograd.Function):
    @staticmethod
    def forward(fctx, lengthscale, outputscale, sigma2, X, y, gp_ctx, options):
        theta = Theta(lengthscale.detach().cpu().numpy().astype(np.float64),
                      float(outputscale), float(sigma2))
        r = gp_logml_and_grad(gp_ctx, X, theta, y, want_grad=True, **(options or {}))
        g = torch.tensor(r["grad"], dtype=torch.float64)
        fctx.save_for_backward(g)
        fctx.d = lengthscale.numel()
        fctx.result = r
        return torch.tensor(r["logml"], dtype=torch.float64)

    @staticmethod
    def backward(fctx, grad_out):
        (g,) = fctx.saved_tensors
        d = fctx.d
        go = grad_out.to(torch.float64)
        return g[:d] * go, g[d] * go, g[d + 1] * go, None, None, None, None
