"""torch.autograd glue for the log-marginal-likelihood gradient.

`mll_surrogate(X, log_sigma, log_gamma, y)` returns a zero-valued scalar whose
gradient with respect to X, log sigma and log gamma is the gradient of the
GP log marginal likelihood (Sec. 2.1's maximum-likelihood fit; see
`krr_mll_grad` in libkrr.h for the estimator).  Adding it to a loss, or
calling backward on it, puts dL/dX, dL/dlog sigma and dL/dlog gamma into the
.grad fields.  Ascend them to maximise L.  Every number comes from one
`krr_mll_grad` call (all of it in libkrr's kernels).  This module only routes
the results through autograd, and the value of L itself is not computed.
"""
import torch

from . import binding


class MLLGrad(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, log_sigma, log_gamma, y, n_probes, seed, opts):
        sigma = float(torch.exp(log_sigma.detach()))
        gamma = float(torch.exp(log_gamma.detach()))
        want_dx = bool(ctx.needs_input_grad[0])
        gs, gg, gX, infos = binding.krr_mll_grad(X.detach().contiguous(), y.detach().contiguous(),
                                                 sigma, gamma, n_probes=n_probes, seed=seed,
                                                 opts=opts, want_dX=want_dx)
        ctx.infos = infos
        ctx.gs = torch.tensor(gs, dtype=log_sigma.dtype, device=log_sigma.device)
        ctx.gg = torch.tensor(gg, dtype=log_gamma.dtype, device=log_gamma.device)
        ctx.save_for_backward(gX if gX is not None else X.new_zeros(0))
        ctx.has_dx = gX is not None
        return X.new_zeros(())

    @staticmethod
    def backward(ctx, g):
        (gX,) = ctx.saved_tensors
        dX = g * gX if ctx.has_dx else None
        return dX, g * ctx.gs, g * ctx.gg, None, None, None, None


def mll_surrogate(X, log_sigma, log_gamma, y, n_probes=32, seed=0, opts=None):
    """Zero-valued scalar carrying the MLL gradient (see the module docstring)."""
    return MLLGrad.apply(X, log_sigma, log_gamma, y, n_probes, seed, opts)
