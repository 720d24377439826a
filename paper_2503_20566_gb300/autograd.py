"""ln|psi| as a differentiable PyTorch function of the PEPS parameters.

Forward: the parameters go to the library (gcf_set_tensors) and gcf_amplitude
gives ln|psi(s)| per configuration.  Backward: the hand-written adjoint of
the boundary contraction, gcf_log_grad_vjp, gives sum_s g_s d ln psi(s) /
d theta for the incoming gradient g.  Real tensors only: for them
d ln psi / d theta = d ln|psi| / d theta (Eq. S3).
"""

from __future__ import annotations

import torch


class LogAbsPsi(torch.autograd.Function):
    @staticmethod
    def forward(fctx, theta, context, configs):
        if context.complex:
            raise TypeError("LogAbsPsi supports real tensors; use Context.log_grad_vjp for complex ones")
        context.set_tensors(theta.detach().to("cpu", torch.float64).numpy())
        la, _ = context.amplitude(configs)
        fctx.context = context
        fctx.configs = configs
        fctx.theta_device = theta.device
        fctx.theta_dtype = theta.dtype
        return la.to(theta.device)

    @staticmethod
    def backward(fctx, grad_la):
        g = fctx.context.log_grad_vjp(fctx.configs, grad_la.detach().to("cuda", torch.float64))
        return g.to(fctx.theta_device, fctx.theta_dtype), None, None


def log_abs_psi(theta, context, configs):
    """ln|psi(s)| for each configuration, differentiable in theta."""
    return LogAbsPsi.apply(theta, context, configs)
