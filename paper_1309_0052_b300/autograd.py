"""Differentiable coherent power for fine acquisition (torch.autograd.Function).

P(f, tau) = |sum_n x[n] exp(-j 2 pi f n / fs) ctilde(n 1023 / N - tau - 1/2)|^2
over the first coh_ms milliseconds of a recording, with its analytic
gradient (dP/df, dP/dtau) computed by the same CUDA kernel as the value
(gnss_refine_eval).  The Function only marshals tensors: forward runs the
kernel once and keeps the gradient for backward.
"""
from __future__ import annotations

import torch

from . import Plan


class CoherentPower(torch.autograd.Function):
    """P = CoherentPower.apply(f, tau, plan, samples, n_samples, prn, coh_ms)

    f, tau: float64 CUDA tensors [n] (Hz, chips); prn: int32 CUDA tensor [n];
    samples: CUDA uint8 tensor holding the recording in the plan's format.
    Returns P (float32 [n]).  Gradients flow to f and tau."""

    @staticmethod
    def forward(ctx, f, tau, plan: Plan, samples, n_samples: int, prn, coh_ms: int):
        if not (f.is_cuda and tau.is_cuda and prn.is_cuda and samples.is_cuda):
            raise ValueError("CoherentPower needs CUDA tensors (no CPU path)")
        f = f.detach().to(torch.float64).contiguous()
        tau = tau.detach().to(torch.float64).contiguous()
        prn = prn.to(torch.int32).contiguous()
        n = f.numel()
        P = torch.empty(n, dtype=torch.float32, device=f.device)
        gf = torch.empty_like(P)
        gt = torch.empty_like(P)
        stream = torch.cuda.current_stream(f.device)
        plan.refine_eval(samples, n_samples, coh_ms, prn, f, tau, P, gf, gt, stream=stream)
        ctx.save_for_backward(gf, gt)
        return P

    @staticmethod
    def backward(ctx, grad_P):
        gf, gt = ctx.saved_tensors
        g = grad_P.to(torch.float64)
        return g * gf.to(torch.float64), g * gt.to(torch.float64), None, None, None, None, None


def coherent_power(f, tau, plan: Plan, samples, n_samples: int, prn, coh_ms: int):
    return CoherentPower.apply(f, tau, plan, samples, n_samples, prn, coh_ms)
