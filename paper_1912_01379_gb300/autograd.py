"""<A(omega)> as a differentiable function (torch.autograd.Function).

forward:  the average spectrum <A> = <fbar>/w of the sampler, with the snapshot
          moments accumulated on the device (asm_sample with ASM_SAMPLE_MOMENTS).
backward: asm_backward, the covariance-identity vector-Jacobian products
          d<A>/dG = Cov(fbar, fbar) K^T C^{-1} / w and
          d<A>/dtheta = Cov(fbar, s_theta) / w - <fbar> dw/dtheta / w^2.
Marshalling only: the sampling, the moments and the products run in the CUDA
library.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Callable

import numpy as np
import torch

from . import asm


@dataclass
class ASMSpec:
    """How to build the problem for given theta and how to sample it.
    build(theta) returns (K, C, w, levels, dK_dtheta, dw_dtheta); theta may be
    empty (no grid parameters), then the last two are None."""
    build: Callable
    chains: int = 1024
    burn_in: int = 200
    sweeps: int = 2000
    seed: int = 1
    precision: int = asm.ASM_MIXED


class ASMAverage(torch.autograd.Function):
    @staticmethod
    def forward(ctx, G, theta, spec: ASMSpec):
        th = theta.detach().cpu().double().numpy()
        K, C, w, levels, dK, dw = spec.build(th)
        if dK is not None and len(th) == 0:
            dK = dw = None
        gp = asm.Problem(K, G.detach().cpu().double().numpy(), C, levels, w=w, dK_dtheta=dK, dw_dtheta=dw)
        gp.sample(spec.chains, spec.burn_in, spec.sweeps, spec.seed, precision=spec.precision, moments=True)
        r = gp.average()
        ctx.gp = gp
        ctx.has_theta = dK is not None
        return torch.from_numpy(r["mean_A"]).to(dtype=G.dtype)

    @staticmethod
    def backward(ctx, v):
        gG, gt = ctx.gp.backward(v.detach().cpu().double().numpy(), want_theta=ctx.has_theta)
        g_G = torch.from_numpy(gG).to(dtype=v.dtype)
        g_t = torch.from_numpy(gt).to(dtype=v.dtype) if gt is not None else None
        return g_G, g_t, None


def average_spectrum(G: torch.Tensor, theta: torch.Tensor, spec: ASMSpec) -> torch.Tensor:
    return ASMAverage.apply(G, theta, spec)
