"""torch.autograd wrappers of the two transforms with the hand-written
adjoints of libsht (no counterpart in the paper; see include/sht.h).

Parameters are real: an a_lm batch is handled as a float64 tensor
[..., nalm, 2] holding (Re, Im); Im a_l0 is ignored on input and its gradient
is zero, matching the real-field convention of the transforms (a real map has
real a_l0 and stores m >= 0 only). Gradients are exact transposes:

    d/d(Re, Im) a of <h, alm2map(a)>      = alm2map_adjoint(h)
    d/d maps     of <g, map2alm(maps)>_ri = map2alm_adjoint(g)

where <., .>_ri is the real inner product over (Re, Im) pairs.
"""
from __future__ import annotations

import torch

from .sht import Plan


class _Alm2Map(torch.autograd.Function):
    @staticmethod
    def forward(ctx, alm_ri: torch.Tensor, plan: Plan) -> torch.Tensor:
        ctx.plan = plan
        return plan.alm2map(torch.view_as_complex(alm_ri.contiguous()))

    @staticmethod
    def backward(ctx, grad_map: torch.Tensor):
        g = ctx.plan.alm2map_adjoint(grad_map.contiguous())
        return torch.view_as_real(g), None


class _Map2Alm(torch.autograd.Function):
    @staticmethod
    def forward(ctx, maps: torch.Tensor, plan: Plan) -> torch.Tensor:
        ctx.plan = plan
        return torch.view_as_real(plan.map2alm(maps.contiguous()))

    @staticmethod
    def backward(ctx, grad_ri: torch.Tensor):
        g = ctx.plan.map2alm_adjoint(torch.view_as_complex(grad_ri.contiguous()))
        return g, None


def alm2map(alm_ri: torch.Tensor, plan: Plan) -> torch.Tensor:
    """Differentiable alm2map: (Re, Im) a_lm [nmaps, ncomp, nalm, 2] -> maps [nmaps, ncomp, npix]."""
    return _Alm2Map.apply(alm_ri, plan)


def map2alm(maps: torch.Tensor, plan: Plan) -> torch.Tensor:
    """Differentiable map2alm (plain quadrature): maps -> (Re, Im) a_lm [nmaps, ncomp, nalm, 2]."""
    return _Map2Alm.apply(maps, plan)


def refine(alm_ri: torch.Tensor, target: torch.Tensor, plan: Plan, niter: int) -> torch.Tensor:
    """Algorithm 2 as a differentiable chain: a <- a + map2alm(target - alm2map(a)), niter times."""
    a = alm_ri
    for _ in range(niter):
        a = a + map2alm(target - alm2map(a, plan), plan)
    return a
