"""torch.autograd wrapper of the moment-only evolution.

``evolve(m0, tau, nsteps)`` advances canonical moments m0 (a CUDA tensor of
shape (10, nz, ny, nx), float64 or float32) by nsteps one-component steps
through libllb and returns the canonical moments at the end; with
``two_component=dict(beta=..., A_s=..., grad_eps=...)`` m0 has the 11
two-component fields (rho1, rho2, j, P) and the colour-gradient step with the
smooth interface normal (no near-contact switch) is used.  Its backward
pass calls ``llb_adjoint`` (hand-written adjoint kernels with checkpoints of
the moments every ``every`` steps), so gradients of any torch loss of the
result flow to m0 -- and through whatever built m0, e.g. an equilibrium
initialisation from a velocity field -- and to tau.

Marshalling only: the forward steps and the adjoint run in the library.
"""
from __future__ import annotations

import torch

from . import llb


def _params(dtype, stream, cg):
    storage = llb.LLB_F64 if dtype == torch.float64 else llb.LLB_F32
    if cg is None:
        return llb.llb_params_default(storage=storage, stream=stream)
    return llb.llb_params_default(storage=storage, stream=stream, ncomp=2, A_h=0.0, **cg)


class MomentOnlyEvolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m0, tau, nsteps: int, lattice: int, every: int, cg):
        nf = 10 if cg is None else 11
        if not m0.is_cuda or m0.dim() != 4 or m0.shape[0] != nf:
            raise ValueError(f"m0 must be a CUDA tensor of shape ({nf}, nz, ny, nx)")
        m0c = m0.detach().contiguous()
        nz, ny, nx = m0c.shape[1:]
        stream = torch.cuda.current_stream().cuda_stream
        c = llb.llb_create(nx, ny, nz, lattice, float(tau), _params(m0c.dtype, stream, cg))
        try:
            llb.llb_init_moments_device(c, m0c)
            llb.llb_step(c, nsteps)
            out = torch.empty_like(m0c)
            llb.llb_get_moments_device(c, out)
            llb.llb_synchronize(c)
        finally:
            llb.llb_destroy(c)
        ctx.save_for_backward(m0c)
        ctx.tau, ctx.nsteps, ctx.lattice, ctx.every, ctx.cg = float(tau), nsteps, lattice, every, cg
        ctx.tau_shape = tau.shape if isinstance(tau, torch.Tensor) else None
        return out

    @staticmethod
    def backward(ctx, gout):
        (m0c,) = ctx.saved_tensors
        nz, ny, nx = m0c.shape[1:]
        stream = torch.cuda.current_stream().cuda_stream
        c = llb.llb_create(nx, ny, nz, ctx.lattice, ctx.tau, _params(m0c.dtype, stream, ctx.cg))
        try:
            llb.llb_init_moments_device(c, m0c)
            ginit = torch.empty_like(m0c)
            dtau = llb.llb_adjoint(c, ctx.nsteps, gout.to(m0c.dtype).contiguous(), ginit, every=ctx.every)
        finally:
            llb.llb_destroy(c)
        gtau = None
        if ctx.tau_shape is not None:
            gtau = torch.full(ctx.tau_shape, dtau, dtype=torch.float64, device=m0c.device)
        return ginit, gtau, None, None, None, None


def evolve(m0: torch.Tensor, tau, nsteps: int, lattice: int = 19, every: int = 0,
           two_component: dict | None = None) -> torch.Tensor:
    """Differentiable nsteps moment-only steps of canonical moments m0 (see module doc)."""
    if not isinstance(tau, torch.Tensor):
        tau = torch.tensor(float(tau), dtype=torch.float64)
    cg = dict(two_component) if two_component is not None else None
    return MomentOnlyEvolve.apply(m0, tau, int(nsteps), int(lattice), int(every), cg)
