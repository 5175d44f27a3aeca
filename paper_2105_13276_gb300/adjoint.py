"""Differentiable DMR run: torch.autograd.Function over the C ABI.

Forward: a run with the given incident amplitude E0 and ionization scale
s_nu, seeded with a density map on the initial fine rectangle (on the coarse
mesh when r = 1), advanced n_steps with checkpoints every K steps; returns
the coarse density map at the end.  Backward: the library's hand-written
adjoint sweep (checkpoint restore, segment recompute onto a tape, reverse
kernels) with the refinement schedule of the forward held fixed.
"""
from __future__ import annotations

import torch

from . import dmr as D


class DMRDensity(torch.autograd.Function):
    @staticmethod
    def forward(ctx, E0, nu_scale, seed_map, cfg, rect, n_steps, K):
        c = dict(cfg, E0=float(E0), nu_scale=float(nu_scale))
        run = D.Run(c, device=seed_map.device)
        level = 0
        if c.get("r", 1) > 1:
            run.set_patch(rect)
            level = 1
        (rows, cols), _ = run.shape("n", level)
        if tuple(seed_map.shape) != (rows, cols):
            raise ValueError("seed map must be %r" % ((rows, cols),))
        dt = torch.float64 if run.fdtype.__name__ == "float64" else torch.float32
        sm = seed_map.detach().to(dt).contiguous()
        torch.cuda.current_stream(seed_map.device).synchronize()
        run.write_from("n", level, sm)
        ckpt = run.adjoint_record(n_steps, K)
        (rc, cc), _ = run.shape("n", 0)
        out = torch.empty((rc, cc), dtype=dt, device=seed_map.device)
        run.read_into("n", 0, out)
        run.sync()
        ctx.run, ctx.ckpt, ctx.dt = run, ckpt, dt
        ctx.seed_shape = tuple(seed_map.shape)
        ctx.seed_dtype = seed_map.dtype
        return out

    @staticmethod
    def backward(ctx, grad):
        run = ctx.run
        g = grad.detach().to(ctx.dt).contiguous()
        torch.cuda.current_stream(g.device).synchronize()
        dseed = torch.empty(ctx.seed_shape, dtype=ctx.dt, device=g.device)
        dE0, dnu = run.adjoint_backward(g, ctx.ckpt, dseed)
        run.sync()
        dev = g.device
        return (torch.tensor(dE0, dtype=torch.float64, device=dev),
                torch.tensor(dnu, dtype=torch.float64, device=dev),
                dseed.to(ctx.seed_dtype), None, None, None, None)


def dmr_density(E0, nu_scale, seed_map, cfg, rect, n_steps, K):
    """Coarse density at t_end as a differentiable function of (E0, s_nu,
    seed map)."""
    return DMRDensity.apply(E0, nu_scale, seed_map, cfg, rect, n_steps, K)
