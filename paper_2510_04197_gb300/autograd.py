"""torch.autograd.Function over the CUDA time step and its hand-written adjoint.

    rho_n, T_n = DVBMFunction.apply(rho0, ux0, uy0, T0, params, nsteps, options)

params = tensor([mu, Pr, gamma]) (float64).  The forward creates a context with
those parameters on the current device and stream, records checkpoints every
ceil(sqrt(nsteps)) steps, applies the equilibrium initial condition and runs
nsteps steps; the backward calls dvbm_adjoint (recompute of each checkpoint
segment, then the adjoint steps).  dt is fixed by the CFL rule at the initial
fields (or options["dt"]) and is not differentiated.  FP64 storage, periodic
domain.
"""
from __future__ import annotations

import math

import torch

from . import dvbm


class DVBMFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho0, ux0, uy0, T0, params, nsteps: int, options: dict | None = None):
        opts = dict(options or {})
        Ny, Nx = rho0.shape
        mu, Pr, gamma = [float(v) for v in params.detach().cpu()]
        sim = dvbm.Simulation(Nx, Ny, Pr, gamma, mu, **opts)
        sim.record(max(1, int(math.ceil(math.sqrt(max(nsteps, 1))))))
        sim.init(rho0.detach(), ux0.detach(), uy0.detach(), T0.detach())
        sim.step(int(nsteps))
        m = sim.moments()
        ctx.sim = sim
        # gradients go back on the devices and dtypes of the inputs
        ctx.like = [(t.device, t.dtype) for t in (rho0, ux0, uy0, T0, params)]
        return m["rho"], m["T"]

    @staticmethod
    def backward(ctx, g_rho, g_T):
        sim = ctx.sim
        if sim is None:
            raise RuntimeError("DVBMFunction supports one backward pass per forward: its recorded run "
                               "is released after the adjoint")
        g = sim.adjoint(g_rho.contiguous() if g_rho is not None else None,
                        g_T.contiguous() if g_T is not None else None)
        gp = torch.tensor([g["mu"], g["Pr"], g["gamma"]], dtype=torch.float64)
        sim.close()
        ctx.sim = None
        out = [g["rho0"], g["ux0"], g["uy0"], g["T0"], gp]
        out = [t.to(device=dev, dtype=dt) for t, (dev, dt) in zip(out, ctx.like)]
        return (*out, None, None)


def run(rho0, ux0, uy0, T0, params, nsteps, **options):
    return DVBMFunction.apply(rho0, ux0, uy0, T0, params, nsteps, options)
