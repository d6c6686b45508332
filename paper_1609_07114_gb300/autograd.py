"""torch.autograd interface to ``fdtd_grad``.

``ProbeEnergy.apply(eps_r, sigma, waves, spec)`` returns the probe energy
J = sum_n sum_p Hz^{n+1/2}(p)^2 of one simulation whose coarse cells have the
given relative permittivity and conductivity, driven by the given source
waveforms; its backward pass returns dJ/deps_r, dJ/dsigma and dJ/dwaves from
the library's discrete adjoint (every step of both passes runs in the CUDA
library; this module only moves arguments).
"""
from __future__ import annotations

import dataclasses

import torch

from . import FdtdContext


@dataclasses.dataclass
class ProbeEnergySpec:
    dx: float
    dy: float
    dt: float
    nsteps: int
    sources: list          # dicts {comp, i, j, len} (waves passed separately)
    probes: list           # (i, j)
    roms: list = dataclasses.field(default_factory=list)   # (RomModel, i0, j0)
    ckpt_every: int = 500


class ProbeEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps_r, sigma, waves, spec: ProbeEnergySpec):
        c = FdtdContext(spec.dx, spec.dy, spec.dt,
                        [(eps_r.detach().double().cpu().numpy(), sigma.detach().double().cpu().numpy())])
        try:
            for (m, i0, j0) in spec.roms:
                c.rom_embed(m, 0, i0, j0)
            w = waves.detach().to(device="cuda", dtype=torch.float32).contiguous()
            src = [dict(s, sim=0, wave=w[k]) for k, s in enumerate(spec.sources)]
            J, ge, gs, gw = c.fdtd_grad(spec.nsteps, src, [(0, i, j) for i, j in spec.probes],
                                        spec.ckpt_every)
        finally:
            c.close()
        ctx.save_for_backward(ge[0].clone(), gs[0].clone(), gw.clone())
        ctx.dev = (eps_r.device, eps_r.dtype, sigma.device, sigma.dtype, waves.device, waves.dtype)
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        ge, gs, gw = ctx.saved_tensors
        de, te, ds, ts, dw, tw = ctx.dev
        g = float(gJ)
        return ((g * ge).to(de, te), (g * gs).to(ds, ts), (g * gw).to(dw, tw), None)
