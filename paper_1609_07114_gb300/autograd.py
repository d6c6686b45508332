"""torch.autograd interface to the library's time march and discrete adjoint.

``FdtdFn.apply(eps_r, sigma, waves, spec)`` returns the probe samples
Hz^{n+1/2} of B simulations of one grid size:
  eps_r, sigma  [B, ny, nx] (or [ny, nx] for one simulation): per-cell
                relative permittivity and conductivity (S/m);
  waves         [B, S, nsteps] (or [S, nsteps]): the samples J(t^{n+1/2}) of
                each simulation's S sources;
  returns       [B, nsteps, P] (or [nsteps, P]) CUDA float32, P probes per
                simulation.
The forward pass is one ``fdtd_run`` (no reverse sweep).  The backward pass
receives dL/dprobes for whatever loss L the caller forms and returns dL/deps_r,
dL/dsigma and dL/dwaves from ``fdtd_vjp``: a checkpointed forward pass and the
exact discrete adjoint seeded with dL/dprobes.  Cells covered by a reduced
model get gradient 0; the cells just outside one include their role in the
coupling of Eq. (19).  Every step of both passes runs in the CUDA library;
this module only moves arguments.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import FdtdContext


@dataclasses.dataclass
class FdtdSpec:
    """What stays fixed between calls.  sources, probes and roms are given per
    simulation as a list of B lists, or as one flat list that every simulation
    uses: sources dicts {comp, i, j, len} (their samples come from `waves`),
    probes (i, j) tuples, roms (RomModel, i0, j0) tuples."""
    dx: float
    dy: float
    dt: float
    nsteps: int
    sources: list
    probes: list
    roms: list = dataclasses.field(default_factory=list)
    ckpt_every: int = 500


def _per_sim(x, B):
    if x and isinstance(x[0], list):
        if len(x) != B:
            raise ValueError(f"per-simulation list of length {len(x)} for {B} simulations")
        return x
    return [x] * B


def _context(spec, eps, sig):
    c = FdtdContext(spec.dx, spec.dy, spec.dt, [(eps[b], sig[b]) for b in range(eps.shape[0])])
    for b, roms in enumerate(_per_sim(spec.roms, eps.shape[0])):
        for (m, i0, j0) in roms:
            c.rom_embed(m, b, i0, j0)
    return c


def _tables(spec, B, waves):
    srcl, prbl = _per_sim(spec.sources, B), _per_sim(spec.probes, B)
    S, P = len(srcl[0]), len(prbl[0])
    if any(len(s) != S for s in srcl) or any(len(p) != P for p in prbl):
        raise ValueError("every simulation needs the same number of sources and of probes")
    srcs = [dict(s, sim=b, wave=waves[b, k]) for b in range(B) for k, s in enumerate(srcl[b])]
    probes = [(b, i, j) for b in range(B) for (i, j) in prbl[b]]
    return srcs, probes, S, P


def _host(t):
    return np.ascontiguousarray(t.detach().to("cpu", torch.float64).numpy())


class FdtdFn(torch.autograd.Function):
    vjp_calls = 0     # reverse sweeps run (backward passes)

    @staticmethod
    def forward(ctx, eps_r, sigma, waves, spec: FdtdSpec):
        single = eps_r.dim() == 2
        eps = _host(eps_r).reshape(-1, *eps_r.shape[-2:])
        sig = _host(sigma).reshape(eps.shape)
        B = eps.shape[0]
        w = waves.detach().to("cuda", torch.float32).reshape(B, -1, waves.shape[-1]).contiguous()
        if w.shape[-1] < spec.nsteps:
            raise ValueError("waves hold fewer samples than spec.nsteps")
        srcs, probes, S, P = _tables(spec, B, w)
        if w.shape[1] != S:
            raise ValueError(f"waves hold {w.shape[1]} sources per simulation, spec {S}")
        out = torch.empty((spec.nsteps, B * P), dtype=torch.float32, device="cuda")
        c = _context(spec, eps, sig)
        try:
            c.fdtd_run(spec.nsteps, srcs, probes, out)
        finally:
            c.close()
        ctx.save_for_backward(eps_r, sigma, waves)
        ctx.spec = spec
        res = out.view(spec.nsteps, B, P).permute(1, 0, 2).contiguous()
        return res[0] if single else res

    @staticmethod
    def backward(ctx, g):
        eps_r, sigma, waves = ctx.saved_tensors
        spec = ctx.spec
        eps = _host(eps_r).reshape(-1, *eps_r.shape[-2:])
        sig = _host(sigma).reshape(eps.shape)
        B = eps.shape[0]
        w = waves.detach().to("cuda", torch.float32).reshape(B, -1, waves.shape[-1]).contiguous()
        srcs, probes, S, P = _tables(spec, B, w)
        cot = g.detach().to("cuda", torch.float32).reshape(B, spec.nsteps, P).permute(1, 0, 2).contiguous()
        c = _context(spec, eps, sig)
        try:
            ge, gs, gw = c.fdtd_vjp(spec.nsteps, srcs, probes, cot.view(spec.nsteps, B * P), spec.ckpt_every,
                                    need_src=ctx.needs_input_grad[2])
        finally:
            c.close()
        FdtdFn.vjp_calls += 1
        d_eps = torch.stack(ge).reshape(eps_r.shape).to(eps_r.device, eps_r.dtype)
        d_sig = torch.stack(gs).reshape(sigma.shape).to(sigma.device, sigma.dtype)
        d_w = None
        if ctx.needs_input_grad[2]:
            gfull = torch.zeros((B * S, waves.shape[-1]), dtype=torch.float32, device="cuda")
            gfull[:, :spec.nsteps] = gw
            d_w = gfull.reshape(waves.shape).to(waves.device, waves.dtype)
        return d_eps, d_sig, d_w, None


def probe_energy(eps_r, sigma, waves, spec: FdtdSpec):
    """J = sum over steps and probes of Hz^2 (per call, all simulations), as a
    differentiable scalar."""
    return (FdtdFn.apply(eps_r, sigma, waves, spec).double() ** 2).sum()
