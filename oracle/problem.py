"""Builds and runs a complete oracle problem from a workload record (FP64).

Per reduced-model region (Secs. III-V):
  1. assemble the fine system (Sec. II);
  2. SPRIM at dt_b = min(dt, 0.99 * fine CFL limit of Eq. (1)), expansion
     point psi0 = tan(pi f0 dt_b), inputs B_in = I (paper rule) or T (dual);
     order 0 means no reduction (V = I);
  3. if any singular value of Eq. (27) exceeds gamma * 2/dt, clamp it
     (Sec. V-E);
  4. couple to the coarse grid at the run dt (Sec. IV, Eq. (23)).
"""
from __future__ import annotations

import dataclasses
import numpy as np

from . import cpml, fine, sprim, passivity, couple, scheme
from .yee import CoarseGrid, cfl_limit


@dataclasses.dataclass
class BuiltROM:
    rom: sprim.ReducedModel
    cpl: couple.Coupled
    s_before: np.ndarray
    s_after: np.ndarray
    T: np.ndarray
    fs: fine.FineSystem


def build_rom(rd, grid: CoarseGrid, k: int, rule=couple.DUAL, gamma=0.99, tol=1e-12,
              order=None) -> BuiltROM:
    r = rd["r"]
    a, b = rd["a"], rd["b"]
    dt = grid.dt
    fs = fine.assemble(r * a, r * b, grid.dx / r, grid.dy / r, rd["eps_r"], rd["sigma"])
    T = fine.interpolation_T(a, b, r)
    q = rd["q"] if order is None else order
    if q == 0:
        rom = sprim.full_order(fs)
    else:
        dt_b = min(dt, 0.99 * cfl_limit(grid.dx / r, grid.dy / r))
        psi0 = np.tan(np.pi * rd["f0"] * dt_b)
        B_in = np.eye(fs.nu) if rule == couple.PAPER else T
        rom = sprim.sprim(fs, q, dt_b, psi0, B_in, tol)
    s = passivity.singular_values_27(rom)
    s_after = s
    if s.size and s[0] > gamma * 2.0 / dt:
        rom, s, s_after = passivity.extend_cfl(rom, dt, gamma)
    cpl = couple.couple(grid.interfaces[k], rom, T, r, dt, rule)
    return BuiltROM(rom, cpl, s, s_after, T, fs)


def make_grid(w) -> CoarseGrid:
    regions = [(rd["i0"], rd["j0"], rd["a"], rd["b"]) for rd in w["roms"]]
    grid = CoarseGrid(w["nx"], w["ny"], w["dx"], w["dy"], w["dt"], w["eps_r"], w["sigma"],
                      regions)
    if w.get("pml"):
        p = w["pml"]
        grid.pml = cpml.CPML(grid, p["n"], p["sides"], p.get("m", 3.0), p.get("sigma_max"),
                             p.get("kappa_max", 1.0), p.get("alpha_max", 0.0))
    return grid


def build(w, rule=couple.DUAL, gamma=0.99, order=None):
    grid = make_grid(w)
    built = [build_rom(rd, grid, k, rule, gamma, order=order) for k, rd in enumerate(w["roms"])]
    emb = [scheme.Embedded.from_coupled(k, b.cpl, b.rom) for k, b in enumerate(built)]
    return grid, emb, built


def run(w, nsteps=None, rule=couple.DUAL, gamma=0.99, order=None):
    grid, emb, built = build(w, rule, gamma, order)
    n = w["nsteps"] if nsteps is None else nsteps
    out, st, _ = scheme.run(grid, emb, n, w["sources"], w["probes"])
    return out, st, grid, emb, built
