"""The complete time loop: coarse Yee + embedded reduced models, FP64 oracle.

Paper, Sec. IV-C (end): "the proposed scheme consists of conventional FDTD
equations to update the coarse grid, and Eq. (23) to update the reduced model
state and the interface", applied to each reduced model.

One step n -> n+1 (a reading of the order, which the paper leaves implicit):
  1. coarse Hz^{n+1/2} from E^n (Eq. (5)); cells beside a region read the
     interface E (= y^n);
  2. probes record Hz^{n+1/2};
  3. coarse E^{n+1} on every edge that is not PEC, interface or inside a
     region (Eq. (3)), with the source current J(t^{n+1/2});
  4. every reduced model: [y; x~]^{n+1} = P [y; x~]^n + Q h^{n+1/2}
     (Eq. (23)); y^{n+1} is written to the interface edges.
Steps 3 and 4 touch disjoint unknowns and commute.

Sources are electric current densities J on E edges (the -area*J term of the
integral form of Ampere's law, Eq. (3)).  A source record is a dict
{comp: 0 (Jx) | 1 (Jy), i, j, len, wave}: ``len`` consecutive edges along the
edge direction starting at (i, j), all driven by wave[n] = J(t^{n+1/2}).
A probe (i, j) records Hz of coarse cell (i, j).
"""
from __future__ import annotations

import dataclasses
import numpy as np

from .yee import CoarseGrid, MU0
from .sprim import ReducedModel
from .couple import Coupled


@dataclasses.dataclass
class Embedded:
    """A reduced model placed in the coarse grid (its state is x~)."""
    itf_index: int           # index into CoarseGrid.interfaces
    P: np.ndarray
    Q: np.ndarray
    rom: ReducedModel        # for the storage function
    x: np.ndarray            # x~ = [x~_E^n; x~_H^{n-1/2}]

    @classmethod
    def from_coupled(cls, itf_index, cpl: Coupled, rom: ReducedModel):
        return cls(itf_index, cpl.P, cpl.Q, rom, np.zeros(rom.q))


@dataclasses.dataclass
class State:
    Ex: np.ndarray
    Ey: np.ndarray
    Hz: np.ndarray


def gather_y(grid: CoarseGrid, k: int, st: State) -> np.ndarray:
    itf = grid.interfaces[k]
    return np.where(itf.comp == 0, st.Ex[itf.ej, np.minimum(itf.ei, grid.nx - 1)],
                    st.Ey[np.minimum(itf.ej, grid.ny - 1), itf.ei])


def scatter_y(grid: CoarseGrid, k: int, st: State, y: np.ndarray):
    itf = grid.interfaces[k]
    mx = itf.comp == 0
    st.Ex[itf.ej[mx], itf.ei[mx]] = y[mx]
    st.Ey[itf.ej[~mx], itf.ei[~mx]] = y[~mx]


def source_edges(src):
    """The (comp, i, j) edges of one source record."""
    out = []
    for t in range(src.get("len", 1)):
        if src["comp"] == 0:
            out.append((0, src["i"] + t, src["j"]))
        else:
            out.append((1, src["i"], src["j"] + t))
    return out


def step(grid: CoarseGrid, st: State, roms, sources=(), n: int = 0, probes=None,
         out=None):
    """One step n -> n+1 of the scheme (module header).  A grid carrying a
    CPML (attribute ``pml``, oracle.cpml) takes its stretched updates."""
    pml = getattr(grid, "pml", None)
    st.Hz = pml.h_update(grid, st.Ex, st.Ey, st.Hz) if pml else grid.h_update(st.Ex, st.Ey, st.Hz)
    if probes is not None and len(probes):
        pi = np.array([p[0] for p in probes])
        pj = np.array([p[1] for p in probes])
        out[n] = st.Hz[pj, pi]
    y_old = [gather_y(grid, e.itf_index, st) for e in roms]
    st.Ex, st.Ey = pml.e_update(grid, st.Ex, st.Ey, st.Hz) if pml else grid.e_update(st.Ex, st.Ey, st.Hz)
    for src in sources:
        for (c, i, j) in source_edges(src):
            grid.add_current(st.Ex, st.Ey, c, i, j, src["wave"][n])
    for e, y in zip(roms, y_old):
        itf = grid.interfaces[e.itf_index]
        h = st.Hz[itf.hj, itf.hi]
        s = np.concatenate([y, e.x])
        s_new = e.P @ s + e.Q @ h
        scatter_y(grid, e.itf_index, st, s_new[: y.size])
        e.x = s_new[y.size:]


def run(grid: CoarseGrid, roms, nsteps: int, sources=(), probes=(), st: State = None,
        energy_every: int = 0):
    """March nsteps.  Returns (probe samples [nsteps, nprobe], state, energies)."""
    if st is None:
        st = State(*grid.zeros())
    out = np.zeros((nsteps, len(probes)))
    energies = []
    for n in range(nsteps):
        step(grid, st, roms, sources, n, probes, out)
        if energy_every and (n + 1) % energy_every == 0:
            energies.append(energy(grid, st, roms))
    return out, st, np.array(energies)


def coarse_energy(grid: CoarseGrid, st: State) -> float:
    """Storage function (dt/2) x^T R x of the coarse system with hanging
    variables, x = [E^n; H^{n-1/2}] (Sec. V-A, Appendix A):
        1/2 E^T D_eps E + 1/2 H^T D_mu H - dt/2 E^T K H,
    where interface edges carry the coarse half-cell area and material of
    Eq. (13) and their K row holds only the outside Hz (Eq. (14))."""
    dx, dy, dt = grid.dx, grid.dy, grid.dt
    area = dx * dy
    Ex, Ey, Hz = st.Ex, st.Ey, st.Hz
    W = 0.5 * np.sum(np.where(grid.hz_active, area * MU0 * Hz**2, 0.0))
    KHx = np.zeros_like(Ex)
    KHx[1:grid.ny] = dx * (Hz[1:] - Hz[:-1])
    KHy = np.zeros_like(Ey)
    KHy[:, 1:grid.nx] = -dy * (Hz[:, 1:] - Hz[:, :-1])
    W += np.sum(np.where(grid.ex_upd, 0.5 * area * grid.eps_x * Ex**2 - 0.5 * dt * Ex * KHx, 0.0))
    W += np.sum(np.where(grid.ey_upd, 0.5 * area * grid.eps_y * Ey**2 - 0.5 * dt * Ey * KHy, 0.0))
    for k, itf in enumerate(grid.interfaces):
        y = gather_y(grid, k, st)
        h = Hz[itf.hj, itf.hi]
        W += np.sum(0.5 * itf.length * itf.half * itf.eps_b * y**2
                    - 0.5 * dt * y * (itf.sign * itf.length * h))
    return float(W)


def energy(grid: CoarseGrid, st: State, roms) -> float:
    """Total storage function: coarse system + (dt/2) x~^T R~ x~ per model."""
    W = coarse_energy(grid, st)
    for e in roms:
        W += 0.5 * grid.dt * float(e.x @ (e.rom.R(grid.dt) @ e.x))
    return W


def fine_fields(e: Embedded, nxf: int, nyf: int):
    """Fine-region fields rebuilt from a model's state (Sec. III: the
    projection x_hat ~ V x~ with V = blkdiag(V1, V2)): Ex [nyf+1][nxf],
    Ey [nyf][nxf+1], Hz [nyf][nxf], the fine state order (all Ex, all Ey, Hz,
    each row-major).  Same time levels as the coarse fields: E^n, Hz^{n-1/2}."""
    r = e.rom
    xE = r.V1 @ e.x[:r.qE]
    xH = r.V2 @ e.x[r.qE:]
    nEx = nxf * (nyf + 1)
    return (xE[:nEx].reshape(nyf + 1, nxf), xE[nEx:].reshape(nyf, nxf + 1), xH.reshape(nyf, nxf))
