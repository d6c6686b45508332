"""Direct subgridding stepper (full fine mesh, no MOR), FP64 oracle.

This is an independent route to the V = I case of the coupled scheme: instead
of the generalised inverse of A1 (Eqs. (19)-(23)), the fine leapfrog
(Eqs. (3)-(5), Eq. (6) with V = I) is stepped directly and the interface
equations are eliminated edge by edge.

For one coarse interface edge k with fine ports p in P(k) (r of them), write
each boundary equation as  alpha x^{n+1} = beta x^n + c + b u, where alpha,
beta are area * (eps/dt +- sigma/2) of the half cell, c the curl of the
already-updated H and b the hanging-variable coefficient (B of Eq. (6) for a
fine port, -Dl G^T of Eq. (14) for the coarse edge).  Since b_p = S_hat_p =
g_k / r with g_k = (Dl G^T)_k:

* paper rule (Eqs. (15)-(16)), E_hat_p = y_k for all p and U_k = mean(u_p):
  summing the r fine equations and the coarse one eliminates the hanging
  variables exactly:
      (alpha_k + sum_p alpha_p) y_k^{n+1}
          = beta_k y_k^n + g_k h_k + sum_p (beta_p E_p^n + c_p);
* dual rule, u_p = U_k for all p and y_k = mean(E_hat_p):
  E_p^{n+1} = (d_p + b_p U)/alpha_p with d_p = beta_p E_p^n + c_p; the coarse
  equation gives U = (beta_k y^n + g_k h - alpha_k y^{n+1}) / g_k, and the
  mean condition gives one scalar equation for y^{n+1}.
"""
from __future__ import annotations

import numpy as np

from .fine import FineSystem
from .yee import CoarseGrid, MU0
from .scheme import State, gather_y, scatter_y, source_edges
from .couple import PAPER, interface_blocks


class FineRegion:
    def __init__(self, grid: CoarseGrid, k: int, fs: FineSystem, T: np.ndarray, r: int,
                 rule: int = PAPER):
        self.k, self.fs, self.T, self.r, self.rule = k, fs, T, r, rule
        dt = grid.dt
        self.alpha = fs.d_eps / dt + fs.d_sig / 2
        self.beta = fs.d_eps / dt - fs.d_sig / 2
        self.E = np.zeros(fs.nE)
        self.H = np.zeros(fs.nH)
        Le = fs.L_E.tocoo()
        self.port_row = np.empty(fs.nu, dtype=int)
        self.port_row[Le.col] = Le.row
        self.b = fs.S_hat.copy()          # B entries of the ports (B = L S_hat)
        self.edge_of_port = np.argmax(T, axis=1)
        self.dplus, self.dminus, self.dlg = interface_blocks(grid.interfaces[k], dt)

    def energy(self, dt):
        fs = self.fs
        x = np.concatenate([self.E, self.H])
        return 0.5 * dt * float(x @ (fs.R(dt) @ x))


def step(grid: CoarseGrid, st: State, regions, sources=(), n=0, probes=None, out=None):
    dt = grid.dt
    st.Hz = grid.h_update(st.Ex, st.Ey, st.Hz)
    if probes is not None and len(probes):
        out[n] = st.Hz[[p[1] for p in probes], [p[0] for p in probes]]
    y_old = [gather_y(grid, reg.k, st) for reg in regions]
    st.Ex, st.Ey = grid.e_update(st.Ex, st.Ey, st.Hz)
    for src in sources:
        for (c, i, j) in source_edges(src):
            grid.add_current(st.Ex, st.Ey, c, i, j, src["wave"][n])
    for reg, y in zip(regions, y_old):
        fs = reg.fs
        itf = grid.interfaces[reg.k]
        h = st.Hz[itf.hj, itf.hi]
        # Fine H (Eq. (5)): D_mu/dt (H^{n+1/2} - H^{n-1/2}) = -K^T E^n.
        reg.H = reg.H - dt * (fs.K.T @ reg.E) / fs.d_mu
        # Fine E without hanging input (Eq. (3)); ports are redone below.
        c = fs.K @ reg.H
        d = reg.beta * reg.E + c
        E_new = d / reg.alpha
        pr = reg.port_row
        ny_ = y.size
        y_new = np.empty(ny_)
        if reg.rule == PAPER:
            num = reg.dminus * y + reg.dlg * h
            den = reg.dplus.copy()
            np.add.at(num, reg.edge_of_port, d[pr])
            np.add.at(den, reg.edge_of_port, reg.alpha[pr])
            y_new = num / den
            E_new[pr] = y_new[reg.edge_of_port]
        else:
            r = reg.r
            Aacc = np.zeros(ny_)
            Bacc = np.zeros(ny_)
            np.add.at(Aacc, reg.edge_of_port, d[pr] / reg.alpha[pr] / r)
            np.add.at(Bacc, reg.edge_of_port, reg.b / reg.alpha[pr] / r)
            g = reg.dlg
            rhs_c = reg.dminus * y + g * h
            y_new = (Aacc + Bacc * rhs_c / g) / (1.0 + Bacc * reg.dplus / g)
            U = (rhs_c - reg.dplus * y_new) / g
            E_new[pr] = (d[pr] + reg.b * U[reg.edge_of_port]) / reg.alpha[pr]
        reg.E = E_new
        scatter_y(grid, reg.k, st, y_new)


def run(grid: CoarseGrid, regions, nsteps, sources=(), probes=(), st=None):
    if st is None:
        st = State(*grid.zeros())
    out = np.zeros((nsteps, len(probes)))
    for n in range(nsteps):
        step(grid, st, regions, sources, n, probes, out)
    return out, st
