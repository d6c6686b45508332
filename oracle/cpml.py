"""Convolutional perfectly matched layer (CPML) for the coarse TEz grid,
FP64 oracle.

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline use this package.

The paper terminates its open structures with PML layers of a few coarse
cells (Sec. VI: the waveguide with irises, 10 cells; the rod reflection test,
15 mm) without stating the formulation.  This is the complex-frequency-shifted
convolutional PML of Roden and Gedney (Microwave Opt. Technol. Lett., 2000),
written from its published definition for the integral form of Eqs. (3), (5):
every spatial difference d/dx is replaced by (1/kappa_x) d/dx + psi_x, with

    psi_x^{n} = b_x psi_x^{n-1} + a_x (d/dx)^{n},
    b_x = exp(-(sigma_x/kappa_x + alpha_x) dt / eps0),
    a_x = sigma_x / (sigma_x kappa_x + kappa_x^2 alpha_x) (b_x - 1),

and likewise in y.  In a layer of n cells the profiles at depth rho in [0, 1]
(0 at the layer's inner face, 1 at the PEC wall behind it) are
sigma = sigma_max rho^m, kappa = 1 + (kappa_max - 1) rho^m,
alpha = alpha_max (1 - rho); outside the layers sigma = alpha = 0, kappa = 1,
so the update is Eqs. (3), (5) unchanged.  Each quantity is sampled where it
is used: Hz and Ex at x = (i + 1/2) dx, Ey at x = i dx (and in y, Hz and Ey
at (j + 1/2) dy, Ex at j dy).  Default sigma_max = 0.8 (m + 1) / (eta0 dx)
(the usual near-optimal choice for a polynomial grading in vacuum).
"""
from __future__ import annotations

import math

import numpy as np

from .yee import CoarseGrid, EPS0, MU0

SIDE_W, SIDE_E, SIDE_S, SIDE_N = 1, 2, 4, 8


def _depth(pos, n, extent, lo, hi):
    """Depth (in cells, 0..n) into the low-side and high-side layers of a
    coordinate pos (in cells) on [0, extent]."""
    d = np.zeros_like(pos, dtype=np.float64)
    if lo:
        d = np.maximum(d, n - pos)
    if hi:
        d = np.maximum(d, pos - (extent - n))
    return np.clip(d, 0.0, n)


class CPML:
    def __init__(self, grid: CoarseGrid, n: int, sides: int, m: float = 3.0, sigma_max: float = None,
                 kappa_max: float = 1.0, alpha_max: float = 0.0):
        self.n, self.sides = n, sides
        eta0 = math.sqrt(MU0 / EPS0)
        dt = grid.dt

        def coefs(pos, extent, lo, hi, h):
            smax = sigma_max if sigma_max is not None else 0.8 * (m + 1) / (eta0 * h)
            rho = _depth(pos, n, extent, lo, hi) / n
            inside = rho > 0
            sig = np.where(inside, smax * rho**m, 0.0)
            kap = np.where(inside, 1.0 + (kappa_max - 1.0) * rho**m, 1.0)
            alp = np.where(inside, alpha_max * (1.0 - rho), 0.0)
            b = np.exp(-(sig / kap + alp) * dt / EPS0)
            den = sig * kap + kap**2 * alp
            a = np.where(sig > 0, sig / np.where(den > 0, den, 1.0) * (b - 1.0), 0.0)
            return a, b, kap

        nx, ny = grid.nx, grid.ny
        W, E, S, N = sides & SIDE_W, sides & SIDE_E, sides & SIDE_S, sides & SIDE_N
        xc = np.arange(nx) + 0.5      # Hz, Ex
        xe = np.arange(nx + 1.0)      # Ey
        yc = np.arange(ny) + 0.5      # Hz, Ey
        ye = np.arange(ny + 1.0)      # Ex
        self.ax_h, self.bx_h, self.kx_h = coefs(xc, nx, W, E, grid.dx)
        self.ay_h, self.by_h, self.ky_h = coefs(yc, ny, S, N, grid.dy)
        self.ax_e, self.bx_e, self.kx_e = coefs(xe, nx, W, E, grid.dx)
        self.ay_e, self.by_e, self.ky_e = coefs(ye, ny, S, N, grid.dy)
        self.psi_hx = np.zeros((ny, nx))       # x-difference of Ey at Hz
        self.psi_hy = np.zeros((ny, nx))       # y-difference of Ex at Hz
        self.psi_ex = np.zeros((ny + 1, nx))   # y-difference of Hz at Ex
        self.psi_ey = np.zeros((ny, nx + 1))   # x-difference of Hz at Ey

    def h_update(self, grid: CoarseGrid, Ex, Ey, Hz):
        """Eq. (5) with stretched differences:
        Hz += dt/mu0 [ (1/ky) dEx/dy + psi_hy - (1/kx) dEy/dx - psi_hx ]."""
        dEx = (Ex[1:, :] - Ex[:-1, :]) / grid.dy
        dEy = (Ey[:, 1:] - Ey[:, :-1]) / grid.dx
        self.psi_hy = self.by_h[:, None] * self.psi_hy + self.ay_h[:, None] * dEx
        self.psi_hx = self.bx_h[None, :] * self.psi_hx + self.ax_h[None, :] * dEy
        Hn = Hz + grid.dt / MU0 * (dEx / self.ky_h[:, None] + self.psi_hy
                                   - dEy / self.kx_h[None, :] - self.psi_hx)
        return np.where(grid.hz_active, Hn, 0.0)

    def e_update(self, grid: CoarseGrid, Ex, Ey, Hz):
        """Eq. (3) with stretched differences, on updated edges:
        alpha Ex' = beta Ex + dx dy [ (1/ky) dHz/dy + psi_ex ],
        alpha Ey' = beta Ey - dx dy [ (1/kx) dHz/dx + psi_ey ]."""
        area = grid.dx * grid.dy
        dHy = np.zeros_like(Ex)
        dHy[1:grid.ny, :] = (Hz[1:, :] - Hz[:-1, :]) / grid.dy
        dHx = np.zeros_like(Ey)
        dHx[:, 1:grid.nx] = (Hz[:, 1:] - Hz[:, :-1]) / grid.dx
        self.psi_ex = np.where(grid.ex_upd, self.by_e[:, None] * self.psi_ex + self.ay_e[:, None] * dHy, 0.0)
        self.psi_ey = np.where(grid.ey_upd, self.bx_e[None, :] * self.psi_ey + self.ax_e[None, :] * dHx, 0.0)
        Exn = np.where(grid.ex_upd,
                       (grid.bx * Ex + area * (dHy / self.ky_e[:, None] + self.psi_ex)) / grid.ax, Ex)
        Eyn = np.where(grid.ey_upd,
                       (grid.by * Ey - area * (dHx / self.kx_e[None, :] + self.psi_ey)) / grid.ay, Ey)
        return Exn, Eyn
