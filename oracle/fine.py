"""Fine-region FDTD equations as a discrete-time descriptor system (oracle).

Paper, Sec. II:  Eqs. (3)-(5) are the integral-form updates; Eq. (6)
    (R + F) x^{n+1} = (R - F) x^n + B u^{n+1/2},   y^n = L^T x^n,
with x^n = [Ex^n; Ey^n; Hz^{n-1/2}] (Eq. (7)) and the ports
u = [H_S; H_N; H_W; H_E], y = [E_S; E_N; E_W; E_E] (Eq. (8)).

The explicit matrices are in a companion paper that is not reproduced; they
are reconstructed here from Eqs. (3)-(5) (a reading).  With E = [Ex; Ey],
H = Hz and

    D_eps, D_sigma : diag(edge area * eps), diag(edge area * sigma)
    D_mu           : diag(cell area * mu0)
    K              : the curl, entries +-dx_hat (Ex-Hz) and +-dy_hat (Ey-Hz),
                     so that the E row of Eq. (3) reads ... + (K H)

the leapfrog of Eqs. (3)-(5) is Eq. (6) with

    R = [[D_eps/dt, -K/2], [-K^T/2, D_mu/dt]],
    F = [[D_sigma/2, -K/2], [K^T/2, 0]],

so R + F = [[D_eps/dt + D_sigma/2, -K], [0, D_mu/dt]] and
R - F = [[D_eps/dt - D_sigma/2, 0], [-K^T, D_mu/dt]].  This matches the block
form printed for the reduced matrix in Eq. (12) (R11 = D_eps, R22 = D_mu).

Boundary E edges use the half-cell area inside the region and that half
cell's material (Eq. (4)); their curl takes the hanging variable as input.
B has entries -dx_hat (South), +dx_hat (North), +dy_hat (West), -dy_hat
(East) on the boundary E rows, and L selects the boundary E, so that
L^T B is exactly S_hat of Eq. (25).

Indexing (0-based): Ex[jh, ih] with ih < nxf, jh <= nyf (row-major, jh major);
Ey[jh, ih] with ih <= nxf, jh < nyf; Hz[jh, ih].  State order: all Ex, then
all Ey, then all Hz.
"""
from __future__ import annotations

import dataclasses
import numpy as np
import scipy.sparse as sp

from .yee import EPS0, MU0


@dataclasses.dataclass
class FineSystem:
    nxf: int
    nyf: int
    dxf: float
    dyf: float
    d_eps: np.ndarray      # (nE,)   diag of D_eps
    d_sig: np.ndarray      # (nE,)   diag of D_sigma
    d_mu: np.ndarray       # (nH,)   diag of D_mu
    K: sp.csr_matrix       # (nE, nH)
    B_E: sp.csr_matrix     # (nE, nu) E rows of B (H rows are zero)
    L_E: sp.csr_matrix     # (nE, nu) E rows of L (H rows are zero)
    S_hat: np.ndarray      # (nu,)   diag of S_hat, Eq. (25)

    @property
    def nE(self):
        return self.d_eps.size

    @property
    def nH(self):
        return self.d_mu.size

    @property
    def n(self):
        return self.nE + self.nH

    @property
    def nu(self):
        return self.S_hat.size

    def R(self, dt):
        """R of Eq. (6) (sparse)."""
        return sp.bmat([[sp.diags(self.d_eps / dt), -0.5 * self.K],
                        [-0.5 * self.K.T, sp.diags(self.d_mu / dt)]], format="csr")

    def F(self):
        """F of Eq. (6) (sparse)."""
        return sp.bmat([[sp.diags(self.d_sig / 2), -0.5 * self.K],
                        [0.5 * self.K.T, None]], format="csr", dtype=np.float64)

    def B(self):
        return sp.vstack([self.B_E, sp.csr_matrix((self.nH, self.nu))], format="csr")

    def L(self):
        return sp.vstack([self.L_E, sp.csr_matrix((self.nH, self.nu))], format="csr")


def state_size(nxf: int, nyf: int) -> int:
    """Size of x_hat in Eq. (7): Ex, Ey and Hz samples of the fine region."""
    return nxf * (nyf + 1) + (nxf + 1) * nyf + nxf * nyf


def assemble(nxf, nyf, dxf, dyf, eps_r, sigma) -> FineSystem:
    """Assemble D_eps, D_sigma, D_mu, K, B, L of the fine region (Sec. II)."""
    eps_r = np.asarray(eps_r, dtype=np.float64).reshape(nyf, nxf)
    sigma = np.asarray(sigma, dtype=np.float64).reshape(nyf, nxf)
    nEx = nxf * (nyf + 1)
    nEy = (nxf + 1) * nyf
    nE = nEx + nEy
    nH = nxf * nyf
    nu = 2 * (nxf + nyf)

    def iex(ih, jh):
        return jh * nxf + ih

    def iey(ih, jh):
        return nEx + jh * (nxf + 1) + ih

    def ihz(ih, jh):
        return jh * nxf + ih

    d_eps = np.zeros(nE)
    d_sig = np.zeros(nE)
    rows, cols, vals = [], [], []
    brow, bcol, bval = [], [], []
    lrow, lcol = [], []
    area = dxf * dyf
    # Ex edges: Eq. (3) inside, Eq. (4) (and its North twin) on the boundary.
    for jh in range(nyf + 1):
        for ih in range(nxf):
            r = iex(ih, jh)
            if jh == 0:
                e, s, ar = eps_r[0, ih], sigma[0, ih], area / 2
            elif jh == nyf:
                e, s, ar = eps_r[nyf - 1, ih], sigma[nyf - 1, ih], area / 2
            else:
                e = 0.5 * (eps_r[jh - 1, ih] + eps_r[jh, ih])
                s = 0.5 * (sigma[jh - 1, ih] + sigma[jh, ih])
                ar = area
            d_eps[r] = ar * EPS0 * e
            d_sig[r] = ar * s
            if jh < nyf:            # + dx_hat Hz above
                rows.append(r); cols.append(ihz(ih, jh)); vals.append(+dxf)
            if jh > 0:              # - dx_hat Hz below
                rows.append(r); cols.append(ihz(ih, jh - 1)); vals.append(-dxf)
    # Ey edges.
    for jh in range(nyf):
        for ih in range(nxf + 1):
            r = iey(ih, jh)
            if ih == 0:
                e, s, ar = eps_r[jh, 0], sigma[jh, 0], area / 2
            elif ih == nxf:
                e, s, ar = eps_r[jh, nxf - 1], sigma[jh, nxf - 1], area / 2
            else:
                e = 0.5 * (eps_r[jh, ih - 1] + eps_r[jh, ih])
                s = 0.5 * (sigma[jh, ih - 1] + sigma[jh, ih])
                ar = area
            d_eps[r] = ar * EPS0 * e
            d_sig[r] = ar * s
            if ih < nxf:            # - dy_hat Hz to the right
                rows.append(r); cols.append(ihz(ih, jh)); vals.append(-dyf)
            if ih > 0:              # + dy_hat Hz to the left
                rows.append(r); cols.append(ihz(ih - 1, jh)); vals.append(+dyf)
    K = sp.csr_matrix((vals, (rows, cols)), shape=(nE, nH))
    # Ports in the order of Eq. (8): S, N, W, E.
    p = 0
    for ih in range(nxf):           # South: hanging Hz below Ex(ih, 0)
        brow.append(iex(ih, 0)); bcol.append(p); bval.append(-dxf)
        lrow.append(iex(ih, 0)); lcol.append(p); p += 1
    for ih in range(nxf):           # North: hanging Hz above Ex(ih, nyf)
        brow.append(iex(ih, nyf)); bcol.append(p); bval.append(+dxf)
        lrow.append(iex(ih, nyf)); lcol.append(p); p += 1
    for jh in range(nyf):           # West: hanging Hz left of Ey(0, jh)
        brow.append(iey(0, jh)); bcol.append(p); bval.append(+dyf)
        lrow.append(iey(0, jh)); lcol.append(p); p += 1
    for jh in range(nyf):           # East: hanging Hz right of Ey(nxf, jh)
        brow.append(iey(nxf, jh)); bcol.append(p); bval.append(-dyf)
        lrow.append(iey(nxf, jh)); lcol.append(p); p += 1
    B_E = sp.csr_matrix((bval, (brow, bcol)), shape=(nE, nu))
    L_E = sp.csr_matrix((np.ones(nu), (lrow, lcol)), shape=(nE, nu))
    S_hat = np.concatenate([np.full(nxf, -dxf), np.full(nxf, dxf),
                            np.full(nyf, dyf), np.full(nyf, -dyf)])
    d_mu = np.full(nH, area * MU0)
    return FineSystem(nxf, nyf, dxf, dyf, d_eps, d_sig, d_mu, K, B_E, L_E, S_hat)


def interpolation_T(a: int, b: int, r: int) -> np.ndarray:
    """T of Eq. (15): n_u x n_y, T[p, k] = 1 when fine port p lies on coarse
    interface edge k (both ordered S, N, W, E)."""
    nxf, nyf = r * a, r * b
    nu, ny_ = 2 * (nxf + nyf), 2 * (a + b)
    T = np.zeros((nu, ny_))
    p = 0
    for side, (nf, off) in enumerate([(nxf, 0), (nxf, a), (nyf, 2 * a), (nyf, 2 * a + b)]):
        for f in range(nf):
            T[p, off + f // r] = 1.0
            p += 1
    return T
