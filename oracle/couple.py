"""Coupling of a reduced model to the coarse grid, FP64 oracle.

Paper, Sec. IV:
* Eq. (14): the coarse interface E (vector y) obeys
      Dl Dl' (Deps_b/dt + Dsig_b/2) y^{n+1} = Dl Dl' (Deps_b/dt - Dsig_b/2) y^n
                                             + Dl G^T H^{n+1/2} - Dl G^T U^{n+1/2};
* Eqs. (15)-(16), the interpolation rule:  y_hat = T y,  U = (1/r) T^T u_hat;
* Eqs. (19)-(22): the combined system A1 z^{n+1} = A2 z^n + [Dl G^T H; 0; 0]
  with z = [y; u_hat^{n-1/2}; x~];
* Eq. (23): z^{n+1} = A1^{-1} A2 z^n + A1^{-1} Dl G^T [H; 0; 0], precomputed
  once.  Only the y and x~ rows are needed at run time, and A2's u_hat column
  is zero, so the run-time map is
      [y; x~]^{n+1} = P [y; x~]^n + Q h^{n+1/2}.

Readings:
* "[H; 0; 0]" in Eqs. (19) and (23) has the wrong size as printed; the forcing
  Dl G^T H enters the y rows only.
* Sign of G per side: see ``yee.Interface`` (S -1, N +1, W +1, E -1).  With
  it, Dl G^T = T^T S_hat T, i.e. the coarse and fine supply rates cancel and
  the interpolation is lossless (Sec. V-A).
* A1 may be singular.  In Eq. (19) the y_hat = T y constraint has n_u rows
  but only n_y + q_E unknowns behind it; when n_y + q_E < n_u (every reduced
  order below the port count) A1 has a null space.  The solution for y and x~
  is still unique (the null directions of u_hat leave T^T u_hat and
  L~ S_hat u_hat unchanged), so Eq. (23) is evaluated with a generalised
  inverse of the equilibrated A1, and the result is checked for consistency
  and for independence from the rank threshold.
* When range(T) is not contained in range(L_E~^T) the constraint forces
  y = 0: the region then acts as a PEC box (stable, but the coupling is
  void).  ``interface_deficiency`` measures this.  For reduced orders the
  dual interpolation, equally lossless, is available:
      y = (1/r) T^T y_hat,   u_hat = T U,
  with z = [y; U; x~] and
      A1 = [[Dy+, Dl G^T, 0], [I, 0, -(1/r) T^T L~^T], [0, -B~ T, R~ + F~]],
  which is nonsingular for any order.
"""
from __future__ import annotations

import dataclasses
import numpy as np

from .sprim import ReducedModel
from .yee import Interface

PAPER = 0   # Eqs. (15)-(16)
DUAL = 1    # y = (1/r) T^T y_hat, u_hat = T U


@dataclasses.dataclass
class Coupled:
    P: np.ndarray            # (n_y + q, n_y + q)
    Q: np.ndarray            # (n_y + q, n_y)
    A1: np.ndarray
    A2: np.ndarray
    forcing: np.ndarray      # (rows of A1, n_y): Dl G^T placed in the y rows
    residual: float          # consistency residual of the generalised solve
    threshold_change: float  # max change of [P Q] when the rank threshold moves x100


def interface_blocks(itf: Interface, dt: float):
    """Diagonals of Dl Dl' (Deps_b/dt +- Dsig_b/2) and Dl G^T (Eq. (14))."""
    lh = itf.length * itf.half
    dplus = lh * (itf.eps_b / dt + itf.sig_b / 2)
    dminus = lh * (itf.eps_b / dt - itf.sig_b / 2)
    dlg = itf.sign * itf.length
    return dplus, dminus, dlg


def assemble_A(itf: Interface, rom: ReducedModel, T: np.ndarray, r: int, dt: float,
               rule: int = PAPER):
    """A1, A2 of Eqs. (21)-(22) (PAPER) or of the dual rule, and the forcing."""
    dplus, dminus, dlg = interface_blocks(itf, dt)
    ny_ = dplus.size
    q = rom.q
    Rt, Ft, Bt, Lt = rom.R(dt), rom.F(), rom.B(), rom.L()
    if rule == PAPER:
        nu = T.shape[0]
        A1 = np.block([
            [np.diag(dplus), (1.0 / r) * (dlg[:, None] * T.T), np.zeros((ny_, q))],
            [T, np.zeros((nu, nu)), -Lt.T],
            [np.zeros((q, ny_)), -Bt, Rt + Ft]])
        nmid = nu
    else:
        A1 = np.block([
            [np.diag(dplus), np.diag(dlg), np.zeros((ny_, q))],
            [np.eye(ny_), np.zeros((ny_, ny_)), -(1.0 / r) * (T.T @ Lt.T)],
            [np.zeros((q, ny_)), -(Bt @ T), Rt + Ft]])
        nmid = ny_
    n = ny_ + nmid + q
    A2 = np.zeros((n, n))
    A2[:ny_, :ny_] = np.diag(dminus)
    A2[ny_ + nmid:, ny_ + nmid:] = Rt - Ft
    forcing = np.zeros((n, ny_))
    forcing[:ny_, :] = np.diag(dlg)
    return A1, A2, forcing, nmid


def _gen_solve(A, Bm, rcond):
    """A generalised-inverse solve of A X = Bm after row/column equilibration."""
    dr = 1.0 / np.maximum(np.abs(A).max(axis=1), 1e-300)
    As = dr[:, None] * A
    dc = 1.0 / np.maximum(np.abs(As).max(axis=0), 1e-300)
    As = As * dc[None, :]
    X = np.linalg.pinv(As, rcond=rcond) @ (dr[:, None] * Bm)
    return dc[:, None] * X


def couple(itf: Interface, rom: ReducedModel, T: np.ndarray, r: int, dt: float,
           rule: int = PAPER, rcond: float = 1e-13) -> Coupled:
    """Precompute the run-time map of Eq. (23)."""
    A1, A2, forcing, nmid = assemble_A(itf, rom, T, r, dt, rule)
    ny_ = forcing.shape[1]
    q = rom.q
    rhs = np.hstack([A2, forcing])
    X = _gen_solve(A1, rhs, rcond)
    X2 = _gen_solve(A1, rhs, rcond * 100)
    keep = np.r_[0:ny_, ny_ + nmid: ny_ + nmid + q]
    # Consistency: A1 X must reproduce the right-hand side.
    res = np.linalg.norm(A1 @ X - rhs) / max(np.linalg.norm(rhs), 1e-300)
    M = X[keep]
    M2 = X2[keep]
    change = np.linalg.norm(M - M2) / max(np.linalg.norm(M), 1e-300)
    P = M[:, keep]
    Q = M[:, A2.shape[1]:]
    return Coupled(P, Q, A1, A2, forcing, float(res), float(change))


def interface_deficiency(rom: ReducedModel, T: np.ndarray) -> float:
    """Largest sine of the principal angles between range(T) and
    range(L_E~^T) (= the boundary rows of V1).  0 means every coarse
    interface field can be matched by the reduced model (Eq. (18))."""
    Pe = rom.L_E.T                     # (nu, qE)
    Qt, _ = np.linalg.qr(T)
    U, s, _ = np.linalg.svd(Pe, full_matrices=False)
    Ub = U[:, s > 1e-12 * max(s[0], 1e-300)] if s.size else U[:, :0]
    resid = Qt - Ub @ (Ub.T @ Qt)
    return float(np.linalg.norm(resid, 2))
