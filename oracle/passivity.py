"""Passivity conditions and CFL-limit extension, FP64 oracle.

Paper, Sec. V-B/V-C: a model of the form of Eq. (6) is passive when
    R = R^T > 0                (Eq. (24a) / (26a): generalised CFL),
    F + F^T >= 0               (Eq. (24b) / (26b): sigma >= 0),
    B = L S_hat                (Eq. (24c) / (26c)), S_hat of Eq. (25).
Theorem 1: the congruence of Sec. III with a full-rank block-diagonal V
preserves all three.

Sec. V-E, Eq. (27): R~ > 0 holds exactly when every singular value s_k of
R11^{-1/2} K~ R22^{-1/2} is below 2/dt.  The perturbation that enforces it is
"the method of" a reference that is not reproduced; the reading used here:
take the SVD  R11^{-1/2} K~ R22^{-1/2} = U diag(s) W^T  (symmetric square
roots), clamp s_k' = min(s_k, gamma * 2/dt) with a margin gamma < 1, and
rebuild K~' = R11^{1/2} U diag(s') W^T R22^{1/2}.  K~' replaces K~ in both R~
and F~, which keeps R~ + F~ block upper-triangular (an explicit leapfrog).
"""
from __future__ import annotations

import dataclasses
import numpy as np

from .sprim import ReducedModel


def sym_pow(A: np.ndarray, p: float) -> np.ndarray:
    """A^p for a symmetric positive definite A (eigendecomposition)."""
    w, Q = np.linalg.eigh(0.5 * (A + A.T))
    return (Q * w**p) @ Q.T


def singular_values_27(rom: ReducedModel) -> np.ndarray:
    """s_k of Eq. (27), in decreasing order."""
    M = sym_pow(rom.R11, -0.5) @ rom.Kt @ sym_pow(rom.R22, -0.5)
    return np.linalg.svd(M, compute_uv=False)


@dataclasses.dataclass
class PassivityReport:
    min_eig_R: float          # smallest eigenvalue of R (Eq. (26a))
    min_eig_FFt: float        # smallest eigenvalue of F + F^T (Eq. (26b))
    cond3_residual: float     # ||B - L S_hat|| / ||B|| (Eq. (26c))

    def passive(self, rtol: float = 1e-13) -> bool:
        return self.min_eig_R > 0 and self.min_eig_FFt >= -rtol and self.cond3_residual <= rtol


def check(R: np.ndarray, F: np.ndarray, B: np.ndarray, L: np.ndarray,
          S_hat: np.ndarray) -> PassivityReport:
    """Evaluate Eq. (26a)-(26c) (dense)."""
    eR = np.linalg.eigvalsh(0.5 * (R + R.T))
    FF = F + F.T
    eF = np.linalg.eigvalsh(FF)
    scale_F = max(np.abs(FF).max(), 1e-300)
    nb = max(np.linalg.norm(B), 1e-300)
    return PassivityReport(float(eR[0] / max(abs(eR[-1]), 1e-300)),
                           float(eF[0] / scale_F),
                           float(np.linalg.norm(B - L * S_hat[None, :]) / nb))


def extend_cfl(rom: ReducedModel, dt: float, gamma: float = 0.99):
    """Sec. V-E: clamp the singular values of Eq. (27) to gamma * 2/dt.

    Returns (perturbed model, s_before, s_after)."""
    r11h = sym_pow(rom.R11, 0.5)
    r22h = sym_pow(rom.R22, 0.5)
    M = sym_pow(rom.R11, -0.5) @ rom.Kt @ sym_pow(rom.R22, -0.5)
    U, s, Wt = np.linalg.svd(M, full_matrices=False)
    s_new = np.minimum(s, gamma * 2.0 / dt)
    Kp = r11h @ (U * s_new) @ Wt @ r22h
    out = dataclasses.replace(rom, Kt=Kp)
    return out, s, s_new
