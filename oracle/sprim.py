"""Structure-preserving model order reduction (SPRIM), FP64 oracle.

Paper, Sec. III: a block-Arnoldi Krylov basis V_hat is split into its E rows
and H rows, each block is orthonormalised separately, giving
V = blkdiag(V1, V2) (Eq. (9)), and the reduced model Eq. (11) is the
congruence R~ = V^T R V, F~ = V^T F V, B~ = V^T B, L~ = V^T L with R~ in the
block form of Eq. (12).

Readings (the paper does not print SPRIM's operator for a discrete-time
pencil, nor its deflation rule):

* With z the shift variable, Eq. (6) gives ((z-1) R + (z+1) F) X = B U, so with
  psi = (z-1)/(z+1) the transfer function is proportional to
  L^T (psi R + F)^{-1} B.  Moments are matched at a real expansion point
  psi0 = tan(pi f0 dt_b) (|psi| at frequency f0):
  Krylov space K_k((psi0 R + F)^{-1} R, (psi0 R + F)^{-1} B B_in).
* The basis is built at dt_b = min(dt, 0.99 * fine CFL limit) so that the
  operator exists whatever dt the model is run at; the reduced matrices are
  then formed from the dt-independent blocks (R11 = V1^T D_eps V1,
  Sigma = V1^T D_sigma V1, R22 = V2^T D_mu V2, K~ = V1^T K V2) at the run dt.
* The ROM order q counts both blocks: k = q/2 Krylov columns, so
  q_E = q_H = k unless a block loses rank.
* Deflation: within each block, columns come from the SVD of the block after
  two Gram-Schmidt passes against the basis so far; a direction is kept when
  its singular value exceeds tol times the block's largest singular value
  before orthogonalisation; columns are taken in order of decreasing singular
  value.  When the last block must be truncated to stay within k columns, the
  cut is moved down to the nearest gap in the singular values (relative gap
  above gap_tol), so that the kept subspace is uniquely defined even when a
  symmetric region gives equal singular values; the basis may then hold
  fewer than k columns.
* B_in selects the model inputs: the identity (all n_u fine hanging
  variables, Eq. (16)) or T (one input per coarse interface edge, the dual
  interpolation; see ``couple``).

A reduced model depends only on span(V1) and span(V2): a change of basis
inside either block is a congruence that leaves every input-output quantity
unchanged.
"""
from __future__ import annotations

import dataclasses
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .fine import FineSystem


@dataclasses.dataclass
class ReducedModel:
    """Eq. (11) with the blocks of Eq. (12) kept separately (dense)."""

    V1: np.ndarray        # (nE, qE)
    V2: np.ndarray        # (nH, qH)
    R11: np.ndarray       # V1^T D_eps V1
    R22: np.ndarray       # V2^T D_mu V2
    Kt: np.ndarray        # V1^T K V2   (possibly perturbed, Sec. V-E)
    Sig: np.ndarray       # V1^T D_sigma V1
    B_E: np.ndarray       # V1^T B_E    (qE, nu)
    L_E: np.ndarray       # V1^T L_E    (qE, nu)
    S_hat: np.ndarray     # (nu,)

    @property
    def qE(self):
        return self.R11.shape[0]

    @property
    def qH(self):
        return self.R22.shape[0]

    @property
    def q(self):
        return self.qE + self.qH

    def R(self, dt):
        """R~ of Eq. (12)."""
        return np.block([[self.R11 / dt, -0.5 * self.Kt],
                         [-0.5 * self.Kt.T, self.R22 / dt]])

    def F(self):
        """F~ = V^T F V."""
        return np.block([[self.Sig / 2, -0.5 * self.Kt],
                         [0.5 * self.Kt.T, np.zeros((self.qH, self.qH))]])

    def B(self):
        return np.vstack([self.B_E, np.zeros((self.qH, self.B_E.shape[1]))])

    def L(self):
        return np.vstack([self.L_E, np.zeros((self.qH, self.L_E.shape[1]))])


def project(fs: FineSystem, V1: np.ndarray, V2: np.ndarray) -> ReducedModel:
    """Congruence of Sec. III (Eqs. (11)-(12))."""
    K = fs.K
    return ReducedModel(
        V1=V1, V2=V2,
        R11=V1.T @ (fs.d_eps[:, None] * V1),
        R22=V2.T @ (fs.d_mu[:, None] * V2),
        Kt=V1.T @ (K @ V2),
        Sig=V1.T @ (fs.d_sig[:, None] * V1),
        B_E=V1.T @ fs.B_E.toarray(),
        L_E=V1.T @ fs.L_E.toarray(),
        S_hat=fs.S_hat.copy())


def full_order(fs: FineSystem) -> ReducedModel:
    """V = I: the fine model itself in reduced-model form (no MOR)."""
    return project(fs, np.eye(fs.nE), np.eye(fs.nH))


def block_arnoldi(apply_A, R0: np.ndarray, k: int, tol: float = 1e-12,
                  gap_tol: float = 1e-8) -> np.ndarray:
    """Orthonormal basis of K_k(A, R0) with SVD deflation (see module header)."""
    N = R0.shape[0]
    Q = np.zeros((N, 0))
    W = np.array(R0, dtype=np.float64)
    while Q.shape[1] < k:
        ref = np.linalg.norm(W, 2)
        if ref == 0.0:
            break
        for _ in range(2):
            W = W - Q @ (Q.T @ W)
        U, s, _ = np.linalg.svd(W, full_matrices=False)
        keep = int(np.sum(s > tol * ref))
        if keep == 0:
            break
        take = min(keep, k - Q.shape[1])
        if take < keep:
            while take > 0 and s[take - 1] - s[take] <= gap_tol * s[take - 1]:
                take -= 1
            if take == 0:
                break
        U = U[:, :take]
        Q = np.hstack([Q, U])
        if take < keep:
            break
        W = apply_A(U)
    return Q


def orth(X: np.ndarray, tol: float = 1e-12) -> np.ndarray:
    """Orthonormal basis of range(X): left singular vectors above tol*s_max."""
    U, s, _ = np.linalg.svd(X, full_matrices=False)
    if s.size == 0 or s[0] == 0.0:
        return U[:, :0]
    return U[:, : int(np.sum(s > tol * s[0]))]


def sprim(fs: FineSystem, q: int, dt_b: float, psi0: float, B_in: np.ndarray,
          tol: float = 1e-12) -> ReducedModel:
    """SPRIM reduction of the fine system to order <= q (Sec. III)."""
    k = q // 2
    Rb = fs.R(dt_b)
    M = (psi0 * Rb + fs.F()).tocsc()
    lu = spla.splu(M)
    R0 = lu.solve(np.asarray(fs.B() @ B_in, dtype=np.float64))

    def apply_A(X):
        return lu.solve(np.asarray(Rb @ X))

    Vhat = block_arnoldi(apply_A, R0, k, tol)
    V1 = orth(Vhat[: fs.nE], tol)
    V2 = orth(Vhat[fs.nE:], tol)
    return project(fs, V1, V2)
