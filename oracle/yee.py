"""Coarse-grid 2D TEz Yee scheme, FP64 (oracle; test infrastructure only).

Paper: Sec. I, Eq. (1) (CFL limit); Sec. II-A, Eqs. (3) and (5) (integral-form
E and H updates, written there for the fine mesh and used unchanged, with the
coarse cell sizes, for the coarse mesh); Sec. IV-A, Eq. (13) (coarse half-cell
update at a reduced-model interface).

Indexing (a reading: the paper numbers nodes from 1 and uses half-integer
field indices; here everything is 0-based):

* cell (i, j), i in [0, nx), j in [0, ny); Hz[j, i] at the cell centre;
* Ex[j, i] on the x-directed edge from node (i, j) to (i+1, j), shape (ny+1, nx);
* Ey[j, i] on the y-directed edge from node (i, j) to (i, j+1), shape (ny, nx+1).

Edge material (Sec. II-A: eps_x, sigma_x are averages over the edge): the
arithmetic mean of the two cells that share the edge.  The outer boundary is a
perfect electric conductor: tangential E on it stays 0.

A reduced-model region occupies coarse cells [i0, i0+a) x [j0, j0+b).  Inside
it the coarse grid has no unknowns.  The coarse E on its boundary ("interface
edges", the vector y of Eq. (14)) is owned by the reduced model's update
(Eq. (23)); the coarse grid only reads it.
"""
from __future__ import annotations

import dataclasses
import numpy as np

# CODATA 2018 constants (the paper does not print them).
EPS0 = 8.8541878128e-12
MU0 = 1.25663706212e-6
C0 = 1.0 / np.sqrt(EPS0 * MU0)


def cfl_limit(dx: float, dy: float, c: float = C0) -> float:
    """Eq. (1): dt < 1 / (c sqrt(1/dx^2 + 1/dy^2))."""
    return 1.0 / (c * np.sqrt(1.0 / dx**2 + 1.0 / dy**2))


def edge_materials(eps_r: np.ndarray, sigma: np.ndarray):
    """Absolute eps (F/m) and sigma (S/m) on Ex and Ey edges.

    Interior edge: mean of the two adjacent cells (Sec. II-A).  Outer-boundary
    edges take their single adjacent cell (they are PEC and never updated).
    """
    ny, nx = eps_r.shape
    e = EPS0 * np.asarray(eps_r, dtype=np.float64)
    s = np.asarray(sigma, dtype=np.float64)
    eps_x = np.empty((ny + 1, nx))
    sig_x = np.empty((ny + 1, nx))
    eps_x[1:ny] = 0.5 * (e[:-1] + e[1:])
    sig_x[1:ny] = 0.5 * (s[:-1] + s[1:])
    eps_x[0], eps_x[ny] = e[0], e[ny - 1]
    sig_x[0], sig_x[ny] = s[0], s[ny - 1]
    eps_y = np.empty((ny, nx + 1))
    sig_y = np.empty((ny, nx + 1))
    eps_y[:, 1:nx] = 0.5 * (e[:, :-1] + e[:, 1:])
    sig_y[:, 1:nx] = 0.5 * (s[:, :-1] + s[:, 1:])
    eps_y[:, 0], eps_y[:, nx] = e[:, 0], e[:, nx - 1]
    sig_y[:, 0], sig_y[:, nx] = s[:, 0], s[:, nx - 1]
    return eps_x, sig_x, eps_y, sig_y


@dataclasses.dataclass
class Interface:
    """The coarse side of one reduced-model region (Sec. IV-A).

    Ordered like the fine ports of Eq. (8): South, North, West, East, each in
    increasing i (S, N) or j (W, E).  For interface edge k:

    * comp[k], ei[k], ej[k]: the coarse E edge holding y_k (0 = Ex, 1 = Ey);
    * hi[k], hj[k]: the coarse cell just outside the region whose Hz is the
      entry of H in Eq. (14) for this edge;
    * sign[k] * length[k]: the entry of D_l G^T in Eq. (14).  The sign follows
      the local Yee curl on each side (a reading: Eq. (14) prints one sign for
      all sides, Eq. (13) shows the South-of-coarse-grid case): S -1, N +1,
      W +1, E -1;
    * length[k] (D_l), half[k] (D_l', the half coarse cell depth), and the
      half-cell material eps_b[k], sig_b[k] (D_eps_b, D_sigma_b): the material
      of the coarse cell just outside (Eq. (13), text below it).
    """

    i0: int
    j0: int
    a: int
    b: int
    comp: np.ndarray
    ei: np.ndarray
    ej: np.ndarray
    hi: np.ndarray
    hj: np.ndarray
    sign: np.ndarray
    length: np.ndarray
    half: np.ndarray
    eps_b: np.ndarray
    sig_b: np.ndarray

    @property
    def ny_(self) -> int:
        return len(self.comp)


def make_interface(i0, j0, a, b, dx, dy, eps_r, sigma) -> Interface:
    comp, ei, ej, hi, hj, sign, length, half = ([] for _ in range(8))
    for i in range(i0, i0 + a):  # South side: Ex on row j0, outside cell below
        comp.append(0); ei.append(i); ej.append(j0); hi.append(i); hj.append(j0 - 1)
        sign.append(-1.0); length.append(dx); half.append(dy / 2)
    for i in range(i0, i0 + a):  # North side: Ex on row j0+b, outside cell above
        comp.append(0); ei.append(i); ej.append(j0 + b); hi.append(i); hj.append(j0 + b)
        sign.append(+1.0); length.append(dx); half.append(dy / 2)
    for j in range(j0, j0 + b):  # West side: Ey on column i0, outside cell left
        comp.append(1); ei.append(i0); ej.append(j); hi.append(i0 - 1); hj.append(j)
        sign.append(+1.0); length.append(dy); half.append(dx / 2)
    for j in range(j0, j0 + b):  # East side: Ey on column i0+a, outside cell right
        comp.append(1); ei.append(i0 + a); ej.append(j); hi.append(i0 + a); hj.append(j)
        sign.append(-1.0); length.append(dy); half.append(dx / 2)
    hi_a, hj_a = np.array(hi), np.array(hj)
    return Interface(
        i0, j0, a, b, np.array(comp), np.array(ei), np.array(ej), hi_a, hj_a,
        np.array(sign), np.array(length), np.array(half),
        EPS0 * np.asarray(eps_r, dtype=np.float64)[hj_a, hi_a],
        np.asarray(sigma, dtype=np.float64)[hj_a, hi_a])


class CoarseGrid:
    """Coarse mesh with PEC walls and reduced-model holes (FP64)."""

    def __init__(self, nx, ny, dx, dy, dt, eps_r, sigma, regions=()):
        self.nx, self.ny, self.dx, self.dy, self.dt = nx, ny, dx, dy, dt
        self.eps_r = np.asarray(eps_r, dtype=np.float64).reshape(ny, nx)
        self.sigma = np.asarray(sigma, dtype=np.float64).reshape(ny, nx)
        self.eps_x, self.sig_x, self.eps_y, self.sig_y = edge_materials(self.eps_r, self.sigma)
        self.hz_active = np.ones((ny, nx), dtype=bool)
        self.ex_upd = np.ones((ny + 1, nx), dtype=bool)
        self.ey_upd = np.ones((ny, nx + 1), dtype=bool)
        self.ex_upd[0, :] = False           # PEC walls
        self.ex_upd[ny, :] = False
        self.ey_upd[:, 0] = False
        self.ey_upd[:, nx] = False
        self.interfaces = []
        for (i0, j0, a, b) in regions:
            self.hz_active[j0:j0 + b, i0:i0 + a] = False
            self.ex_upd[j0:j0 + b + 1, i0:i0 + a] = False   # interface + inside
            self.ey_upd[j0:j0 + b, i0:i0 + a + 1] = False
            self.interfaces.append(make_interface(i0, j0, a, b, dx, dy, self.eps_r, self.sigma))
        # Eq. (3) written as alpha E^{n+1} = beta E^n + curl - area J.
        area = dx * dy
        self.ax = area * (self.eps_x / dt + self.sig_x / 2)
        self.bx = area * (self.eps_x / dt - self.sig_x / 2)
        self.ay = area * (self.eps_y / dt + self.sig_y / 2)
        self.by = area * (self.eps_y / dt - self.sig_y / 2)

    def zeros(self):
        return (np.zeros((self.ny + 1, self.nx)), np.zeros((self.ny, self.nx + 1)),
                np.zeros((self.ny, self.nx)))

    def h_update(self, Ex, Ey, Hz):
        """Eq. (5) on the coarse mesh: Hz^{n+1/2} from Hz^{n-1/2} and E^n.

        dx dy mu/dt (H^{n+1/2} - H^{n-1/2})
            = -dx Ex_{j} + dx Ex_{j+1} + dy Ey_{i} - dy Ey_{i+1}.
        mu = mu0 everywhere (the text below Eq. (5) says "permittivity"; read
        as permeability of a non-magnetic medium).
        """
        dx, dy = self.dx, self.dy
        curl = -dx * Ex[:-1, :] + dx * Ex[1:, :] + dy * Ey[:, :-1] - dy * Ey[:, 1:]
        Hn = Hz + (self.dt / (dx * dy * MU0)) * curl
        return np.where(self.hz_active, Hn, 0.0)

    def e_update(self, Ex, Ey, Hz):
        """Eq. (3) on the coarse mesh (and its Ey counterpart), no source.

        dx dy (eps/dt + sigma/2) Ex^{n+1} = dx dy (eps/dt - sigma/2) Ex^n
                                            + dx Hz_{j+1/2} - dx Hz_{j-1/2},
        dx dy (eps/dt + sigma/2) Ey^{n+1} = dx dy (eps/dt - sigma/2) Ey^n
                                            - dy Hz_{i+1/2} + dy Hz_{i-1/2}.
        Edges that are PEC, interface or inside a region keep their value.
        """
        dx, dy = self.dx, self.dy
        Exn = Ex.copy()
        Eyn = Ey.copy()
        cx = np.zeros_like(Ex)
        cx[1:self.ny, :] = dx * (Hz[1:, :] - Hz[:-1, :])
        cy = np.zeros_like(Ey)
        cy[:, 1:self.nx] = -dy * (Hz[:, 1:] - Hz[:, :-1])
        Exn = np.where(self.ex_upd, (self.bx * Ex + cx) / self.ax, Ex)
        Eyn = np.where(self.ey_upd, (self.by * Ey + cy) / self.ay, Ey)
        return Exn, Eyn

    def add_current(self, Ex, Ey, comp, i, j, J):
        """Electric current density J (A/m^2) on one updated edge at t^{n+1/2}:
        the term - dx dy J on the right of Eq. (3), i.e. E -= dx dy J / alpha."""
        area = self.dx * self.dy
        if comp == 0:
            assert self.ex_upd[j, i], "source on a non-updated Ex edge"
            Ex[j, i] -= area * J / self.ax[j, i]
        else:
            assert self.ey_upd[j, i], "source on a non-updated Ey edge"
            Ey[j, i] -= area * J / self.ay[j, i]
