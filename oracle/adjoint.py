"""Discrete adjoint of the Yee + embedded-ROM time loop, FP64 oracle.

Objective (probe energy):  J = sum_n sum_p (Hz^{n+1/2}(probe p))^2, or, given
a cotangent c[n][p] of the probe samples o^n_p = Hz^{n+1/2}(probe p), the
vector-Jacobian product of the probe series, i.e. the gradient of the linear
functional L = sum_n sum_p c[n][p] o^n_p (c = 2 o gives J's gradient).
Parameters: per-cell eps_r and sigma of the coarse grid and the source
samples J^n.  The forward step n (``scheme.step``) is

  H'  = H + dt/(mu0 dx dy) (-dx Ex_j + dx Ex_{j+1} + dy Ey_i - dy Ey_{i+1})   (Eq. (5))
  o^n = H'(probes)
  alpha E' = beta E + curl(H') - A J^n         on updated edges              (Eq. (3))
  s'  = P s + Q h(H'),  E'(interface) = s'[:n_y]                              (Eq. (23))

with s = [y; x~], alpha/beta = A (eps/dt +- sigma/2) per edge.  Its exact
transpose, run backwards over stored forward states, gives the gradient
(g = dJ/d(state after the step)):

  1. g_s[:n_y] += g_E(interface); g_E(interface) = 0   (E' there is a copy of s')
  2. t = Q^T g_s;  g_H'(h cells) += t;  g_s <- P^T g_s
  3. g_H' += curl^T(g_E / alpha);  dJ/dJ^n = -A g_E / alpha on source edges;
     dJ/deps_edge += g_E A (E - E') / (alpha dt);
     dJ/dsigma_edge -= g_E A (E + E') / (2 alpha);  g_E <- (beta/alpha) g_E
  4. g_H'(probes) += dL/do^n   (2 o^n for J, c[n] for a given cotangent)
  5. g_E += (H update)^T g_H';  g_H <- g_H' on coarse cells
Edge materials are cell means, so a cell receives half of each adjacent edge's
eps/sigma gradient.  The coarse half cell of interface edge k (the cell just
outside, Eq. (13)) also enters A1 and A2 of Eq. (19): with
c_k = A1^{-1} e_k = Q[:, k] / (Dl G^T)_k, d[P|Q]/d(dplus_k) = -c_k [P|Q]_k and
d[P|Q]/d(dminus_k) = c_k e_{y_k}^T, which gives in step 2
  dJ/deps_b,k   += (Dl Dl')_k / dt * t_k / (Dl G^T)_k * (y_k^n - y_k^{n+1})
  dJ/dsigma_b,k -= (Dl Dl')_k / 2  * t_k / (Dl G^T)_k * (y_k^n + y_k^{n+1}).
(Valid when A1 is nonsingular: the dual rule, or the paper rule at full order.)
"""
from __future__ import annotations

import numpy as np

from . import problem, scheme
from .yee import EPS0, MU0


def forward_store(grid, emb, nsteps, sources, probes):
    """Run forward, keeping every state (E^n, H^{n-1/2}, s^n) n = 0..nsteps."""
    st = scheme.State(*grid.zeros())
    states = []

    def snap():
        s = [np.concatenate([scheme.gather_y(grid, e.itf_index, st), e.x]) for e in emb]
        states.append((st.Ex.copy(), st.Ey.copy(), st.Hz.copy(), s))

    out = np.zeros((nsteps, len(probes)))
    snap()
    for n in range(nsteps):
        scheme.step(grid, st, emb, sources, n, probes, out)
        snap()
    return states, out


def gradients(w, nsteps=None, rule=None, order=None, cotangent=None):
    """J and dJ/d(eps_r, sigma, source samples) for workload w (FP64); with a
    cotangent c ([nsteps][nprobe]), L = sum c o and dL/d(...) instead."""
    kw = {} if rule is None else {"rule": rule}
    grid, emb, built = problem.build(w, order=order, **kw)
    n_steps = w["nsteps"] if nsteps is None else nsteps
    sources, probes = w["sources"], w["probes"]
    states, out = forward_store(grid, emb, n_steps, sources, probes)
    if cotangent is None:
        J = float(np.sum(out**2))
        seed = 2.0 * out
    else:
        seed = np.asarray(cotangent, dtype=np.float64).reshape(n_steps, len(probes))
        J = float(np.sum(seed * out))
    nx, ny, dx, dy, dt = grid.nx, grid.ny, grid.dx, grid.dy, grid.dt
    area = dx * dy
    ch = dt / (dx * dy * MU0)
    gEx = np.zeros((ny + 1, nx))
    gEy = np.zeros((ny, nx + 1))
    gH = np.zeros((ny, nx))
    gs = [np.zeros(e.P.shape[0]) for e in emb]
    geps_x = np.zeros((ny + 1, nx))
    gsig_x = np.zeros((ny + 1, nx))
    geps_y = np.zeros((ny, nx + 1))
    gsig_y = np.zeros((ny, nx + 1))
    geps_b = [np.zeros(grid.interfaces[e.itf_index].ny_) for e in emb]
    gsig_b = [np.zeros(grid.interfaces[e.itf_index].ny_) for e in emb]
    gsrc = [np.zeros(n_steps) for _ in sources]
    pi = np.array([p[0] for p in probes], dtype=int)
    pj = np.array([p[1] for p in probes], dtype=int)
    for n in range(n_steps - 1, -1, -1):
        Ex0, Ey0, _, s0 = states[n]
        Ex1, Ey1, _, s1 = states[n + 1]
        gHp = gH.copy()
        # 1. interface E is a copy of the model's y
        for k, e in enumerate(emb):
            itf = grid.interfaces[e.itf_index]
            mx = itf.comp == 0
            nyk = itf.ny_
            gs[k][:nyk][mx] += gEx[itf.ej[mx], itf.ei[mx]]
            gs[k][:nyk][~mx] += gEy[itf.ej[~mx], itf.ei[~mx]]
            gEx[itf.ej[mx], itf.ei[mx]] = 0.0
            gEy[itf.ej[~mx], itf.ei[~mx]] = 0.0
        # 2. transposed model map and the half-cell material terms
        for k, e in enumerate(emb):
            itf = grid.interfaces[e.itf_index]
            t = e.Q.T @ gs[k]
            np.add.at(gHp, (itf.hj, itf.hi), t)
            lh = itf.length * itf.half
            dlg = itf.sign * itf.length
            yn, yn1 = s0[k][:itf.ny_], s1[k][:itf.ny_]
            geps_b[k] += lh / dt * t / dlg * (yn - yn1)
            gsig_b[k] -= lh / 2 * t / dlg * (yn + yn1)
            gs[k] = e.P.T @ gs[k]
        # 3. transposed E update on updated edges
        mux = np.where(grid.ex_upd, gEx / grid.ax, 0.0)
        muy = np.where(grid.ey_upd, gEy / grid.ay, 0.0)
        geps_x += np.where(grid.ex_upd, mux * area * (Ex0 - Ex1) / dt, 0.0)
        gsig_x -= np.where(grid.ex_upd, mux * area * (Ex0 + Ex1) / 2, 0.0)
        geps_y += np.where(grid.ey_upd, muy * area * (Ey0 - Ey1) / dt, 0.0)
        gsig_y -= np.where(grid.ey_upd, muy * area * (Ey0 + Ey1) / 2, 0.0)
        for q, src in enumerate(sources):
            for (c, i, j) in scheme.source_edges(src):
                gsrc[q][n] += -area * (mux[j, i] if c == 0 else muy[j, i])
        # Ex'(i,j) has + dx Hz(i,j) - dx Hz(i,j-1); Ey'(i,j) has - dy Hz(i,j) + dy Hz(i-1,j)
        gHp += dx * mux[:-1, :] - dx * mux[1:, :]
        gHp += -dy * muy[:, :-1] + dy * muy[:, 1:]
        gEx = np.where(grid.ex_upd, grid.bx / grid.ax * gEx, 0.0)
        gEy = np.where(grid.ey_upd, grid.by / grid.ay * gEy, 0.0)
        # 4. probes: o^n = H'(probes), dL/do^n = seed[n]
        np.add.at(gHp, (pj, pi), seed[n])
        # 5. transposed H update (coarse cells only)
        gHp = np.where(grid.hz_active, gHp, 0.0)
        gEx[:-1, :] += -ch * dx * gHp
        gEx[1:, :] += ch * dx * gHp
        gEy[:, :-1] += ch * dy * gHp
        gEy[:, 1:] += -ch * dy * gHp
        # PEC and covered edges are constants, not state
        cov_x = ~grid.ex_upd
        cov_y = ~grid.ey_upd
        for e in emb:
            itf = grid.interfaces[e.itf_index]
            cov_x[itf.ej[itf.comp == 0], itf.ei[itf.comp == 0]] = False
            cov_y[itf.ej[itf.comp == 1], itf.ei[itf.comp == 1]] = False
        gEx[cov_x] = 0.0
        gEy[cov_y] = 0.0
        gH = gHp
    # edge gradients to cells: each edge's material is the mean of its cells
    deps = np.zeros((ny, nx))
    dsig = np.zeros((ny, nx))
    deps[:-1, :] += 0.5 * EPS0 * geps_x[1:ny, :]
    deps[1:, :] += 0.5 * EPS0 * geps_x[1:ny, :]
    dsig[:-1, :] += 0.5 * gsig_x[1:ny, :]
    dsig[1:, :] += 0.5 * gsig_x[1:ny, :]
    deps[:, :-1] += 0.5 * EPS0 * geps_y[:, 1:nx]
    deps[:, 1:] += 0.5 * EPS0 * geps_y[:, 1:nx]
    dsig[:, :-1] += 0.5 * gsig_y[:, 1:nx]
    dsig[:, 1:] += 0.5 * gsig_y[:, 1:nx]
    for k, e in enumerate(emb):
        itf = grid.interfaces[e.itf_index]
        np.add.at(deps, (itf.hj, itf.hi), EPS0 * geps_b[k])
        np.add.at(dsig, (itf.hj, itf.hi), gsig_b[k])
    for k, e in enumerate(emb):     # cells covered by a model are not coarse unknowns
        itf = grid.interfaces[e.itf_index]
        deps[itf.j0:itf.j0 + itf.b, itf.i0:itf.i0 + itf.a] = 0.0
        dsig[itf.j0:itf.j0 + itf.b, itf.i0:itf.i0 + itf.a] = 0.0
    return J, deps, dsig, gsrc


def objective(w, nsteps=None, rule=None, order=None, cotangent=None):
    """J (sum of probe Hz^2), or L = sum c o for a cotangent c."""
    kw = {} if rule is None else {"rule": rule}
    out, *_ = problem.run(w, nsteps, order=order, **kw)
    if cotangent is None:
        return float(np.sum(out**2))
    return float(np.sum(np.asarray(cotangent, dtype=np.float64).reshape(out.shape) * out))
