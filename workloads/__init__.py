"""Seeded synthetic inputs for the Yee + embedded-ROM scheme.

This module only draws random numbers and lays out geometry: grids, per-cell
materials, region placements, fine-region materials, source waveforms and
probe positions.  It holds none of the scheme's arithmetic, and it is the only
code that the FP64 oracle and the GPU library both consume.

All generators use numpy ``Generator(PCG64(seed))`` with
seed = 1609071140 + workload index unless a seed is given.  Units: metres,
seconds, S/m, A/m^2.  Layout conventions: cell arrays are [ny][nx] (row j,
column i); a source drives ``len`` consecutive E edges starting at edge
(i, j) along the edge direction (comp 0 = Ex, 1 = Ey); a probe (i, j) reads
Hz of coarse cell (i, j).

The time step is part of a workload's recipe: a stated multiple of the 2D
CFL limit 1/(c0 sqrt(1/dx^2 + 1/dy^2)) of the fine mesh (dx/r, dy/r).
"""
from __future__ import annotations

import math
import numpy as np

SEED0 = 1609071140
_C0 = 299792458.0   # exact speed of light in vacuum (m/s), for time-step recipes


def rng_for(index: int, seed: int | None = None) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED0 + index if seed is None else seed))


def fine_cfl(dx: float, dy: float, r: int) -> float:
    """Recipe time step unit: the vacuum CFL limit of a mesh of dx/r x dy/r."""
    return 1.0 / (_C0 * math.sqrt((r / dx) ** 2 + (r / dy) ** 2))


def diff_gaussian(nsteps: int, dt: float, fc: float, t0_mult: float = 4.0) -> np.ndarray:
    """Differentiated-Gaussian current density J(t) = -sqrt(2e) u exp(-u^2),
    u = (t - t0)/tau, tau = 1/(sqrt(2) pi fc), t0 = t0_mult * tau; peak 1 A/m^2.
    Sampled at t = (n + 1/2) dt, n = 0 .. nsteps-1 (FP64)."""
    tau = 1.0 / (math.sqrt(2.0) * math.pi * fc)
    t = (np.arange(nsteps) + 0.5) * dt
    u = (t - t0_mult * tau) / tau
    return -math.sqrt(2.0 * math.e) * u * np.exp(-u * u)


def rect_fine(a, b, r, lo, hi, eps_in, sig_in):
    """Fine-region materials [r*b][r*a]: vacuum with a rectangle of
    (eps_in, sig_in) over fine cells [lo[0], hi[0]) x [lo[1], hi[1])."""
    e = np.ones((r * b, r * a))
    s = np.zeros((r * b, r * a))
    e[lo[1]:hi[1], lo[0]:hi[0]] = eps_in
    s[lo[1]:hi[1], lo[0]:hi[0]] = sig_in
    return e, s


def cavity_60(nsteps: int = 2000):
    """60 x 60 PEC cavity, dx = dy = 1 mm, vacuum.  One 10 x 10-cell region at
    [25, 35)^2 refined r = 3 (30 x 30 fine) holding a centred 12 x 12-fine-cell
    block eps_r = 4, sigma = 0.01 S/m; ROM order 60.  A differentiated-Gaussian
    Jy current (fc = 30 GHz) on the Ey edge at (15, 30); Hz probes at (45, 30)
    and (30, 45); dt = 0.9 x the fine-mesh CFL limit."""
    nx = ny = 60
    dx = dy = 1e-3
    r = 3
    dt = 0.9 * fine_cfl(dx, dy, r)
    ef, sf = rect_fine(10, 10, r, (9, 9), (21, 21), 4.0, 0.01)
    return dict(
        name="cavity_60", nx=nx, ny=ny, dx=dx, dy=dy, dt=dt,
        eps_r=np.ones((ny, nx)), sigma=np.zeros((ny, nx)),
        roms=[dict(i0=25, j0=25, a=10, b=10, r=r, eps_r=ef, sigma=sf, q=60, f0=30e9)],
        sources=[dict(comp=1, i=15, j=30, len=1, wave=diff_gaussian(nsteps, dt, 30e9))],
        probes=[(45, 30), (30, 45)], nsteps=nsteps)


def random_grid(index, nx, ny, n_regions, a, r, q, nsteps, dt_factor=0.95, fc=30e9,
                n_probes=16, eps_range=(1.0, 4.0), sig_range=(0.0, 0.02), seed=None,
                inclusion=True, margin=2):
    """Inhomogeneous lossy grid with seeded non-overlapping a x a regions.

    eps_r ~ U[eps_range], sigma ~ U[sig_range] per coarse cell.  Each region
    holds a seeded rectangular inclusion (side U[a*r/4, a*r) fine cells,
    eps_r ~ U[2, 10], sigma ~ U[0.01, 0.1]).  Regions keep `margin` coarse
    cells from the walls and from each other.  One Jy point source and
    n_probes Hz probes are placed outside every region."""
    g = rng_for(index, seed)
    dx = dy = 1e-3
    eps = g.uniform(*eps_range, size=(ny, nx))
    sig = g.uniform(*sig_range, size=(ny, nx))
    occ = np.zeros((ny, nx), dtype=bool)
    roms = []
    tries = 0
    while len(roms) < n_regions:
        tries += 1
        if tries > 10000:
            raise RuntimeError("cannot place regions")
        i0 = int(g.integers(margin, nx - a - margin + 1))
        j0 = int(g.integers(margin, ny - a - margin + 1))
        if occ[j0 - margin:j0 + a + margin, i0 - margin:i0 + a + margin].any():
            continue
        occ[j0 - 1:j0 + a + 1, i0 - 1:i0 + a + 1] = True
        nf = a * r
        if inclusion:
            w = int(g.integers(max(1, nf // 4), nf))
            h = int(g.integers(max(1, nf // 4), nf))
            x0 = int(g.integers(0, nf - w + 1))
            y0 = int(g.integers(0, nf - h + 1))
            ef, sf = rect_fine(a, a, r, (x0, y0), (x0 + w, y0 + h),
                               g.uniform(2.0, 10.0), g.uniform(0.01, 0.1))
        else:
            ef, sf = np.ones((nf, nf)), np.zeros((nf, nf))
        roms.append(dict(i0=i0, j0=j0, a=a, b=a, r=r, eps_r=ef, sigma=sf, q=q, f0=fc))
    dt = dt_factor * fine_cfl(dx, dy, r)

    def free_cell():
        while True:
            i = int(g.integers(1, nx - 1))
            j = int(g.integers(1, ny - 1))
            if not occ[max(j - 1, 0):j + 2, max(i - 1, 0):i + 2].any():
                return i, j

    si, sj = free_cell()
    probes = [free_cell() for _ in range(n_probes)]
    return dict(
        name=f"random_{nx}x{ny}", nx=nx, ny=ny, dx=dx, dy=dy, dt=dt, eps_r=eps, sigma=sig,
        roms=roms, sources=[dict(comp=1, i=si, j=sj, len=1, wave=diff_gaussian(nsteps, dt, fc))],
        probes=probes, nsteps=nsteps)


def grid_4096(nsteps: int = 20000):
    """4096^2 cells at dx = 1 mm, eps_r ~ U[1,4], sigma ~ U[0,0.02] per cell;
    8 regions of 16 x 16 coarse cells refined r = 4, each with a seeded lossy
    inclusion; ROM order 200; one Jy point source (fc = 30 GHz) and 16 probes;
    dt = 0.95 x the fine-mesh CFL limit."""
    return random_grid(1, 4096, 4096, 8, 16, 4, 200, nsteps, dt_factor=0.95)


def lattice_lossless(n=256, nsteps=1_000_000, seed=None, lossless=True):
    """Scaled-down form of the many-heterogeneous-ROM workload with CFL
    extension: an n x n vacuum grid (dx = 1 mm), a 2 x 2 lattice of regions
    drawn from three fine-region types refined r = 5 (regions of 6, 12 and 20
    coarse cells, ROM orders 60, 180, 400), each holding a seeded dielectric
    scatterer; dt = 2 x the fine-mesh CFL limit (0.4 x the coarse one).  One
    Jy pulse (fc = 10 GHz) that has died out after ~1000 steps.  lossless:
    sigma = 0 everywhere (energy must stay constant)."""
    g = rng_for(4, seed)
    dx = dy = 1e-3
    r = 5
    types = [(6, 60), (12, 180), (20, 400)]
    roms = []
    pitch = n // 2
    k = 0
    for ty in range(2):
        for tx in range(2):
            a, q = types[k % 3]
            k += 1
            i0 = tx * pitch + int(g.integers(4, pitch - a - 4))
            j0 = ty * pitch + int(g.integers(4, pitch - a - 4))
            nf = a * r
            w = int(g.integers(nf // 4, nf // 2))
            x0 = int(g.integers(0, nf - w))
            y0 = int(g.integers(0, nf - w))
            ef, sf = rect_fine(a, a, r, (x0, y0), (x0 + w, y0 + w), g.uniform(2.0, 6.0),
                               0.0 if lossless else g.uniform(0.0, 0.05))
            roms.append(dict(i0=i0, j0=j0, a=a, b=a, r=r, eps_r=ef, sigma=sf, q=q, f0=10e9))
    dt = 2.0 * fine_cfl(dx, dy, r)
    src = dict(comp=1, i=n // 2, j=n // 2 + 3, len=1, wave=diff_gaussian(min(nsteps, 4000), dt, 10e9))
    return dict(name=f"lattice_{n}", nx=n, ny=n, dx=dx, dy=dy, dt=dt,
                eps_r=np.ones((n, n)), sigma=np.zeros((n, n)) if lossless else 0.01 * g.random((n, n)),
                roms=roms, sources=[src], probes=[(n // 4, n // 4), (3 * n // 4, n // 4)], nsteps=nsteps)


def lattice_8192(nsteps: int = 10000, n: int = 8192, pitch: int = 1024, lossless: bool = False,
                 fill: float = 0.01, n_line: int = 4, n_probes: int = 16, seed=None):
    """Many heterogeneous reduced models with CFL extension: an n x n vacuum
    grid (dx = 1 mm) with seeded lossy rectangular scatterers (sides U[4, 16]
    cells, eps_r ~ U[2, 6], sigma ~ U[0, 0.05]) covering a fraction `fill` of
    the cells, and one embedded region per pitch x pitch lattice cell (seeded
    jitter of up to pitch/4), drawn from three fine-region types refined r = 5
    (regions of 6, 12 and 20 coarse cells, ROM orders 60, 180, 400; each type
    holds one seeded dielectric inclusion).  Scatterers keep two cells from
    every region, so each region's ring of outside half cells is vacuum.
    n_line Jy line sources, each a full column of Ey edges at a seeded x clear
    of the regions (fc = 10 GHz differentiated Gaussian); n_probes Hz probes;
    dt = 2 x the fine-mesh CFL limit (0.4 x the coarse one).  lossless: sigma
    = 0 everywhere, including the inclusions."""
    g = rng_for(6, seed)
    dx = dy = 1e-3
    r = 5
    types = []
    for a, q in [(6, 60), (12, 180), (20, 400)]:
        nf = a * r
        w = int(g.integers(nf // 4, nf // 2))
        x0, y0 = int(g.integers(0, nf - w)), int(g.integers(0, nf - w))
        ef, sf = rect_fine(a, a, r, (x0, y0), (x0 + w, y0 + w), g.uniform(2.0, 6.0),
                           0.0 if lossless else g.uniform(0.0, 0.05))
        types.append(dict(a=a, b=a, r=r, eps_r=ef, sigma=sf, q=q, f0=10e9))
    m = n // pitch
    occ = np.zeros((n, n), dtype=bool)   # regions plus a two-cell margin
    roms = []
    for ty in range(m):
        for tx in range(m):
            t = types[int(g.integers(0, 3))]
            a = t["a"]
            c = pitch // 2 - a // 2
            i0 = tx * pitch + c + int(g.integers(-(pitch // 4), pitch // 4 + 1))
            j0 = ty * pitch + c + int(g.integers(-(pitch // 4), pitch // 4 + 1))
            occ[j0 - 3:j0 + a + 3, i0 - 3:i0 + a + 3] = True
            roms.append(dict(t, i0=i0, j0=j0))
    eps = np.ones((n, n))
    sig = np.zeros((n, n))
    cov = np.zeros((n, n), dtype=bool)
    pre = np.zeros((n + 1, n + 1), dtype=np.int64)   # prefix sums of occ
    pre[1:, 1:] = np.cumsum(np.cumsum(occ, axis=0), axis=1)
    target = int(fill * n * n)
    while cov.sum() < target:
        k = int(min(256, max(4, (target - cov.sum()) // 100)))
        w = g.integers(4, 17, size=k)
        h = g.integers(4, 17, size=k)
        x = g.integers(1, n - 17, size=k)
        y = g.integers(1, n - 17, size=k)
        e_in = g.uniform(2.0, 6.0, size=k)
        s_in = np.zeros(k) if lossless else g.uniform(0.0, 0.05, size=k)
        hit = pre[y + h, x + w] - pre[y, x + w] - pre[y + h, x] + pre[y, x]
        for t in np.nonzero(hit == 0)[0]:
            sl = (slice(y[t], y[t] + h[t]), slice(x[t], x[t] + w[t]))
            eps[sl] = e_in[t]
            sig[sl] = s_in[t]
            cov[sl] = True
    dt = 2.0 * fine_cfl(dx, dy, r)
    blocked = occ.any(axis=0)
    xs = []
    while len(xs) < n_line:
        x = int(g.integers(8, n - 8))
        if not blocked[x - 2:x + 3].any() and all(abs(x - u) > 8 for u in xs):
            xs.append(x)
    wave = diff_gaussian(nsteps, dt, 10e9)
    sources = [dict(comp=1, i=x, j=0, len=n, wave=wave) for x in xs]
    probes = []
    while len(probes) < n_probes:
        i, j = int(g.integers(1, n - 1)), int(g.integers(1, n - 1))
        if not occ[j, i]:
            probes.append((i, j))
    return dict(name=f"lattice_{n}", nx=n, ny=n, dx=dx, dy=dy, dt=dt, eps_r=eps, sigma=sig,
                roms=roms, sources=sources, probes=probes, nsteps=nsteps, types=types)


def batched_256(nsteps: int = 5000, per_size: int = 64, sizes=(128, 256, 512, 1024), seed=None):
    """Batch of independent simulations of uneven sizes sharing four reduced
    models (r = 3; regions of 8, 12, 16 and 24 coarse cells, orders 40, 80,
    160 and 320; vacuum fine interior with a centred lossy block).  Each
    simulation: eps_r ~ U[1,4], sigma ~ U[0,0.02] per cell, the four regions
    at seeded positions, one quadrant each, with a vacuum ring of coarse cells
    around every region (so that all simulations share one coupled map per
    model), one Jy point source at a seeded position with fc ~ U[10, 30] GHz,
    and one Hz probe.  dt = 0.9 x the fine-mesh CFL limit for every one."""
    g = rng_for(3, seed)
    dx = dy = 1e-3
    r = 3
    types = [(8, 40), (12, 80), (16, 160), (24, 320)]
    models = []
    for a, q in types:
        nf = a * r
        lo, hi = nf // 3, nf - nf // 3
        ef, sf = rect_fine(a, a, r, (lo, lo), (hi, hi), 3.0, 0.05)
        models.append(dict(a=a, b=a, r=r, eps_r=ef, sigma=sf, q=q, f0=20e9))
    dt = 0.9 * fine_cfl(dx, dy, r)
    sims = []
    for n in sizes:
        for _ in range(per_size):
            eps = g.uniform(1.0, 4.0, size=(n, n))
            sig = g.uniform(0.0, 0.02, size=(n, n))
            occ = np.zeros((n, n), dtype=bool)
            place = []
            h = n // 2
            for k, (a, q) in enumerate(types):
                qx, qy = (k % 2) * h, (k // 2) * h
                i0 = qx + int(g.integers(3, h - a - 3))
                j0 = qy + int(g.integers(3, h - a - 3))
                eps[j0 - 1:j0 + a + 1, i0 - 1:i0 + a + 1] = 1.0
                sig[j0 - 1:j0 + a + 1, i0 - 1:i0 + a + 1] = 0.0
                occ[j0 - 2:j0 + a + 2, i0 - 2:i0 + a + 2] = True
                place.append((k, i0, j0))
            while True:
                si, sj = int(g.integers(2, n - 2)), int(g.integers(2, n - 2))
                if not occ[sj, si]:
                    break
            while True:
                pi, pj = int(g.integers(1, n - 1)), int(g.integers(1, n - 1))
                if not occ[pj, pi]:
                    break
            fc = float(g.uniform(10e9, 30e9))
            sims.append(dict(nx=n, ny=n, eps_r=eps, sigma=sig, place=place,
                             source=dict(comp=1, i=si, j=sj, len=1, wave=diff_gaussian(nsteps, dt, fc)),
                             probe=(pi, pj)))
    return dict(name="batched_256", dx=dx, dy=dy, dt=dt, models=models, sims=sims, nsteps=nsteps)


def adjoint_16(nsteps: int = 10000, nsim: int = 16, n: int = 1024, seed=None):
    """Gradient workload: nsim simulations of n x n cells (eps_r ~ U[1,4],
    sigma ~ U[0,0.02] per cell), each embedding the same two reduced models
    (r = 3, q = 120, 16 x 16-cell regions; a lossy block and a dielectric
    block) with vacuum rings, one Jy point source (fc = 20 GHz) and 8 Hz
    probes per simulation; dt = 0.9 x the fine-mesh CFL limit.  The
    objective is J = sum over steps and probes of Hz^2."""
    g = rng_for(5, seed)
    dx = dy = 1e-3
    r, a = 3, 16
    nf = a * r
    m0 = rect_fine(a, a, r, (nf // 4, nf // 4), (3 * nf // 4, 3 * nf // 4), 4.0, 0.05)
    m1 = rect_fine(a, a, r, (nf // 3, nf // 6), (2 * nf // 3, 5 * nf // 6), 8.0, 0.0)
    models = [dict(a=a, b=a, r=r, eps_r=m0[0], sigma=m0[1], q=120, f0=20e9),
              dict(a=a, b=a, r=r, eps_r=m1[0], sigma=m1[1], q=120, f0=20e9)]
    dt = 0.9 * fine_cfl(dx, dy, r)
    sims = []
    for _ in range(nsim):
        eps = g.uniform(1.0, 4.0, size=(n, n))
        sig = g.uniform(0.0, 0.02, size=(n, n))
        occ = np.zeros((n, n), dtype=bool)
        place = []
        for k in range(2):
            while True:
                i0 = int(g.integers(4, n - a - 4))
                j0 = int(g.integers(4, n - a - 4))
                if not occ[j0 - 3:j0 + a + 3, i0 - 3:i0 + a + 3].any():
                    break
            eps[j0 - 1:j0 + a + 1, i0 - 1:i0 + a + 1] = 1.0
            sig[j0 - 1:j0 + a + 1, i0 - 1:i0 + a + 1] = 0.0
            occ[j0 - 2:j0 + a + 2, i0 - 2:i0 + a + 2] = True
            place.append((k, i0, j0))

        def free():
            while True:
                i, j = int(g.integers(2, n - 2)), int(g.integers(2, n - 2))
                if not occ[j, i]:
                    return i, j

        si, sj = free()
        sims.append(dict(nx=n, ny=n, eps_r=eps, sigma=sig, place=place,
                         source=dict(comp=1, i=si, j=sj, len=1, wave=diff_gaussian(nsteps, dt, 20e9)),
                         probes=[free() for _ in range(8)]))
    return dict(name="adjoint_16", dx=dx, dy=dy, dt=dt, models=models, sims=sims, nsteps=nsteps)
