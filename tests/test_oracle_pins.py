"""Pins for the FP64 oracle: each test checks the oracle against something the
paper or the mathematics fixes, never against the oracle itself.

* printed values: fine-model state sizes (Sec. VI), S_hat (Eq. (25));
* closed forms: PEC-cavity eigenmodes of the Yee scheme, the fine-region CFL
  limit of Eq. (1);
* invariants: discrete energy conservation / dissipation (Sec. V, Appendix A),
  the energy balance of a current source, Theorem 1 (passivity preserved by a
  full-rank block-diagonal congruence), brute-force one-step spectra (Theorem
  2), Krylov moment matching (Sec. III);
* special cases: a full-order model through Eq. (23) equals direct
  subgridding; r = 1 with V = I equals the plain Yee scheme.
Mutation tests at the end plant plausible mistakes in the oracle and check that
a pin catches each.
"""
import json
import os

import numpy as np
import pytest

from oracle import couple, fine, passivity, problem, scheme, sprim, subgrid, yee
from oracle.yee import EPS0, MU0, C0

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def load_golden():
    with open(GOLDEN) as f:
        return json.load(f)


# --------------------------------------------------------------------------- printed values
def test_state_sizes_match_paper():
    for rec in load_golden()["fine_state_sizes"]:
        assert fine.state_size(rec["nxf"], rec["nyf"]) == rec["size"], rec["cite"]
        fs = fine.assemble(rec["nxf"], rec["nyf"], 1e-3, 1e-3,
                           np.ones((rec["nyf"], rec["nxf"])), np.zeros((rec["nyf"], rec["nxf"])))
        assert fs.n == rec["size"]


def test_S_hat_is_the_printed_matrix():
    g = load_golden()["S_hat_signs"]
    nxf, nyf, dxf, dyf = 7, 5, 0.3e-3, 0.45e-3
    rng = np.random.default_rng(3)
    fs = fine.assemble(nxf, nyf, dxf, dyf, 1 + 3 * rng.random((nyf, nxf)), rng.random((nyf, nxf)))
    S = (fs.L_E.T @ fs.B_E).toarray()
    expect = np.concatenate([np.full(nxf, g["S"] * dxf), np.full(nxf, g["N"] * dxf),
                             np.full(nyf, g["W"] * dyf), np.full(nyf, g["E"] * dyf)])
    np.testing.assert_array_equal(S, np.diag(expect))
    # Eq. (24c): B = L S_hat, exactly.
    np.testing.assert_array_equal(fs.B_E.toarray(), fs.L_E.toarray() * expect[None, :])


# --------------------------------------------------------------------------- closed forms
@pytest.mark.parametrize("nx,ny,dx,dy,m,n,eps_r,sig", [
    (16, 12, 1e-3, 1e-3, 1, 0, 1.0, 0.0),
    (16, 12, 1e-3, 1e-3, 3, 2, 1.0, 0.0),
    (10, 14, 0.7e-3, 1.3e-3, 2, 5, 2.5, 0.0),
    (10, 14, 0.7e-3, 1.3e-3, 4, 1, 3.0, 0.05),
    (9, 9, 1e-3, 1e-3, 8, 8, 1.0, 0.0),          # highest mode: checkerboard
])
def test_pec_cavity_mode_recurrence(nx, ny, dx, dy, m, n, eps_r, sig):
    """A PEC-cavity mode Hz ~ cos(m pi (i+1/2)/nx) cos(n pi (j+1/2)/ny) is an
    exact eigenvector of the Yee curl-curl with eigenvalue
    lam = (2 sin(m pi/2nx)/dx)^2 + (2 sin(n pi/2ny)/dy)^2, so the leapfrog
    obeys H^{k+3/2} = (1 + ca - dt cb lam / mu0) H^{k+1/2} - ca H^{k-1/2};
    lossless, 1 + ca - dt cb lam/mu0 = 2 cos(w dt) with
    w = (2/dt) asin(c dt sqrt(sin^2(m pi/2nx)/dx^2 + sin^2(n pi/2ny)/dy^2))."""
    dt = 0.8 * yee.cfl_limit(dx, dy, C0 / np.sqrt(eps_r))
    grid = yee.CoarseGrid(nx, ny, dx, dy, dt, np.full((ny, nx), eps_r), np.full((ny, nx), sig))
    st = scheme.State(*grid.zeros())
    ii, jj = np.meshgrid(np.arange(nx), np.arange(ny))
    st.Hz = np.cos(m * np.pi * (ii + 0.5) / nx) * np.cos(n * np.pi * (jj + 0.5) / ny)
    hist = [st.Hz.copy()]
    for _ in range(40):
        scheme.step(grid, st, [])
        hist.append(st.Hz.copy())
    eps = EPS0 * eps_r
    ca = (eps / dt - sig / 2) / (eps / dt + sig / 2)
    cb = 1.0 / (eps / dt + sig / 2)
    lam = (2 * np.sin(m * np.pi / (2 * nx)) / dx) ** 2 + (2 * np.sin(n * np.pi / (2 * ny)) / dy) ** 2
    coef = 1 + ca - dt * cb * lam / MU0
    if sig == 0.0:
        c = C0 / np.sqrt(eps_r)
        w = (2 / dt) * np.arcsin(c * dt * np.sqrt(np.sin(m * np.pi / (2 * nx)) ** 2 / dx**2
                                                  + np.sin(n * np.pi / (2 * ny)) ** 2 / dy**2))
        assert abs(coef - 2 * np.cos(w * dt)) < 1e-12
    scale = max(np.abs(h).max() for h in hist)
    for k in range(1, len(hist) - 1):
        err = hist[k + 1] - (coef * hist[k] - ca * hist[k - 1])
        assert np.abs(err).max() < 1e-12 * scale


@pytest.mark.parametrize("n,dxf,dyf", [(4, 1e-3, 1e-3), (12, 1e-3, 1e-3), (9, 0.5e-3, 1.2e-3)])
def test_fine_region_cfl_is_eq1(n, dxf, dyf):
    """Eq. (24a) <=> s_max(D_eps^-1/2 K D_mu^-1/2) < 2/dt (Eq. (27) at full
    order).  For a vacuum region with hanging-variable half cells the largest
    singular value equals 2/dt of Eq. (1) exactly, so R > 0 just below the
    Eq. (1) limit and not just above it."""
    fs = fine.assemble(n, n + 1, dxf, dyf, np.ones((n + 1, n)), np.zeros((n + 1, n)))
    M = (fs.K.toarray() / np.sqrt(fs.d_eps)[:, None]) / np.sqrt(fs.d_mu)[None, :]
    s = np.linalg.svd(M, compute_uv=False)[0]
    dt1 = yee.cfl_limit(dxf, dyf)
    assert abs(s * dt1 / 2 - 1.0) < 1e-10
    assert np.linalg.eigvalsh(fs.R(0.999 * dt1).toarray())[0] > 0
    assert np.linalg.eigvalsh(fs.R(1.001 * dt1).toarray())[0] < 0


# --------------------------------------------------------------------------- helpers
def small_problem(nx=14, ny=13, r=2, a=4, b=3, i0=5, j0=4, lossy=False, seed=0, dt_fac=0.9):
    rng = np.random.default_rng(seed)
    dx, dy = 1e-3, 1.2e-3
    eps = 1 + 2 * rng.random((ny, nx))
    sig = 0.05 * rng.random((ny, nx)) if lossy else np.zeros((ny, nx))
    ef = 1 + 3 * rng.random((r * b, r * a))
    sf = 0.2 * rng.random((r * b, r * a)) if lossy else np.zeros((r * b, r * a))
    dt = dt_fac * yee.cfl_limit(dx / r, dy / r)
    return dict(nx=nx, ny=ny, dx=dx, dy=dy, dt=dt, eps_r=eps, sigma=sig,
                roms=[dict(i0=i0, j0=j0, a=a, b=b, r=r, eps_r=ef, sigma=sf, q=0, f0=30e9)],
                sources=[], probes=[(1, 1), (nx - 2, ny - 2), (i0 - 1, j0)], nsteps=0)


def random_state(grid, rng):
    st = scheme.State(*grid.zeros())
    st.Hz = np.where(grid.hz_active, rng.standard_normal(st.Hz.shape), 0.0)
    st.Ex = np.where(grid.ex_upd, rng.standard_normal(st.Ex.shape) * 300, 0.0)
    st.Ey = np.where(grid.ey_upd, rng.standard_normal(st.Ey.shape) * 300, 0.0)
    return st


def copy_state(st):
    return scheme.State(st.Ex.copy(), st.Ey.copy(), st.Hz.copy())


# --------------------------------------------------------------------------- special cases
@pytest.mark.parametrize("rule", [couple.PAPER, couple.DUAL])
@pytest.mark.parametrize("lossy", [False, True])
def test_full_order_model_equals_direct_subgridding(rule, lossy):
    """V = I through Eq. (23) (generalised inverse of A1) must equal the
    independent edge-by-edge subgridding stepper."""
    w = small_problem(lossy=lossy)
    grid, emb, built = problem.build(w, rule=rule, order=0)
    rng = np.random.default_rng(7)
    st1 = random_state(grid, rng)
    st2 = copy_state(st1)
    reg = subgrid.FineRegion(grid, 0, built[0].fs, built[0].T, w["roms"][0]["r"], rule)
    x0 = rng.standard_normal(built[0].rom.q) * 1e-2
    emb[0].x = x0.copy()
    reg.E, reg.H = x0[:reg.fs.nE].copy(), x0[reg.fs.nE:].copy()
    assert built[0].cpl.residual < 1e-11
    o1, st1, _ = scheme.run(grid, emb, 150, probes=w["probes"], st=st1)
    o2, st2 = subgrid.run(grid, [reg], 150, probes=w["probes"], st=st2)
    ref = np.abs(o2).max()
    assert np.abs(o1 - o2).max() < 1e-11 * ref
    x2 = np.concatenate([reg.E, reg.H])
    # internal states agree to the conditioning of the equilibrated A1 solve
    assert np.abs(emb[0].x - x2).max() < 1e-9 * np.abs(x2).max()
    assert np.abs(st1.Ex - st2.Ex).max() < 1e-11 * np.abs(st2.Ex).max()


@pytest.mark.parametrize("rule", [couple.PAPER, couple.DUAL])
def test_r1_full_order_is_plain_yee(rule):
    """r = 1, V = I: coarse and fine half cells form a full cell and the
    hanging variables cancel, so the embedded scheme is the plain Yee scheme
    on the same grid (with the region's cells given the fine materials)."""
    w = small_problem(r=1, lossy=True)
    rd = w["roms"][0]
    grid, emb, built = problem.build(w, rule=rule, order=0)
    eps = w["eps_r"].copy()
    sig = w["sigma"].copy()
    eps[rd["j0"]:rd["j0"] + rd["b"], rd["i0"]:rd["i0"] + rd["a"]] = rd["eps_r"]
    sig[rd["j0"]:rd["j0"] + rd["b"], rd["i0"]:rd["i0"] + rd["a"]] = rd["sigma"]
    plain = yee.CoarseGrid(w["nx"], w["ny"], w["dx"], w["dy"], w["dt"], eps, sig)
    rng = np.random.default_rng(11)
    st1 = random_state(grid, rng)
    st2 = copy_state(st1)
    src = [dict(comp=1, i=2, j=3, len=2, wave=np.sin(np.arange(120) * 0.3))]
    o1, st1, _ = scheme.run(grid, emb, 120, src, w["probes"], st=st1)
    o2, st2, _ = scheme.run(plain, [], 120, src, w["probes"], st=st2)
    assert np.abs(o1 - o2).max() < 1e-12 * np.abs(o2).max()
    # the interface E of the embedded run equals the plain run's edges
    y = scheme.gather_y(grid, 0, st1)
    y2 = scheme.gather_y(grid, 0, st2)
    assert np.abs(y - y2).max() < 1e-10 * np.abs(y2).max()


# --------------------------------------------------------------------------- invariants
@pytest.mark.parametrize("rule,order,dt_fac", [
    (couple.PAPER, 0, 0.9), (couple.DUAL, 0, 0.9), (couple.DUAL, 16, 0.9),
    (couple.DUAL, 40, 1.9),           # reduced, above the fine CFL limit
    (couple.DUAL, 0, 1.9),            # full order, extended by the perturbation
    (couple.PAPER, 0, 1.9),           # (coarse limit is 2x fine at r = 2)
])
def test_energy_conserved_lossless(rule, order, dt_fac):
    """Lossless and source-free, the storage function (dt/2) x^T R x of the
    whole coupled system (coarse with hanging variables + every reduced model)
    is constant: F + F^T = 0 and the interpolation is lossless (Sec. V,
    Appendix A)."""
    w = small_problem(lossy=False, dt_fac=dt_fac)
    grid, emb, built = problem.build(w, rule=rule, order=order)
    if dt_fac > 1 and order == 0:
        assert built[0].s_before[0] > 2 / w["dt"]          # perturbation was needed
        assert built[0].s_after[0] <= 0.99 * 2 / w["dt"] * (1 + 1e-12)
    rng = np.random.default_rng(5)
    st = random_state(grid, rng)
    emb[0].x = rng.standard_normal(built[0].rom.q) * 1e-2
    # a random start violates the interpolation constraint; one step restores it
    scheme.step(grid, st, emb)
    W0 = scheme.energy(grid, st, emb)
    _, st, Ws = scheme.run(grid, emb, 400, st=st, energy_every=20)
    assert np.abs(Ws - W0).max() < 1e-11 * W0


@pytest.mark.parametrize("rule,order", [(couple.PAPER, 0), (couple.DUAL, 20)])
def test_energy_nonincreasing_lossy(rule, order):
    w = small_problem(lossy=True)
    grid, emb, built = problem.build(w, rule=rule, order=order)
    rng = np.random.default_rng(6)
    st = random_state(grid, rng)
    scheme.step(grid, st, emb)
    W0 = scheme.energy(grid, st, emb)
    _, st, Ws = scheme.run(grid, emb, 300, st=st, energy_every=1)
    Ws = np.concatenate([[W0], Ws])
    assert np.all(np.diff(Ws) <= 1e-13 * W0)
    assert Ws[-1] < 0.999 * W0


def test_source_energy_balance():
    """With a current J on edge e (lossless), the storage function changes by
    exactly the work of the source: W^{n+1} - W^n = -(dt/2) A J (E_e^{n+1} + E_e^n)
    (the B u term of Eq. (6) with B = -area on that edge)."""
    w = small_problem(lossy=False)
    w["roms"][0]["q"] = 12
    grid, emb, built = problem.build(w, rule=couple.DUAL)
    rng = np.random.default_rng(8)
    st = random_state(grid, rng)
    wave = rng.standard_normal(50) * 1e3
    src = [dict(comp=0, i=2, j=6, len=1, wave=wave)]
    area = w["dx"] * w["dy"]
    for n in range(50):
        W0 = scheme.energy(grid, st, emb)
        e0 = st.Ex[6, 2]
        scheme.step(grid, st, emb, src, n)
        W1 = scheme.energy(grid, st, emb)
        expect = -(w["dt"] / 2) * area * wave[n] * (st.Ex[6, 2] + e0)
        assert abs((W1 - W0) - expect) < 1e-11 * W0


def test_theorem1_random_block_diagonal_congruence():
    """Theorem 1: any full-rank V = blkdiag(V1, V2) keeps Eqs. (26a)-(26c)."""
    rng = np.random.default_rng(9)
    nxf, nyf = 6, 5
    fs = fine.assemble(nxf, nyf, 1e-3, 1e-3, 1 + 3 * rng.random((nyf, nxf)), 0.1 * rng.random((nyf, nxf)))
    dt = 0.95 * yee.cfl_limit(1e-3, 1e-3)
    for qE, qH in [(5, 4), (20, 17), (fs.nE, fs.nH)]:
        V1 = rng.standard_normal((fs.nE, qE))
        V2 = rng.standard_normal((fs.nH, qH))
        rom = sprim.project(fs, V1, V2)
        rep = passivity.check(rom.R(dt), rom.F(), rom.B(), rom.L(), rom.S_hat)
        assert rep.min_eig_R > 0
        assert rep.min_eig_FFt > -1e-13
        assert rep.cond3_residual < 1e-13
        # the dense congruence equals the block form of Eq. (12)
        V = np.block([[V1, np.zeros((fs.nE, qH))], [np.zeros((fs.nH, qE)), V2]])
        np.testing.assert_allclose(V.T @ fs.R(dt).toarray() @ V, rom.R(dt), rtol=1e-12,
                                   atol=1e-12 * np.abs(rom.R(dt)).max())


def _pack(grid, st, emb):
    parts = [st.Hz[grid.hz_active]]
    exm = grid.ex_upd.copy()
    eym = grid.ey_upd.copy()
    for itf in grid.interfaces:
        exm[itf.ej[itf.comp == 0], itf.ei[itf.comp == 0]] = True
        eym[itf.ej[itf.comp == 1], itf.ei[itf.comp == 1]] = True
    parts += [st.Ex[exm], st.Ey[eym]] + [e.x for e in emb]
    return np.concatenate(parts), exm, eym


def one_step_matrix(grid, emb):
    st = scheme.State(*grid.zeros())
    v0, exm, eym = _pack(grid, st, emb)
    N = v0.size
    Phi = np.zeros((N, N))
    nh, nex, ney = grid.hz_active.sum(), exm.sum(), eym.sum()
    for c in range(N):
        v = np.zeros(N)
        v[c] = 1.0
        st = scheme.State(*grid.zeros())
        st.Hz[grid.hz_active] = v[:nh]
        st.Ex[exm] = v[nh:nh + nex]
        st.Ey[eym] = v[nh + nex:nh + nex + ney]
        off = nh + nex + ney
        for e in emb:
            e.x = v[off:off + e.x.size].copy()
            off += e.x.size
        scheme.step(grid, st, emb)
        Phi[:, c] = _pack(grid, st, emb)[0]
    return Phi


@pytest.mark.parametrize("rule,order,lossy", [(couple.PAPER, 0, False), (couple.DUAL, 0, True),
                                              (couple.DUAL, 12, False)])
def test_one_step_spectrum_inside_unit_circle(rule, order, lossy):
    """Theorem 2 on a tiny grid: the brute-force one-step map has no
    eigenvalue outside the unit circle."""
    w = small_problem(nx=8, ny=8, a=2, b=2, i0=3, j0=3, lossy=lossy)
    grid, emb, built = problem.build(w, rule=rule, order=order)
    lam = np.abs(np.linalg.eigvals(one_step_matrix(grid, emb)))
    assert lam.max() <= 1 + 1e-6


def test_cfl_extension_restores_stability():
    """Negative control (Sec. V-E): above the fine CFL limit the unperturbed
    full-order model is unstable; the clamp of Eq. (27) makes it stable."""
    w = small_problem(nx=8, ny=8, a=2, b=2, i0=3, j0=3, dt_fac=1.9)
    grid, emb, built = problem.build(w, rule=couple.PAPER, order=0, gamma=np.inf)
    lam_bad = np.abs(np.linalg.eigvals(one_step_matrix(grid, emb))).max()
    assert lam_bad > 1.01
    grid, emb, built = problem.build(w, rule=couple.PAPER, order=0, gamma=0.99)
    lam_ok = np.abs(np.linalg.eigvals(one_step_matrix(grid, emb))).max()
    assert lam_ok <= 1 + 1e-6


def test_extension_clamps_only_offending_singular_values():
    rng = np.random.default_rng(2)
    fs = fine.assemble(6, 6, 1e-3, 1e-3, 1 + rng.random((6, 6)), np.zeros((6, 6)))
    rom = sprim.full_order(fs)
    dt = 1.6 * yee.cfl_limit(1e-3, 1e-3)
    s0 = passivity.singular_values_27(rom)
    rom2, s_b, s_a = passivity.extend_cfl(rom, dt, 0.99)
    s1 = passivity.singular_values_27(rom2)
    lim = 0.99 * 2 / dt
    np.testing.assert_allclose(s1, np.minimum(s0, lim), rtol=1e-10, atol=1e-10 * s0[0])
    assert np.linalg.eigvalsh(rom2.R(dt))[0] > 0
    assert np.linalg.eigvalsh(rom.R(dt))[0] < 0


def test_sprim_matches_moments():
    """Sec. III: V contains K_2((psi0 R + F)^-1 R, (psi0 R + F)^-1 B T), so the
    reduced transfer function and its first derivative at psi0 equal the fine
    model's."""
    rng = np.random.default_rng(4)
    a, b, r = 3, 2, 3
    fs = fine.assemble(r * a, r * b, 1e-3 / r, 1e-3 / r, 1 + 3 * rng.random((r * b, r * a)),
                       0.1 * rng.random((r * b, r * a)))
    T = fine.interpolation_T(a, b, r)
    dt = 0.9 * yee.cfl_limit(1e-3 / r, 1e-3 / r)
    psi0 = np.tan(np.pi * 30e9 * dt)
    rom = sprim.sprim(fs, 4 * T.shape[1], dt, psi0, T)     # two full blocks
    R, F, B, L = fs.R(dt).toarray(), fs.F().toarray(), fs.B().toarray(), fs.L().toarray()
    Rt, Ft, Bt, Lt = rom.R(dt), rom.F(), rom.B(), rom.L()
    X = np.linalg.solve(psi0 * R + F, B @ T)
    Xt = np.linalg.solve(psi0 * Rt + Ft, Bt @ T)
    m0, m0t = L.T @ X, Lt.T @ Xt
    m1 = L.T @ np.linalg.solve(psi0 * R + F, R @ X)
    m1t = Lt.T @ np.linalg.solve(psi0 * Rt + Ft, Rt @ Xt)
    assert np.linalg.norm(m0 - m0t) < 1e-9 * np.linalg.norm(m0)
    assert np.linalg.norm(m1 - m1t) < 1e-8 * np.linalg.norm(m1)


def test_paper_rule_degenerates_below_port_count():
    """Reading of Eq. (19): with the paper's interpolation and a reduced
    order q_E + n_y < n_u, range(T) is not inside the model's output space,
    so the constraint y_hat = T y forces y = 0 and decouples the model (the
    region acts as a PEC box).  The dual rule keeps a live interface."""
    w = small_problem(nx=20, ny=20, r=3, a=6, b=6, i0=7, j0=7)
    w["roms"][0]["q"] = 40
    ny_ = 24
    grid, emb, dual = problem.build(w, rule=couple.DUAL)
    qscale = np.abs(dual[0].cpl.Q).max()
    assert np.abs(dual[0].cpl.Q[:ny_]).max() > 1e-3 * qscale
    grid, emb, built = problem.build(w, rule=couple.PAPER)
    assert couple.interface_deficiency(built[0].rom, built[0].T) > 0.5
    assert np.abs(built[0].cpl.P[:ny_]).max() < 1e-12
    assert np.abs(built[0].cpl.Q).max() < 1e-12 * qscale
    assert built[0].cpl.residual < 1e-11 and built[0].cpl.threshold_change < 1e-9
    assert couple.interface_deficiency(sprim.full_order(built[0].fs), built[0].T) < 1e-12


# --------------------------------------------------------------------------- planted mistakes
def test_pins_catch_wrong_interface_sign(monkeypatch):
    """Flip the G sign of the East side: energy conservation must fail."""
    orig = yee.make_interface

    def bad(*args, **kw):
        itf = orig(*args, **kw)
        itf.sign = itf.sign.copy()
        itf.sign[-itf.b:] *= -1
        return itf

    monkeypatch.setattr(yee, "make_interface", bad)
    w = small_problem(lossy=False)
    grid, emb, built = problem.build(w, rule=couple.DUAL, order=0)
    rng = np.random.default_rng(5)
    st = random_state(grid, rng)
    scheme.step(grid, st, emb)
    W0 = scheme.energy(grid, st, emb)
    _, st, Ws = scheme.run(grid, emb, 200, st=st, energy_every=20)
    assert np.abs(Ws - W0).max() > 1e-6 * W0


def test_pins_catch_dropped_loss_term(monkeypatch):
    """Drop sigma/2 from the left side of Eq. (3): the lossy mode recurrence fails."""
    orig_init = yee.CoarseGrid.__init__

    def bad_init(self, *a, **k):
        orig_init(self, *a, **k)
        self.ax = self.dx * self.dy * self.eps_x / self.dt
        self.ay = self.dx * self.dy * self.eps_y / self.dt

    monkeypatch.setattr(yee.CoarseGrid, "__init__", bad_init)
    with pytest.raises(AssertionError):
        test_pec_cavity_mode_recurrence(10, 14, 0.7e-3, 1.3e-3, 4, 1, 3.0, 0.05)


def test_pins_catch_wrong_port_order(monkeypatch):
    """Reverse the port order along the North side in T (a wrong index): the
    r = 1 special case no longer reduces to the plain Yee scheme."""
    orig = fine.interpolation_T

    def bad(a, b, r):
        T = orig(a, b, r)
        n = r * a
        T[n:2 * n] = T[n:2 * n][::-1]
        return T

    monkeypatch.setattr(fine, "interpolation_T", bad)
    with pytest.raises(AssertionError):
        test_r1_full_order_is_plain_yee(couple.PAPER)


# --------------------------------------------------------------------------- field reconstruction
@pytest.mark.parametrize("rule", [couple.PAPER, couple.DUAL])
def test_r1_reconstructed_fields_are_plain_yee_fields(rule):
    """r = 1, V = I: the fields rebuilt from the model state are the plain
    Yee scheme's Hz in the covered cells and its E on the region's inner
    edges (pins the state layout of the reconstruction)."""
    w = small_problem(r=1, lossy=True)
    rd = w["roms"][0]
    i0, j0, a, b = rd["i0"], rd["j0"], rd["a"], rd["b"]
    grid, emb, built = problem.build(w, rule=rule, order=0)
    eps = w["eps_r"].copy()
    sig = w["sigma"].copy()
    eps[j0:j0 + b, i0:i0 + a] = rd["eps_r"]
    sig[j0:j0 + b, i0:i0 + a] = rd["sigma"]
    plain = yee.CoarseGrid(w["nx"], w["ny"], w["dx"], w["dy"], w["dt"], eps, sig)
    src = [dict(comp=1, i=2, j=3, len=2, wave=np.sin(np.arange(90) * 0.3))]
    _, st1, _ = scheme.run(grid, emb, 90, src, [])
    _, st2, _ = scheme.run(plain, [], 90, src, [])
    Exf, Eyf, Hzf = scheme.fine_fields(emb[0], a, b)
    scale = np.abs(st2.Hz).max()
    assert np.abs(Hzf - st2.Hz[j0:j0 + b, i0:i0 + a]).max() < 1e-10 * scale
    escale = np.abs(st2.Ex).max()
    assert np.abs(Exf[1:-1, :] - st2.Ex[j0 + 1:j0 + b, i0:i0 + a]).max() < 1e-10 * escale
    assert np.abs(Eyf[:, 1:-1] - st2.Ey[j0:j0 + b, i0 + 1:i0 + a]).max() < 1e-10 * escale
    # the region's boundary edges are the interface values y
    assert np.abs(Exf[0, :] - st2.Ex[j0, i0:i0 + a]).max() < 1e-10 * escale


def test_reconstruction_error_shrinks_with_order():
    """Information, not a bound from the paper: the rebuilt fine Hz of
    reduced models approaches the direct subgridding field as q grows."""
    w = small_problem(lossy=False)
    rd = w["roms"][0]
    a, b, r = rd["a"], rd["b"], rd["r"]
    src = [dict(comp=1, i=2, j=3, len=1, wave=np.sin(np.arange(200) * 0.05) * np.exp(-((np.arange(200) - 60) / 25.0) ** 2))]
    grid, emb, built = problem.build(w, rule=couple.DUAL, order=0)
    reg = subgrid.FineRegion(grid, 0, built[0].fs, built[0].T, r, couple.DUAL)
    subgrid.run(grid, [reg], 200, src, [])
    ref = reg.H.reshape(r * b, r * a)
    errs = []
    for q in (42, 84, 0):
        grid, emb, built = problem.build(w, rule=couple.DUAL, order=q)
        scheme.run(grid, emb, 200, src, [])
        Hzf = scheme.fine_fields(emb[0], r * a, r * b)[2]
        errs.append(np.linalg.norm(Hzf - ref) / np.linalg.norm(ref))
    assert errs[2] < 1e-9
    assert errs[1] < 0.1 * errs[0]
