"""Host-side checks of the C-ABI library (no GPU needed).

* the shared library loads and exports every function declared in
  include/fdtd.h;
* the library's FP64 reduced-model build (its own C++ code) agrees with the
  oracle's on every basis-independent quantity: achieved orders, the
  input-output (Markov) parameters of the run-time map of Eq. (23), and its
  eigenvalues;
* argument validation and the passivity / degeneracy errors.
"""
import os
import re

import numpy as np
import pytest

import paper_1609_07114_gb300 as pg
import workloads
from oracle import couple, problem, yee

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    names = declared_functions()
    assert len(names) >= 18
    L = pg.lib()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def rule_of(r):
    return pg.FDTD_RULE_DUAL if r == couple.DUAL else pg.FDTD_RULE_PAPER


def markov(P, Q, ny, K=10):
    out, X, Y = [], Q.copy(), np.eye(P.shape[0])[:, :ny]
    for _ in range(K):
        out += [X[:ny].copy(), Y[:ny].copy()]
        X, Y = P @ X, P @ Y
    return out


def compare_to_oracle(w, rule, order, tol=1e-9):
    grid, emb, built = problem.build(w, rule=rule, order=order)
    rd = w["roms"][0]
    b = built[0]
    q = rd["q"] if order is None else order
    m = pg.rom_build(rd["a"], rd["b"], rd["r"], w["dx"], w["dy"], w["dt"], rd["eps_r"],
                     rd["sigma"], q, rule=rule_of(rule), f0=rd["f0"])
    assert (m.qE, m.qH) == (b.rom.qE, b.rom.qH)
    itf = grid.interfaces[0]
    P, Q = m.couple(itf.eps_b / yee.EPS0, itf.sig_b)
    ny = itf.ny_
    for a_, b_ in zip(markov(b.cpl.P, b.cpl.Q, ny), markov(P, Q, ny)):
        assert np.linalg.norm(a_ - b_) <= tol * max(np.linalg.norm(a_), 1e-300)
    ev_o = np.sort(np.abs(np.linalg.eigvals(b.cpl.P)))
    ev_p = np.sort(np.abs(np.linalg.eigvals(P)))
    assert np.abs(ev_o - ev_p).max() < 1e-8
    # reported smax of Eq. (27) (as a fraction of 2/dt) matches the oracle
    assert abs(m.report.smax_before - b.s_before[0] * w["dt"] / 2) < 1e-8
    return m, b


def small_region(a=4, b=3, r=2, q=0, lossy=True, seed=0, dt_fac=0.9, nx=14, ny=13):
    rng = np.random.default_rng(seed)
    dx, dy = 1e-3, 1.2e-3
    ef = 1 + 3 * rng.random((r * b, r * a))
    sf = 0.2 * rng.random((r * b, r * a)) if lossy else np.zeros((r * b, r * a))
    return dict(nx=nx, ny=ny, dx=dx, dy=dy, dt=dt_fac * yee.cfl_limit(dx / r, dy / r),
                eps_r=1 + 2 * rng.random((ny, nx)), sigma=0.02 * rng.random((ny, nx)),
                roms=[dict(i0=5, j0=4, a=a, b=b, r=r, eps_r=ef, sigma=sf, q=q, f0=30e9)],
                sources=[], probes=[], nsteps=0)


@pytest.mark.parametrize("rule,order", [(couple.DUAL, 60), (couple.DUAL, 120)])
def test_rom_build_matches_oracle_cavity(rule, order):
    compare_to_oracle(workloads.cavity_60(10), rule, order)


@pytest.mark.parametrize("rule", [couple.PAPER, couple.DUAL])
def test_full_order_build_matches_oracle(rule):
    compare_to_oracle(small_region(), rule, 0)


def test_cfl_extension_matches_oracle():
    w = small_region(dt_fac=1.9, lossy=False)
    m, b = compare_to_oracle(w, couple.DUAL, 0, tol=1e-8)
    assert m.report.n_clamped > 0 and m.report.smax_before > 1.0
    assert m.report.smax_after <= 0.99 + 1e-12
    assert m.report.min_eig_R > 0


def test_reduced_blocks_are_passive():
    w = workloads.cavity_60(10)
    rd = w["roms"][0]
    m = pg.rom_build(rd["a"], rd["b"], rd["r"], w["dx"], w["dy"], w["dt"], rd["eps_r"], rd["sigma"], 80)
    R11, R22, Kt, Sig, LE = m.blocks()
    dt = w["dt"]
    R = np.block([[R11 / dt, -Kt / 2], [-Kt.T / 2, R22 / dt]])
    assert np.linalg.eigvalsh(R)[0] > 0                       # Eq. (26a)
    assert np.linalg.eigvalsh(Sig)[0] > -1e-12 * np.abs(Sig).max()   # Eq. (26b)
    assert m.report.cond3_residual < 1e-14                     # Eq. (26c)


def test_paper_rule_reduced_is_rejected():
    w = workloads.cavity_60(10)
    rd = w["roms"][0]
    m = pg.rom_build(rd["a"], rd["b"], rd["r"], w["dx"], w["dy"], w["dt"], rd["eps_r"], rd["sigma"],
                     60, rule=pg.FDTD_RULE_PAPER)
    with pytest.raises(pg.FdtdError) as ei:
        m.couple(np.ones(40), np.zeros(40))
    assert ei.value.code == -5


def test_not_passive_without_extension():
    w = small_region(dt_fac=1.9, lossy=False)
    rd = w["roms"][0]
    m = pg.rom_build(rd["a"], rd["b"], rd["r"], w["dx"], w["dy"], w["dt"], rd["eps_r"], rd["sigma"],
                     0, gamma=0.0)
    assert m.report.smax_after > 1.0
    with pytest.raises(pg.FdtdError) as ei:
        m.couple(np.ones(14), np.zeros(14))
    assert ei.value.code == -4


def test_bad_descriptors():
    with pytest.raises(pg.FdtdError) as ei:
        pg.rom_build(2, 2, 2, 1e-3, 1e-3, 1e-13, np.ones(16), -np.ones(16), 0)
    assert ei.value.code == -1
    with pytest.raises(pg.FdtdError):
        pg.rom_build(2, 2, 2, 1e-3, 1e-3, 1e-13, np.ones(16), np.zeros(16), 3)   # odd order
    assert abs(pg.fdtd_cfl_limit(1e-3, 2e-3) - yee.cfl_limit(1e-3, 2e-3)) < 1e-25


@pytest.mark.parametrize("order", [60, 120])
def test_projection_bases_span_the_oracle_bases(order):
    """rom_get_basis: orthonormal V1, V2 spanning the oracle's subspaces
    (principal angles ~ 0; the model depends only on the spans)."""
    w = workloads.cavity_60(10)
    m, b = compare_to_oracle(w, couple.DUAL, order)
    V1, V2 = m.basis()
    for Vg, Vo in ((V1, b.rom.V1), (V2, b.rom.V2)):
        assert Vg.shape == Vo.shape
        assert np.abs(Vg.T @ Vg - np.eye(Vg.shape[1])).max() < 1e-10
        cosines = np.linalg.svd(Vg.T @ Vo, compute_uv=False)
        assert cosines.min() > 1 - 1e-8
