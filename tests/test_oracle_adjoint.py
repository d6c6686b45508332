"""Pins for the FP64 oracle adjoint: central finite differences of the oracle's
own forward objective (J = sum of probe Hz^2, and a linear functional
L = sum c o of the probe series with a random cotangent c), on interior cells,
cells beside a model (whose material also enters the coupling of Eq. (19)),
the source cell, and source samples (J is quadratic and L linear in the
sources, so those difference quotients are exact up to rounding)."""
import copy

import numpy as np
import pytest

import workloads
from oracle import adjoint, couple, problem


def small_w(seed=50, q=20, r=2):
    w = workloads.random_grid(seed, 40, 34, 1, 5, r, q, 150, n_probes=3)
    rd = w["roms"][0]
    w["probes"] = w["probes"] + [(rd["i0"] - 1, rd["j0"] + 1)]
    return w


def fd(w, arr, i, j, h=1e-4, **kw):
    """Central difference of the oracle objective (J, or L = sum c o with a
    cotangent c given in kw) in one cell's material."""
    base = w[arr][j, i]
    hh = h * max(abs(base), 1.0)
    wp = copy.deepcopy(w)
    wp[arr][j, i] = base + hh
    wm = copy.deepcopy(w)
    wm[arr][j, i] = base - hh
    return (adjoint.objective(wp, **kw) - adjoint.objective(wm, **kw)) / (2 * hh)


@pytest.mark.parametrize("rule,order", [(couple.DUAL, None), (couple.DUAL, 0), (couple.PAPER, 0)])
def test_material_gradients_match_finite_differences(rule, order):
    w = small_w()
    J, deps, dsig, _ = adjoint.gradients(w, rule=rule, order=order)
    rd = w["roms"][0]
    i0, j0, a, b = rd["i0"], rd["j0"], rd["a"], rd["b"]
    cells = [(i0 - 1, j0 + 2), (i0 + a, j0 + 1), (i0 + 1, j0 - 1), (i0 + 2, j0 + b),   # ring cells
             (3, 4), (20, 15), (w["sources"][0]["i"], w["sources"][0]["j"])]
    for (i, j) in cells:
        for arr, g in (("eps_r", deps), ("sigma", dsig)):
            ref = fd(w, arr, i, j, rule=rule, order=order)
            scale = max(abs(ref), 1e-3 * np.abs(g).max())
            assert abs(g[j, i] - ref) <= 1e-6 * scale, (arr, i, j, g[j, i], ref)
    # covered cells are not coarse unknowns
    assert np.all(deps[j0:j0 + b, i0:i0 + a] == 0.0)


def test_source_gradient_is_exact():
    w = small_w()
    J, _, _, gsrc = adjoint.gradients(w)
    for n in (5, 40, 120):
        hh = 1e-2
        wp = copy.deepcopy(w)
        wp["sources"][0]["wave"][n] += hh
        wm = copy.deepcopy(w)
        wm["sources"][0]["wave"][n] -= hh
        ref = (adjoint.objective(wp) - adjoint.objective(wm)) / (2 * hh)
        assert abs(gsrc[0][n] - ref) <= 1e-9 * max(abs(ref), 1e-6 * np.abs(gsrc[0]).max())
    # J is quadratic in the sources: J = 1/2 s . grad_s J (Euler's theorem)
    s = w["sources"][0]["wave"][:150]
    assert abs(0.5 * float(s @ gsrc[0]) - J) < 1e-10 * J


def test_planted_mistake_is_caught(monkeypatch):
    """Drop the eps0 factor of the edge-to-cell chain rule (a plausible slip):
    the finite-difference pin fails."""
    w = small_w()
    i, j = 20, 15
    ref = fd(w, "eps_r", i, j)
    monkeypatch.setattr(adjoint, "EPS0", 1.0)
    _, deps, _, _ = adjoint.gradients(w)
    assert abs(deps[j, i] - ref) > 1e-3 * abs(ref)


def test_cotangent_gradients_match_finite_differences():
    """A random cotangent c of the probe series: the gradient of
    L = sum_n sum_p c[n][p] Hz^{n+1/2}(p) against central differences of L,
    on ring, interior and source cells and on source samples (L is linear in
    the sources: its difference quotient is exact)."""
    w = small_w(seed=52)
    c = np.random.default_rng(9).standard_normal((150, len(w["probes"])))
    L, deps, dsig, gsrc = adjoint.gradients(w, cotangent=c)
    rd = w["roms"][0]
    i0, j0, a, b = rd["i0"], rd["j0"], rd["a"], rd["b"]
    for (i, j) in [(i0 - 1, j0 + 2), (i0 + a, j0 + 1), (i0 + 1, j0 - 1), (5, 6), (22, 14),
                   (w["sources"][0]["i"], w["sources"][0]["j"])]:
        for arr, g in (("eps_r", deps), ("sigma", dsig)):
            ref = fd(w, arr, i, j, cotangent=c)
            scale = max(abs(ref), 1e-3 * np.abs(g).max())
            assert abs(g[j, i] - ref) <= 1e-6 * scale, (arr, i, j, g[j, i], ref)
    for n in (3, 60, 149):
        hh = 1e-2
        wp = copy.deepcopy(w)
        wp["sources"][0]["wave"][n] += hh
        wm = copy.deepcopy(w)
        wm["sources"][0]["wave"][n] -= hh
        ref = (adjoint.objective(wp, cotangent=c) - adjoint.objective(wm, cotangent=c)) / (2 * hh)
        assert abs(gsrc[0][n] - ref) <= 1e-9 * max(abs(ref), 1e-6 * np.abs(gsrc[0]).max())
    # L is linear in the sources: L = s . dL/ds
    s = w["sources"][0]["wave"][:150]
    assert abs(float(s @ gsrc[0]) - L) < 1e-10 * abs(L)
    # c = 2 o reproduces J's gradient
    J, dj, _, _ = adjoint.gradients(w)
    out, *_ = problem.run(w)
    _, dj2, _, _ = adjoint.gradients(w, cotangent=2.0 * out)
    np.testing.assert_allclose(dj2, dj, rtol=1e-12, atol=1e-12 * np.abs(dj).max())


def test_planted_cotangent_slip_is_caught():
    """Seed the probe term one step late (c[n-1] at reverse step n, a
    plausible indexing slip): the source-sample pin fails."""
    w = small_w(seed=52)
    c = np.random.default_rng(9).standard_normal((150, len(w["probes"])))
    _, _, _, good = adjoint.gradients(w, cotangent=c)
    late = np.vstack([np.zeros((1, c.shape[1])), c[:-1]])
    _, _, _, bad = adjoint.gradients(w, cotangent=late)
    n = 60
    hh = 1e-2
    wp = copy.deepcopy(w)
    wp["sources"][0]["wave"][n] += hh
    wm = copy.deepcopy(w)
    wm["sources"][0]["wave"][n] -= hh
    ref = (adjoint.objective(wp, cotangent=c) - adjoint.objective(wm, cotangent=c)) / (2 * hh)
    assert abs(good[0][n] - ref) <= 1e-9 * abs(ref)
    assert abs(bad[0][n] - ref) > 1e-3 * abs(ref)
