"""Pins for the oracle's CPML: it reduces to Eqs. (3), (5) when its
conductivity profile is zero, and it absorbs: the probe traces of a pulse in
an 80 x 80 grid with 10-cell layers on all sides equal, to ~1e-4 of the
peak, those of the same pulse in a 400 x 400 PEC grid whose wall echoes
cannot reach the probes in the window (the same grid without the layers is
off by ~100%).  A planted sign error in the auxiliary update is caught."""
import numpy as np
import pytest

import workloads
from oracle import cpml, problem, scheme, yee

DX = 1e-3
DT = 0.9 * yee.cfl_limit(DX, DX)
STEPS = 400
OFF = 25


def pulse_problem(n, pml=None, eps=None):
    c = n // 2
    w = dict(nx=n, ny=n, dx=DX, dy=DX, dt=DT, eps_r=np.ones((n, n)) if eps is None else eps,
             sigma=np.zeros((n, n)), roms=[],
             sources=[dict(comp=1, i=c, j=c, len=1, wave=workloads.diff_gaussian(STEPS, DT, 10e9))],
             probes=[(c + OFF, c), (c, c + OFF), (c + OFF, c + OFF), (c - OFF, c - 12)], nsteps=STEPS)
    if pml:
        w["pml"] = pml
    return w


@pytest.fixture(scope="module")
def reference():
    out, *_ = problem.run(pulse_problem(400), STEPS)
    return out


def err(out, ref):
    return np.abs(out - ref).max() / np.abs(ref).max()


def test_zero_profile_is_plain_yee():
    rng = np.random.default_rng(3)
    n = 30
    eps = 1 + 3 * rng.random((n, n))
    a = pulse_problem(n, dict(n=6, sides=15, sigma_max=0.0, kappa_max=1.0, alpha_max=0.0), eps=eps)
    b = pulse_problem(n, None, eps=eps)
    a["probes"] = b["probes"] = [(3, 4), (20, 25), (15, 1)]
    oa, sa, *_ = problem.run(a, 150)
    ob, sb, *_ = problem.run(b, 150)
    assert np.abs(oa - ob).max() <= 1e-12 * np.abs(ob).max()
    assert np.abs(sa.Ex - sb.Ex).max() <= 1e-12 * np.abs(sb.Ex).max()


@pytest.mark.parametrize("prof", [dict(), dict(kappa_max=5.0, alpha_max=0.05), dict(m=4.0)])
def test_layers_absorb(reference, prof):
    out, *_ = problem.run(pulse_problem(80, dict(n=10, sides=15, **prof)), STEPS)
    assert err(out, reference) < 1e-3
    pec, *_ = problem.run(pulse_problem(80), STEPS)
    assert err(pec, reference) > 0.3


def test_layers_on_two_sides_only(reference):
    """Layers on W and E only: the traces match until the echo of the S/N
    PEC walls (36 cells away from the source) can reach the probes."""
    out, *_ = problem.run(pulse_problem(80, dict(n=10, sides=cpml.SIDE_W | cpml.SIDE_E)), STEPS)
    c_cells = 3e8 * DT / DX                      # cells per step (~0.64)
    first_echo = int((40 + 40 - OFF) / c_cells) - 10
    assert err(out[:first_echo], reference[:first_echo]) < 1e-3
    assert err(out, reference) > 1e-2


def test_planted_sign_error_is_caught(reference, monkeypatch):
    orig = cpml.CPML.__init__

    def bad_init(self, *a, **k):
        orig(self, *a, **k)
        self.ax_h, self.ay_h = -self.ax_h, -self.ay_h

    monkeypatch.setattr(cpml.CPML, "__init__", bad_init)
    out, *_ = problem.run(pulse_problem(80, dict(n=10, sides=15)), STEPS)
    assert not err(out, reference) < 1e-3
