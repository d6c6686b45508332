"""GPU storage function (Sec. V, Appendix A) and long-run stability.

* the GPU's energy after N steps equals the oracle's (its own run, its own
  reduced models: the storage function does not depend on the model basis);
* a lossless grid with four embedded models, run 10^6 steps at twice the
  fine-mesh CFL limit (the Sec. V-E extension active on the largest model):
  after the source has died out the energy stays constant within FP32 drift
  and shows no upward trend (Theorem 2);
* with losses the energy never increases.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1609_07114_gb300 as pg
import workloads
from oracle import problem, scheme

pytestmark = pytest.mark.gpu


def build_ctx(w):
    ctx = pg.FdtdContext(w["dx"], w["dy"], w["dt"], [(w["eps_r"], w["sigma"])])
    models = []
    for rd in w["roms"]:
        m = pg.rom_build(rd["a"], rd["b"], rd["r"], w["dx"], w["dy"], w["dt"], rd["eps_r"],
                         rd["sigma"], rd["q"], f0=rd["f0"])
        ctx.rom_embed(m, 0, rd["i0"], rd["j0"])
        models.append(m)
    return ctx, models


def run(ctx, w, n, with_source=True, n0=0):
    src = []
    if with_source:
        for so in w["sources"]:
            src.append(dict(so, sim=0, wave=torch.tensor(np.asarray(so["wave"][n0:n0 + n], np.float32),
                                                         device="cuda")))
    ctx.fdtd_run(n, src, [], None)


def test_energy_matches_oracle():
    w = workloads.random_grid(30, 200, 150, 2, 6, 3, 40, 300, n_probes=2)
    ctx, _ = build_ctx(w)
    run(ctx, w, 300)
    Wg = ctx.energy()[0]
    _, st, grid, emb, _ = problem.run(w, 300)
    Wo = scheme.energy(grid, st, emb)
    assert abs(Wg - Wo) < 1e-4 * abs(Wo)


def energy_trace(w, total, chunk, warm):
    ctx, models = build_ctx(w)
    run(ctx, w, warm)                       # the pulse, then silence
    W = [ctx.energy()[0]]
    done = warm
    while done < total:
        n = min(chunk, total - done)
        run(ctx, w, n, with_source=False)
        done += n
        W.append(ctx.energy()[0])
    return np.array(W), models


def test_lossless_energy_constant_over_1e6_steps():
    w = workloads.lattice_lossless(256, 1_000_000)
    W, models = energy_trace(w, 1_000_000, 50_000, 4000)
    assert any(m.report.n_clamped > 0 for m in models)       # CFL extension active
    assert np.all(np.isfinite(W))
    drift = np.abs(W / W[0] - 1.0).max()
    slope = np.polyfit(np.arange(W.size), W / W[0], 1)[0] * (W.size - 1)
    print(f"lossless 1e6 steps: max |W/W0 - 1| = {drift:.3e}, fitted trend = {slope:.3e}")
    assert drift < 1e-4
    assert slope < 1e-4


def test_lossy_energy_never_increases():
    w = workloads.lattice_lossless(192, 200_000, lossless=False)
    W, _ = energy_trace(w, 200_000, 10_000, 4000)
    assert np.all(np.diff(W) <= 1e-7 * W[0])
    assert W[-1] < W[0]
