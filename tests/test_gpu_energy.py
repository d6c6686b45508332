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


def test_batched_chain_energy_constant_over_1e6_steps(monkeypatch):
    """The batched layout (four simulations of two sizes sharing the four
    models, made lossless: sigma = 0 in the coarse cells and the fine
    regions) on the benchmark's two-step path with the shared maps as GEMMs
    in the zone chain, 10^6 steps: after the pulse the storage function stays
    constant within FP32 drift, with no upward trend."""
    monkeypatch.setenv("FDTD_TB", "1")
    monkeypatch.setenv("FDTD_ROM_GEMM_MIN", "1")
    monkeypatch.delenv("FDTD_TB_CHAIN", raising=False)
    wb = workloads.batched_256(4000, per_size=2, sizes=(128, 256))
    models = [pg.rom_build(md["a"], md["b"], md["r"], wb["dx"], wb["dy"], wb["dt"], md["eps_r"],
                           0.0 * md["sigma"], md["q"], f0=md["f0"]) for md in wb["models"]]
    ctx = pg.FdtdContext(wb["dx"], wb["dy"], wb["dt"], [(s["eps_r"], 0.0 * s["sigma"]) for s in wb["sims"]])
    for k, s in enumerate(wb["sims"]):
        for (mi, i0, j0) in s["place"]:
            ctx.rom_embed(models[mi], k, i0, j0)
    plan = ctx.plan()
    assert plan["steps_per_launch"] == 2 and plan["chained_models"] == 16
    src = [dict(s["source"], sim=k, wave=torch.tensor(np.asarray(s["source"]["wave"][:4000], np.float32),
                                                      device="cuda")) for k, s in enumerate(wb["sims"])]
    ctx.fdtd_run(4000, src, [], None)          # the pulses, then silence
    W = [ctx.energy()]
    for _ in range(20):
        ctx.fdtd_run(49_800, [], [], None)
        W.append(ctx.energy())
    W = np.array(W)
    assert np.all(np.isfinite(W)) and np.all(W[0] > 0)
    rel = W / W[0] - 1.0
    slope = np.array([np.polyfit(np.arange(W.shape[0]), W[:, k] / W[0, k], 1)[0] * (W.shape[0] - 1)
                      for k in range(W.shape[1])])
    print(f"batched chain 1e6 steps: max |W/W0 - 1| = {np.abs(rel).max():.3e}, trends = {slope}")
    assert np.abs(rel).max() < 1e-4
    assert np.all(slope < 1e-4)


def test_adjoint_sweep_stays_bounded_over_1e6_steps(monkeypatch):
    """The reverse sweep over 10^6 steps of a lossless grid with models at
    twice the fine-mesh CFL limit (the Eq. (27) extension active): the
    vector-Jacobian product seeded only in the last 1000 steps at one probe
    carries the adjoint fields back through every step; the source gradient
    stays finite and does not grow as it is carried back (its largest value
    in the first 10^5 steps is within a factor 10 of that in the last 10^5).
    The transposed scheme inherits the forward scheme's stability."""
    monkeypatch.delenv("FDTD_TB", raising=False)
    N = 1_000_000
    w = workloads.lattice_lossless(64, N)
    ctx, _ = build_ctx(w)
    so = w["sources"][0]
    wave = torch.zeros(N, dtype=torch.float32, device="cuda")
    wave[:4000] = torch.tensor(np.asarray(so["wave"][:4000], np.float32), device="cuda")
    pi, pj = w["nx"] // 2, w["ny"] // 2 - 2                 # between the regions, near the source
    assert not any(rd["i0"] <= pi < rd["i0"] + rd["a"] and rd["j0"] <= pj < rd["j0"] + rd["b"] for rd in w["roms"])
    probes = [(0, pi, pj)]
    cot = torch.zeros((N, 1), dtype=torch.float32, device="cuda")
    cot[-1000:, 0] = 1.0
    ge, gs, gw = ctx.fdtd_vjp(N, [dict(so, sim=0, wave=wave)], probes, cot, ckpt_every=2000)
    g = gw[0].abs().cpu().numpy()
    assert np.all(np.isfinite(g)) and np.all(np.isfinite(ge[0].cpu().numpy()))
    early, late = g[:100_000].max(), g[-100_000:].max()
    print(f"adjoint over 1e6 steps: max |dL/dJ| first 1e5 steps {early:.3e}, last 1e5 {late:.3e}")
    assert late > 0 and early < 10.0 * late
