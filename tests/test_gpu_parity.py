"""GPU parity: the CUDA time-marching path (through the C ABI) against the
FP64 oracle on the same seeded inputs.

Tolerance: relative L2 error <= 1e-4 on probe waveforms and on final fields.
The GPU steps FP32 fields with FP32 edge coefficients computed from FP32 cell
materials; the oracle steps FP64.  The gap is FP32 rounding (about 1e-7 per
operation, accumulated as a random walk over the steps) plus a phase drift
from coefficient rounding (FP32 materials and the hardware reciprocal in the
edge coefficients, relative ~1e-7 per wave speed, times the phase
travelled), both well below 1e-4 at these sizes and step counts.  Each side
builds its own reduced models (the library in C++, the oracle in numpy);
the two agree to 1e-12 on every input-output quantity (test_library_host).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1609_07114_gb300 as pg
import workloads
from oracle import couple, problem, scheme, yee

pytestmark = pytest.mark.gpu
TOL = 1e-4


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def gpu_context(ws, rule=pg.FDTD_RULE_DUAL, order=None):
    """One context holding every workload in ws (same dx, dy, dt)."""
    w0 = ws[0]
    ctx = pg.FdtdContext(w0["dx"], w0["dy"], w0["dt"], [(w["eps_r"], w["sigma"]) for w in ws])
    models = []
    for s, w in enumerate(ws):
        for rd in w["roms"]:
            q = rd["q"] if order is None else order
            m = pg.rom_build(rd["a"], rd["b"], rd["r"], w["dx"], w["dy"], w["dt"], rd["eps_r"],
                             rd["sigma"], q, rule=rule, f0=rd["f0"])
            ctx.rom_embed(m, s, rd["i0"], rd["j0"])
            models.append(m)
    return ctx, models


def gpu_run(ctx, ws, nsteps):
    srcs, probes = [], []
    keep = []
    for s, w in enumerate(ws):
        for so in w["sources"]:
            t = torch.tensor(np.asarray(so["wave"][:nsteps], np.float32), device="cuda")
            keep.append(t)
            srcs.append(dict(so, sim=s, wave=t))
        probes += [(s, i, j) for (i, j) in w["probes"]]
    out = torch.zeros((nsteps, len(probes)), dtype=torch.float32, device="cuda")
    ctx.fdtd_run(nsteps, srcs, probes, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def oracle_run(w, nsteps, rule=couple.DUAL, order=None):
    out, st, grid, emb, built = problem.run(w, nsteps, rule=rule, order=order)
    return out, st


def check_fields(ctx, sim, st):
    Ex, Ey, Hz = ctx.get_fields(sim)
    assert rel_l2(Ex, st.Ex) < TOL
    assert rel_l2(Ey, st.Ey) < TOL
    assert rel_l2(Hz, st.Hz) < TOL


def test_cavity_60_full_length():
    """60 x 60 PEC cavity, 10 x 10-cell region at r = 3, q = 60, 2000 steps."""
    w = workloads.cavity_60(2000)
    ctx, _ = gpu_context([w])
    g = gpu_run(ctx, [w], 2000)
    o, st = oracle_run(w, 2000)
    assert rel_l2(g, o) < TOL
    check_fields(ctx, 0, st)


def test_multi_tile_ragged_lossy_grid():
    """Several tiles in x and y with ragged tails, three lossy reduced
    models, a point source and a line source, probes beside the regions."""
    w = workloads.random_grid(7, 700, 150, 3, 6, 3, 40, 400, n_probes=12)
    w["sources"].append(dict(comp=1, i=3, j=10, len=100, wave=workloads.diff_gaussian(400, w["dt"], 20e9)))
    for rd in w["roms"]:
        w["probes"] += [(rd["i0"] - 1, rd["j0"]), (rd["i0"] + rd["a"], rd["j0"] + rd["b"] - 1)]
    ctx, _ = gpu_context([w])
    g = gpu_run(ctx, [w], 400)
    o, st = oracle_run(w, 400)
    assert rel_l2(g, o) < TOL
    check_fields(ctx, 0, st)


def test_batch_of_uneven_grids():
    """Three simulations of different sizes advance in one context; each
    matches its own oracle run."""
    ws = [workloads.random_grid(10 + k, nx, ny, 1, 5, 3, 30, 300, n_probes=4)
          for k, (nx, ny) in enumerate([(130, 97), (64, 200), (257, 33)])]
    dt = ws[0]["dt"]
    for w in ws:
        assert w["dt"] == dt
    ctx, _ = gpu_context(ws)
    g = gpu_run(ctx, ws, 300)
    col = 0
    for s, w in enumerate(ws):
        o, st = oracle_run(w, 300)
        np_ = len(w["probes"])
        assert rel_l2(g[:, col:col + np_], o) < TOL
        check_fields(ctx, s, st)
        col += np_


@pytest.mark.parametrize("rule", [pg.FDTD_RULE_PAPER, pg.FDTD_RULE_DUAL])
def test_full_order_model(rule):
    """V = I (no reduction) through the same kernels, both interpolation rules."""
    w = workloads.random_grid(20, 90, 70, 1, 4, 2, 0, 300, n_probes=6)
    ctx, _ = gpu_context([w], rule=rule, order=0)
    g = gpu_run(ctx, [w], 300)
    o, st = oracle_run(w, 300, rule=couple.PAPER if rule == pg.FDTD_RULE_PAPER else couple.DUAL, order=0)
    assert rel_l2(g, o) < TOL
    check_fields(ctx, 0, st)


def test_cfl_extension_run():
    """dt = 1.9 x the fine-mesh CFL limit (r = 2), extended model."""
    w = workloads.random_grid(21, 120, 90, 2, 4, 2, 0, 400, dt_factor=1.9, n_probes=6)
    ctx, models = gpu_context([w], order=0)
    assert any(m.report.n_clamped > 0 for m in models)
    g = gpu_run(ctx, [w], 400)
    o, st = oracle_run(w, 400, order=0)
    assert rel_l2(g, o) < TOL


def test_random_initial_state_and_tiny_grid():
    """Arbitrary initial fields (set through the C ABI), a 3 x 5 grid and a
    grid whose width is not a multiple of the vector width."""
    for (nx, ny) in [(3, 5), (37, 29)]:
        rng = np.random.default_rng(nx)
        dx = dy = 1e-3
        dt = 0.9 * yee.cfl_limit(dx, dy)
        eps = 1 + 3 * rng.random((ny, nx))
        sig = 0.03 * rng.random((ny, nx))
        grid = yee.CoarseGrid(nx, ny, dx, dy, dt, eps, sig)
        st = scheme.State(*grid.zeros())
        st.Ex = np.where(grid.ex_upd, rng.standard_normal(st.Ex.shape), 0.0)
        st.Ey = np.where(grid.ey_upd, rng.standard_normal(st.Ey.shape), 0.0)
        st.Hz = rng.standard_normal(st.Hz.shape) / 377
        ctx = pg.FdtdContext(dx, dy, dt, [(eps, sig)])
        ctx.set_fields(0, st.Ex, st.Ey, st.Hz)
        probes = [(0, 0), (nx - 1, ny - 1)]
        out = torch.zeros((50, 2), dtype=torch.float32, device="cuda")
        ctx.fdtd_run(50, [], [(0, i, j) for i, j in probes], out)
        o, st, _ = scheme.run(grid, [], 50, probes=probes, st=st)
        assert rel_l2(out.cpu().numpy(), o) < TOL
        check_fields(ctx, 0, st)
        assert ctx.step_count() == 50


def test_run_host_equals_run():
    """The host-buffer entry point computes exactly what the device one does."""
    w = workloads.cavity_60(300)
    ctx1, _ = gpu_context([w])
    g1 = gpu_run(ctx1, [w], 300)
    ctx2, _ = gpu_context([w])
    g2 = ctx2.fdtd_run_host(300, [dict(s, sim=0) for s in w["sources"]], [(0, i, j) for i, j in w["probes"]])
    np.testing.assert_array_equal(g1, g2)


def test_split_runs_equal_one_run():
    """37 + 100 + 1 steps (graph chunks and a remainder, parity carried over)
    equal one run of 138 steps, bit for bit."""
    w = workloads.cavity_60(138)
    ctx1, _ = gpu_context([w])
    g1 = gpu_run(ctx1, [w], 138)
    ctx2, _ = gpu_context([w])
    parts, n0 = [], 0
    for n in (37, 100, 1):
        wn = dict(w, sources=[dict(s, wave=s["wave"][n0:n0 + n]) for s in w["sources"]])
        parts.append(gpu_run(ctx2, [wn], n))
        n0 += n
    np.testing.assert_array_equal(g1, np.concatenate(parts))
    assert ctx2.step_count() == 138


def test_repeated_runs_reuse_and_rebuild_their_lists(monkeypatch):
    """Runs that repeat the previous run's sources and probes keep the device
    lists (only the run record and the wave pointers are copied, without
    waiting for the stream); a run with other probes, and one after a
    re-plan, rebuild them.  On the two-step path with chained models, 30 +
    30 + 20 (other probes) + 20 + 20 (after the autotuner) steps, issued
    without synchronising in between, equal one run of 120 steps bit for
    bit."""
    monkeypatch.setenv("FDTD_TB", "1")
    w = workloads.random_grid(3, 700, 300, 3, 12, 3, 40, 120)
    ctx1, _ = gpu_context([w])
    assert ctx1.steps_per_launch() == 2
    g1 = gpu_run(ctx1, [w], 120)
    F1 = ctx1.get_fields(0)
    ctx2, _ = gpu_context([w])
    waves = [torch.tensor(np.asarray(so["wave"][:120], np.float32), device="cuda") for so in w["sources"]]
    probes = [(0, i, j) for (i, j) in w["probes"]]
    other = probes[4::-1]
    outs, n0 = [], 0
    for n, pr in ((30, probes), (30, probes), (20, other), (20, probes), (20, probes)):
        if n0 == 100:
            ctx2.autotune()
        src = [dict(so, sim=0, wave=wv[n0:n0 + n]) for so, wv in zip(w["sources"], waves)]
        out = torch.zeros((n, len(pr)), dtype=torch.float32, device="cuda")
        ctx2.fdtd_run(n, src, pr, out)
        outs.append((n0, n, pr, out))
        n0 += n
    torch.cuda.synchronize()
    for n0, n, pr, out in outs:
        if pr is probes:
            np.testing.assert_array_equal(out.cpu().numpy(), g1[n0:n0 + n])
    for a, b in zip(ctx2.get_fields(0), F1):
        np.testing.assert_array_equal(a, b)
    assert ctx2.step_count() == 120


def test_invalid_inputs_are_rejected():
    w = workloads.cavity_60(10)
    ctx, _ = gpu_context([w])
    rd = w["roms"][0]
    bad_src = [dict(comp=1, i=rd["i0"], j=rd["j0"], len=1, wave=torch.zeros(10, device="cuda"))]
    with pytest.raises(pg.FdtdError):                 # source on an interface edge
        ctx.fdtd_run(10, bad_src, [], None)
    with pytest.raises(pg.FdtdError):                 # probe outside the grid
        ctx.fdtd_run(10, [], [(0, 60, 0)], torch.zeros((10, 1), device="cuda"))
    m = pg.rom_build(rd["a"], rd["b"], rd["r"], w["dx"], w["dy"], w["dt"], rd["eps_r"], rd["sigma"], 20)
    with pytest.raises(pg.FdtdError):                 # overlaps the first region
        ctx.rom_embed(m, 0, rd["i0"] + 2, rd["j0"] + 2)
    with pytest.raises(pg.FdtdError) as ei:           # dt above the coarse CFL limit
        pg.FdtdContext(1e-3, 1e-3, 1.01 * yee.cfl_limit(1e-3, 1e-3), [(np.ones((8, 8)), np.zeros((8, 8)))])
    assert ei.value.code == -3
    ctx.fdtd_run(0, [], [], None)                    # empty run is a no-op


def test_full_size_grid_sampled_outputs():
    """4096^2 grid with eight r = 4, q = 200 models, in the launch
    configuration the benchmark times.  After N steps from rest only cells
    within N of the source can be nonzero; the oracle recomputes that window
    (and every model inside it) exactly, and the probes and sampled fields
    are compared one by one."""
    N = 160
    w = workloads.grid_4096(N)
    ctx, _ = gpu_context([w])
    src = w["sources"][0]
    si, sj = src["i"], src["j"]
    # window around the source, enlarged to contain whole regions
    lo_i, hi_i, lo_j, hi_j = si - N - 3, si + N + 3, sj - N - 3, sj + N + 3
    changed = True
    while changed:
        changed = False
        for rd in w["roms"]:
            inside = not (rd["i0"] + rd["a"] < lo_i or rd["i0"] > hi_i or rd["j0"] + rd["b"] < lo_j or rd["j0"] > hi_j)
            if inside and not (lo_i < rd["i0"] - 1 and rd["i0"] + rd["a"] + 1 < hi_i
                               and lo_j < rd["j0"] - 1 and rd["j0"] + rd["b"] + 1 < hi_j):
                lo_i, hi_i = min(lo_i, rd["i0"] - 3), max(hi_i, rd["i0"] + rd["a"] + 3)
                lo_j, hi_j = min(lo_j, rd["j0"] - 3), max(hi_j, rd["j0"] + rd["b"] + 3)
                changed = True
    lo_i, lo_j = max(lo_i, 0), max(lo_j, 0)
    hi_i, hi_j = min(hi_i, w["nx"]), min(hi_j, w["ny"])
    win_probes = [(i, j) for (i, j) in w["probes"] if lo_i <= i < hi_i and lo_j <= j < hi_j]
    win_probes += [(min(si + 5, hi_i - 1), sj), (si, min(sj + 20, hi_j - 1))]
    w["probes"] = win_probes
    g = gpu_run(ctx, [w], N)
    sub = dict(w, nx=hi_i - lo_i, ny=hi_j - lo_j,
               eps_r=w["eps_r"][lo_j:hi_j, lo_i:hi_i], sigma=w["sigma"][lo_j:hi_j, lo_i:hi_i],
               roms=[dict(rd, i0=rd["i0"] - lo_i, j0=rd["j0"] - lo_j) for rd in w["roms"]
                     if lo_i < rd["i0"] and rd["i0"] + rd["a"] < hi_i and lo_j < rd["j0"] and rd["j0"] + rd["b"] < hi_j],
               sources=[dict(src, i=si - lo_i, j=sj - lo_j)],
               probes=[(i - lo_i, j - lo_j) for (i, j) in win_probes])
    o, st = oracle_run(sub, N)
    assert rel_l2(g, o) < TOL
    Ex, Ey, Hz = ctx.get_fields(0)
    assert rel_l2(Hz[lo_j:hi_j, lo_i:hi_i], st.Hz) < TOL
    assert rel_l2(Ex[lo_j:hi_j, lo_i:hi_i], st.Ex[:-1, :]) < TOL
    # causality: nothing outside the window moved
    mask = np.ones_like(Hz, dtype=bool)
    mask[lo_j:hi_j, lo_i:hi_i] = False
    assert np.abs(Hz[mask]).max() == 0.0


def test_batched_layout_parity():
    """Two simulations of the batched layout (four shared models of orders
    40-320 in each, vacuum rings, per-simulation sources), advanced together;
    each matches its own oracle run."""
    N = 500
    wb = workloads.batched_256(N, per_size=1, sizes=(128, 256))
    ws = []
    for s in wb["sims"]:
        si, sj = s["source"]["i"], s["source"]["j"]
        near = [(min(max(si + di, 1), s["nx"] - 2), min(max(sj + dj, 1), s["ny"] - 2))
                for di, dj in ((6, 0), (0, -9), (-12, 4))]
        near += [(i0 - 1, j0 + 2) for (_, i0, j0) in s["place"]]
        ws.append(dict(nx=s["nx"], ny=s["ny"], dx=wb["dx"], dy=wb["dy"], dt=wb["dt"], eps_r=s["eps_r"],
                       sigma=s["sigma"], roms=[dict(wb["models"][k], i0=i0, j0=j0) for (k, i0, j0) in s["place"]],
                       sources=[s["source"]], probes=[s["probe"]] + near, nsteps=N))
    ctx = pg.FdtdContext(wb["dx"], wb["dy"], wb["dt"], [(w["eps_r"], w["sigma"]) for w in ws])
    models = [pg.rom_build(md["a"], md["b"], md["r"], wb["dx"], wb["dy"], wb["dt"], md["eps_r"],
                           md["sigma"], md["q"], f0=md["f0"]) for md in wb["models"]]
    insts = []
    for s, sim in enumerate(wb["sims"]):
        for (k, i0, j0) in sim["place"]:
            insts.append(ctx.rom_embed(models[k], s, i0, j0))
    # the vacuum rings make the two simulations' maps identical
    P0, _ = ctx.get_rom_map(insts[3])
    P1, _ = ctx.get_rom_map(insts[7])
    np.testing.assert_array_equal(P0, P1)
    g = gpu_run(ctx, ws, N)
    col = 0
    for s, w in enumerate(ws):
        o, st = oracle_run(w, N)
        npr = len(w["probes"])
        assert np.abs(o).max() > 1e-6
        assert rel_l2(g[:, col:col + npr], o) < TOL
        check_fields(ctx, s, st)
        col += npr


def test_save_load_resume_is_bit_identical():
    """Checkpoint / resume: N steps = k steps + save + (fresh context) load +
    N - k steps, bit for bit."""
    w = workloads.random_grid(70, 150, 120, 2, 5, 3, 30, 300, n_probes=4)
    ctx1, _ = gpu_context([w])
    g1 = gpu_run(ctx1, [w], 300)
    ctx2, _ = gpu_context([w])
    wa = dict(w, sources=[dict(s, wave=s["wave"][:110]) for s in w["sources"]])
    ga = gpu_run(ctx2, [wa], 110)
    blob = ctx2.save_state()
    ctx3, _ = gpu_context([w])
    ctx3.load_state(blob)
    assert ctx3.step_count() == 110
    wb = dict(w, sources=[dict(s, wave=s["wave"][110:]) for s in w["sources"]])
    gb = gpu_run(ctx3, [wb], 190)
    np.testing.assert_array_equal(g1, np.concatenate([ga, gb]))
    with pytest.raises(pg.FdtdError):
        ctx3.load_state(blob[:-4])


def test_non_finite_state_is_reported():
    """Non-finite values reaching a probe make the host entry point return
    FDTD_EUNSTABLE (and fdtd_energy too); a model that is not passive at the
    run's dt is refused at embedding (FDTD_ENOTPASSIVE)."""
    w = workloads.random_grid(71, 60, 60, 1, 4, 2, 0, 50, dt_factor=1.9, n_probes=2)
    rd = w["roms"][0]
    m = pg.rom_build(rd["a"], rd["b"], rd["r"], w["dx"], w["dy"], w["dt"], rd["eps_r"], rd["sigma"], 0,
                     gamma=0.0)
    ctx = pg.FdtdContext(w["dx"], w["dy"], w["dt"], [(w["eps_r"], w["sigma"])])
    with pytest.raises(pg.FdtdError) as ei:
        ctx.rom_embed(m, 0, rd["i0"], rd["j0"])
    assert ei.value.code == -4
    Ex, Ey, Hz = ctx.get_fields(0)
    Hz[30, 30] = np.nan
    ctx.set_fields(0, Ex, Ey, Hz)
    with pytest.raises(pg.FdtdError) as ei:
        ctx.fdtd_run_host(5, [], [(0, 31, 30)])
    assert ei.value.code == -6
    with pytest.raises(pg.FdtdError) as ei:
        ctx.energy()
    assert ei.value.code == -6


@pytest.mark.parametrize("rpw", ["1", "2"])
def test_batched_layout_through_gemm_form(monkeypatch, rpw):
    """The same case with every shared map stepped as a GEMM (threshold 1),
    both CTA shapes of the GEMM form."""
    monkeypatch.setenv("FDTD_ROM_GEMM_MIN", "1")
    monkeypatch.setenv("FDTD_GEMM_RPW", rpw)
    test_batched_layout_parity()


def test_full_batched_256_sampled_simulations():
    """All 256 simulations of the batched configuration (four maps shared by
    64 simulations each, so the GEMM form with 16-row CTAs) in one context,
    as the benchmark runs them; one simulation of each size is recomputed by
    the oracle and compared probe by probe and field by field."""
    N = 300
    wb = workloads.batched_256(N)
    ctx = pg.FdtdContext(wb["dx"], wb["dy"], wb["dt"], [(s["eps_r"], s["sigma"]) for s in wb["sims"]])
    models = [pg.rom_build(md["a"], md["b"], md["r"], wb["dx"], wb["dy"], wb["dt"], md["eps_r"],
                           md["sigma"], md["q"], f0=md["f0"]) for md in wb["models"]]
    for k, s in enumerate(wb["sims"]):
        for (mi, i0, j0) in s["place"]:
            ctx.rom_embed(models[mi], k, i0, j0)
    waves, srcs, probes = [], [], []
    for k, s in enumerate(wb["sims"]):
        t = torch.tensor(np.asarray(s["source"]["wave"], np.float32), device="cuda")
        waves.append(t)
        srcs.append(dict(s["source"], sim=k, wave=t))
        si, sj = s["source"]["i"], s["source"]["j"]
        probes.append((k, s["probe"][0], s["probe"][1]))
        probes.append((k, min(si + 5, s["nx"] - 2), sj))
    out = torch.zeros((N, len(probes)), dtype=torch.float32, device="cuda")
    ctx.fdtd_run(N, srcs, probes, out)
    g = out.cpu().numpy()
    for k in (0, 64, 128, 192):          # one of each size
        s = wb["sims"][k]
        w = dict(nx=s["nx"], ny=s["ny"], dx=wb["dx"], dy=wb["dy"], dt=wb["dt"], eps_r=s["eps_r"],
                 sigma=s["sigma"], roms=[dict(wb["models"][mi], i0=i0, j0=j0) for (mi, i0, j0) in s["place"]],
                 sources=[s["source"]], probes=[p[1:] for p in probes[2 * k:2 * k + 2]], nsteps=N)
        o, st = oracle_run(w, N)
        assert np.abs(o).max() > 0
        assert rel_l2(g[:, 2 * k:2 * k + 2], o) < TOL
        check_fields(ctx, k, st)
