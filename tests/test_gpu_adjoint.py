"""GPU discrete adjoint (fdtd_grad) against the FP64 oracle adjoint, which is
itself pinned to central finite differences (test_oracle_adjoint).

Tolerance: relative L2 error <= 1e-3 on the gradients (FP32 forward and
adjoint arithmetic accumulated over a few hundred steps), 1e-4 on J.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1609_07114_gb300 as pg
from paper_1609_07114_gb300.autograd import FdtdFn, FdtdSpec, probe_energy
import workloads
from oracle import adjoint

pytestmark = pytest.mark.gpu
GTOL = 1e-3


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def grad_case(seed=60, nx=100, ny=80, nsteps=300):
    w = workloads.random_grid(seed, nx, ny, 2, 5, 2, 20, nsteps, n_probes=3)
    for rd in w["roms"]:
        w["probes"].append((rd["i0"] - 1, rd["j0"] + 2))
        w["probes"].append((rd["i0"] + rd["a"], rd["j0"] + 1))
    si, sj = w["sources"][0]["i"], w["sources"][0]["j"]
    w["probes"].append((min(si + 4, nx - 1), sj))
    return w


def gpu_grad(ws, nsteps, ckpt):
    ctx = pg.FdtdContext(ws[0]["dx"], ws[0]["dy"], ws[0]["dt"], [(w["eps_r"], w["sigma"]) for w in ws])
    models = []
    for s, w in enumerate(ws):
        for rd in w["roms"]:
            m = pg.rom_build(rd["a"], rd["b"], rd["r"], w["dx"], w["dy"], w["dt"], rd["eps_r"],
                             rd["sigma"], rd["q"], f0=rd["f0"])
            ctx.rom_embed(m, s, rd["i0"], rd["j0"])
            models.append(m)
    srcs, probes = [], []
    for s, w in enumerate(ws):
        for so in w["sources"]:
            srcs.append(dict(so, sim=s, wave=torch.tensor(so["wave"][:nsteps].astype(np.float32), device="cuda")))
        probes += [(s, i, j) for (i, j) in w["probes"]]
    J, ge, gs, gw = ctx.fdtd_grad(nsteps, srcs, probes, ckpt)
    torch.cuda.synchronize()
    return J, [g.cpu().numpy() for g in ge], [g.cpu().numpy() for g in gs], gw.cpu().numpy(), ctx


def test_gradients_match_oracle_adjoint():
    w = grad_case()
    J, ge, gs, gw, ctx = gpu_grad([w], 300, 64)      # 4 full segments + a remainder
    Jo, deps, dsig, gsrc = adjoint.gradients(w)
    assert abs(J - Jo) < 1e-4 * Jo
    assert rel_l2(ge[0], deps) < GTOL
    assert rel_l2(gs[0], dsig) < GTOL
    assert rel_l2(gw[0], gsrc[0]) < GTOL
    # cells beside the models (their material also enters the coupling)
    for rd in w["roms"]:
        for (i, j) in [(rd["i0"] - 1, rd["j0"] + 2), (rd["i0"] + rd["a"], rd["j0"] + 1)]:
            assert abs(ge[0][j, i] - deps[j, i]) < 1e-2 * np.abs(deps).max()
    assert ctx.step_count() == 300


def test_checkpoint_spacing_does_not_change_the_result():
    """The recomputed forward states are bit-identical whatever the segment
    length; only the grouping of the FP32 gradient sums (flushed to FP64 per
    segment) and the order of atomic additions change, at FP32 rounding."""
    w = grad_case(seed=61, nsteps=150)
    a = gpu_grad([w], 150, 7)
    b = gpu_grad([w], 150, 150)
    assert a[0] == b[0]
    assert rel_l2(a[1][0], b[1][0]) < 1e-5
    assert rel_l2(a[2][0], b[2][0]) < 1e-5
    assert rel_l2(a[3], b[3]) < 1e-5


def test_batch_gradients_are_per_simulation():
    ws = [grad_case(seed=62, nx=90, ny=70, nsteps=200), grad_case(seed=63, nx=70, ny=90, nsteps=200)]
    J, ge, gs, gw, _ = gpu_grad(ws, 200, 50)
    Jt = 0.0
    for s, w in enumerate(ws):
        Jo, deps, dsig, gsrc = adjoint.gradients(w, 200)
        Jt += Jo
        assert rel_l2(ge[s], deps) < GTOL
        assert rel_l2(gs[s], dsig) < GTOL
        assert rel_l2(gw[s], gsrc[0]) < GTOL
    assert abs(J - Jt) < 1e-4 * Jt


def _autograd_case(ws, nsteps, ckpt=40):
    """FdtdSpec and leaf tensors (eps, sigma, waves) of a batch of workloads
    with one grid size; models are built per simulation."""
    w0 = ws[0]
    roms = [[(pg.rom_build(rd["a"], rd["b"], rd["r"], w["dx"], w["dy"], w["dt"], rd["eps_r"], rd["sigma"],
                           rd["q"], f0=rd["f0"]), rd["i0"], rd["j0"]) for rd in w["roms"]] for w in ws]
    spec = FdtdSpec(w0["dx"], w0["dy"], w0["dt"], nsteps,
                    [[{k: v for k, v in so.items() if k != "wave"} for so in w["sources"]] for w in ws],
                    [list(w["probes"]) for w in ws], roms, ckpt_every=ckpt)
    eps = torch.tensor(np.stack([w["eps_r"] for w in ws]), requires_grad=True)
    sig = torch.tensor(np.stack([w["sigma"] for w in ws]), requires_grad=True)
    wav = torch.tensor(np.stack([np.stack([so["wave"][:nsteps] for so in w["sources"]]) for w in ws])
                       .astype(np.float32), requires_grad=True)
    return spec, eps, sig, wav


def test_autograd_probe_energy():
    """J = sum of probe Hz^2 through FdtdFn (forward: the probe series) and
    autograd (backward: fdtd_vjp seeded with dJ/dprobes = 2 o), against the
    FP64 oracle adjoint."""
    w = grad_case(seed=64, nx=60, ny=50, nsteps=120)
    spec, eps, sig, wav = _autograd_case([w], 120)
    J = probe_energy(eps, sig, wav, spec)
    (3.0 * J).backward()
    Jo, deps, dsig, gsrc = adjoint.gradients(w, 120)
    assert abs(float(J) - Jo) < 1e-4 * Jo
    assert rel_l2(eps.grad.numpy()[0] / 3.0, deps) < GTOL
    assert rel_l2(sig.grad.numpy()[0] / 3.0, dsig) < GTOL
    assert rel_l2(wav.grad.numpy()[0, 0] / 3.0, gsrc[0]) < GTOL


def test_autograd_linear_functional_of_probes():
    """L = sum c * probes with a random cotangent c: torch.autograd.grad
    through fdtd_vjp against the oracle adjoint seeded with the same c
    (pinned by central differences)."""
    N = 150
    w = grad_case(seed=66, nx=90, ny=70, nsteps=N)
    spec, eps, sig, wav = _autograd_case([w], N)
    c = np.random.default_rng(3).standard_normal((N, len(w["probes"])))
    probes = FdtdFn.apply(eps, sig, wav, spec)
    assert probes.shape == (1, N, len(w["probes"]))
    L = (torch.tensor(c[None], device="cuda") * probes.double()).sum()
    ge, gs, gw = torch.autograd.grad(L, (eps, sig, wav))
    Lo, deps, dsig, gsrc = adjoint.gradients(w, N, cotangent=c)
    scale = float((np.abs(c)[None] * probes.detach().cpu().double().abs().numpy()).sum())
    assert abs(float(L) - Lo) < 1e-4 * scale
    assert rel_l2(ge.numpy()[0], deps) < GTOL
    assert rel_l2(gs.numpy()[0], dsig) < GTOL
    assert rel_l2(gw.numpy()[0, 0], gsrc[0]) < GTOL


def test_autograd_forward_runs_no_reverse_sweep():
    """The forward pass alone is one fdtd_run: the same probe series bit for
    bit, and no reverse sweep until backward is called."""
    N = 80
    w = grad_case(seed=65, nx=60, ny=50, nsteps=N)
    spec, eps, sig, wav = _autograd_case([w], N)
    before = FdtdFn.vjp_calls
    probes = FdtdFn.apply(eps, sig, wav, spec)
    assert FdtdFn.vjp_calls == before
    ctx = pg.FdtdContext(w["dx"], w["dy"], w["dt"], [(w["eps_r"], w["sigma"])])
    for (m, i0, j0) in spec.roms[0]:
        ctx.rom_embed(m, 0, i0, j0)
    ref = torch.zeros((N, len(w["probes"])), dtype=torch.float32, device="cuda")
    ctx.fdtd_run(N, [dict(s, sim=0, wave=wav.detach()[0, k].cuda()) for k, s in enumerate(spec.sources[0])],
                 [(0, i, j) for (i, j) in w["probes"]], ref)
    assert torch.equal(probes[0], ref)
    (probes.double() ** 2).sum().backward()
    assert FdtdFn.vjp_calls == before + 1
    assert eps.grad is not None and float(eps.grad.abs().max()) > 0


def test_autograd_batch_is_per_simulation():
    """Two simulations of one grid size in one call (models, sources and
    probes per simulation): each simulation's gradient of the summed probe
    energy matches its own oracle adjoint."""
    N = 120
    ws = [grad_case(seed=67, nx=80, ny=64, nsteps=N), grad_case(seed=68, nx=80, ny=64, nsteps=N)]
    spec, eps, sig, wav = _autograd_case(ws, N)
    J = probe_energy(eps, sig, wav, spec)
    J.backward()
    Jt = 0.0
    for b, w in enumerate(ws):
        Jo, deps, dsig, gsrc = adjoint.gradients(w, N)
        Jt += Jo
        assert rel_l2(eps.grad.numpy()[b], deps) < GTOL
        assert rel_l2(sig.grad.numpy()[b], dsig) < GTOL
        assert rel_l2(wav.grad.numpy()[b, 0], gsrc[0]) < GTOL
    assert abs(float(J) - Jt) < 1e-4 * Jt


def test_vjp_with_twice_the_probes_equals_grad():
    """fdtd_vjp seeded with 2 o equals fdtd_grad (the probe energy)."""
    w = grad_case(seed=69, nx=70, ny=60, nsteps=100)
    J, ge, gs, gw, ctx = gpu_grad([w], 100, 30)
    ctx2 = pg.FdtdContext(w["dx"], w["dy"], w["dt"], [(w["eps_r"], w["sigma"])])
    for rd in w["roms"]:
        m = pg.rom_build(rd["a"], rd["b"], rd["r"], w["dx"], w["dy"], w["dt"], rd["eps_r"], rd["sigma"],
                         rd["q"], f0=rd["f0"])
        ctx2.rom_embed(m, 0, rd["i0"], rd["j0"])
    srcs = [dict(so, sim=0, wave=torch.tensor(so["wave"][:100].astype(np.float32), device="cuda"))
            for so in w["sources"]]
    probes = [(0, i, j) for (i, j) in w["probes"]]
    out = torch.zeros((100, len(probes)), dtype=torch.float32, device="cuda")
    ctx2.fdtd_run(100, srcs, probes, out)
    ctx3 = pg.FdtdContext(w["dx"], w["dy"], w["dt"], [(w["eps_r"], w["sigma"])])
    for rd in w["roms"]:
        m = pg.rom_build(rd["a"], rd["b"], rd["r"], w["dx"], w["dy"], w["dt"], rd["eps_r"], rd["sigma"],
                         rd["q"], f0=rd["f0"])
        ctx3.rom_embed(m, 0, rd["i0"], rd["j0"])
    fwd = torch.zeros_like(out)
    ve, vs, vw = ctx3.fdtd_vjp(100, srcs, probes, (2.0 * out).contiguous(), 30, probe_out=fwd)
    assert torch.equal(fwd, out)
    assert ctx3.step_count() == 100
    assert rel_l2(ve[0].cpu().numpy(), ge[0]) < 1e-6
    assert rel_l2(vs[0].cpu().numpy(), gs[0]) < 1e-6
    assert rel_l2(vw.cpu().numpy(), gw) < 1e-6


@pytest.mark.parametrize("nx,ny", [(100, 80), (300, 230)])
def test_fused_and_two_pass_reverse_steps_agree(monkeypatch, nx, ny):
    """The fused reverse cell pass and the two-pass form (adj_h + adj_e) are
    the same arithmetic up to FP32 contraction (300 x 230: several strips,
    tiles and halo columns)."""
    w = grad_case(seed=62, nx=nx, ny=ny, nsteps=120)
    res = {}
    for f in ("0", "1"):
        monkeypatch.setenv("FDTD_ADJ_FUSED", f)
        res[f] = gpu_grad([w], 120, 50)
    assert abs(res["0"][0] - res["1"][0]) <= 1e-12 * res["0"][0]
    for k in (1, 2):
        assert rel_l2(res["1"][k][0], res["0"][k][0]) < 1e-5
    assert rel_l2(res["1"][3], res["0"][3]) < 1e-5


def _off_ring_case(nx, ny, nsteps=120):
    """A gradient case whose probes sit off the cells beside the models
    (their probe and model additions would otherwise meet in atomics of
    either order, so two runs could differ in the last bit)."""
    w = workloads.random_grid(64, nx, ny, 2, 5, 2, 20, nsteps, n_probes=6)
    near = set()
    for rd in w["roms"]:
        for j in range(rd["j0"] - 1, rd["j0"] + rd["b"] + 1):
            for i in range(rd["i0"] - 1, rd["i0"] + rd["a"] + 1):
                near.add((i, j))
    si, sj = w["sources"][0]["i"], w["sources"][0]["j"]
    cand = w["probes"] + [(min(si + 4, nx - 1), sj), (si, min(sj + 5, ny - 1)), (max(si - 6, 0), sj)]
    w["probes"] = [p for p in cand if p not in near]
    assert len(w["probes"]) >= 3
    return w


@pytest.mark.parametrize("nx,ny,ckpt", [(100, 80, 7), (100, 80, 50), (300, 230, 25)])
def test_two_step_recomputation_is_bit_identical(monkeypatch, nx, ny, ckpt):
    """The recomputation in pairs of steps (the march and the zone chain also
    writing the E frame between the sub-steps; odd segments end with one
    single step) against one step per launch (FDTD_ADJ_RECOMP2=0): the same
    frames, so the same gradient bits (one reverse step per launch, whose
    additions are in a fixed order)."""
    monkeypatch.delenv("FDTD_TB", raising=False)
    monkeypatch.setenv("FDTD_ADJ_TB2", "0")
    w = _off_ring_case(nx, ny)
    res = {}
    for r in ("0", "1"):
        monkeypatch.setenv("FDTD_ADJ_RECOMP2", r)
        res[r] = gpu_grad([w], 120, ckpt)
        assert res[r][4].steps_per_launch() == 2
    assert np.abs(res["0"][1][0]).max() > 0
    assert res["1"][0] == res["0"][0]
    for k in (1, 2):
        np.testing.assert_array_equal(res["1"][k][0], res["0"][k][0])
    np.testing.assert_array_equal(res["1"][3], res["0"][3])


@pytest.mark.parametrize("nx,ny", [(100, 80), (300, 230)])
def test_staged_reverse_rows_are_bit_identical(monkeypatch, nx, ny):
    """The fused reverse cell pass with its row loads staged one or two rows
    ahead through shared memory (FDTD_ADJ_RING=2 / 3) against its register
    form: the same arithmetic, so the same bits (one reverse step per
    launch)."""
    monkeypatch.setenv("FDTD_ADJ_TB2", "0")
    w = _off_ring_case(nx, ny)
    res = {}
    for r in ("0", "2", "3"):
        monkeypatch.setenv("FDTD_ADJ_RING", r)
        res[r] = gpu_grad([w], 120, 50)
    assert np.abs(res["0"][1][0]).max() > 0
    for r in ("2", "3"):
        assert res[r][0] == res["0"][0]
        for k in (1, 2):
            np.testing.assert_array_equal(res[r][k][0], res["0"][k][0])
        np.testing.assert_array_equal(res[r][3], res["0"][3])


@pytest.mark.parametrize("nx,ny,ckpt", [(100, 80, 50), (100, 80, 7), (300, 230, 25), (700, 300, 40)])
def test_two_step_reverse_agrees_with_one_step(monkeypatch, nx, ny, ckpt):
    """Two reverse steps per launch (the additions before the second step,
    from the models' transposed maps and the probe seeds, made afterwards as
    local corrections) against one reverse step per launch: the same
    gradients up to FP32 rounding at the corrected cells (several strips,
    tiles and halo columns; odd segments end with one single step; probes on
    the cells beside the models and by the source)."""
    w = grad_case(seed=65, nx=nx, ny=ny, nsteps=120)
    res = {}
    for r in ("0", "1"):
        monkeypatch.setenv("FDTD_ADJ_TB2", r)
        res[r] = gpu_grad([w], 120, ckpt)
    assert np.abs(res["0"][1][0]).max() > 0
    assert res["1"][0] == res["0"][0]
    for k in (1, 2):
        assert rel_l2(res["1"][k][0], res["0"][k][0]) < 1e-5
    assert rel_l2(res["1"][3], res["0"][3]) < 1e-5


def test_multi_strip_gradients_match_oracle():
    """Several 128-column strips and tiles (halo rows and columns of the
    fused reverse pass) against the FP64 adjoint."""
    w = grad_case(seed=63, nx=300, ny=230, nsteps=150)
    J, ge, gs, gw, _ = gpu_grad([w], 150, 40)
    Jo, deps, dsig, gsrc = adjoint.gradients(w, nsteps=150)
    assert abs(J - Jo) < 1e-4 * Jo
    assert rel_l2(ge[0], deps) < GTOL
    assert rel_l2(gs[0], dsig) < GTOL
    assert rel_l2(gw[0], gsrc[0]) < GTOL


def test_full_size_gradients_against_finite_differences(monkeypatch):
    """The gradient configuration at full size (16 x 1024^2, two shared
    q = 120 models per simulation, 8 probes each, J = sum Hz^2 over 10^4
    steps, checkpoints every 500) in the library's default launch
    configuration.  fdtd_grad against finite differences through the GPU
    forward (an FP64 forward of this size exists only in the oracle, hours
    per run), J split per simulation by its own probes so that every pair of
    runs checks one cell in each of the 16 simulations:
      - eps_r at 32 seeded random coarse cells and at 16 cells beside a model
        (their material also enters the coupling of Eq. (19)): central
        differences, h = 10% of eps_r;
      - sigma at the same cells: one-sided second-order differences
        (-3 J(s) + 4 J(s + h) - J(s + 2h)) / 2h, h = 0.04 S/m;
      - the sources: J is quadratic in them, so J = 1/2 s . dJ/ds (Euler).
    Tolerance |D - g| <= t_rel |g| + t_abs max|g| (per simulation and
    parameter): the FP32 forward leaves a noise floor in the difference
    quotients of at most 5e-6 (eps) and 3.1e-5 (sigma) of the simulation's
    largest gradient (measured on GB300 at these step sizes), taken with a
    margin of 4 and 3; t_rel = 2% (eps) and 5% (sigma) covers the truncation
    error (0.6% and 4.7% at most where the noise is small).  At least 24 of
    the 32 random cells must agree to 1% (eps) and 20 to 5% (sigma), so
    that the floor does not carry the test."""
    monkeypatch.delenv("FDTD_TB", raising=False)
    N = 10000
    w = workloads.adjoint_16(N)
    S = len(w["sims"])
    models = [pg.rom_build(md["a"], md["b"], md["r"], w["dx"], w["dy"], w["dt"], md["eps_r"],
                           md["sigma"], md["q"], f0=md["f0"]) for md in w["models"]]

    def ctx_for(eps, sig):
        ctx = pg.FdtdContext(w["dx"], w["dy"], w["dt"], [(e, x) for e, x in zip(eps, sig)])
        for k, s in enumerate(w["sims"]):
            for (mi, i0, j0) in s["place"]:
                ctx.rom_embed(models[mi], k, i0, j0)
        return ctx

    waves = [torch.tensor(np.asarray(s["source"]["wave"], np.float32), device="cuda") for s in w["sims"]]
    src = [dict(s["source"], sim=k, wave=waves[k]) for k, s in enumerate(w["sims"])]
    probes = [(k, i, j) for k, s in enumerate(w["sims"]) for (i, j) in s["probes"]]
    eps0 = [s["eps_r"] for s in w["sims"]]
    sig0 = [s["sigma"] for s in w["sims"]]
    J, ge, gs, gw = ctx_for(eps0, sig0).fdtd_grad(N, src, probes, 500)
    ge = [g.cpu().numpy() for g in ge]
    gs = [g.cpu().numpy() for g in gs]
    gw = gw.cpu().numpy()
    euler = 0.5 * sum(float(np.dot(np.asarray(s["source"]["wave"][:N], np.float64), gw[k]))
                      for k, s in enumerate(w["sims"]))
    assert abs(euler - J) < 1e-3 * J

    def J_sims(eps, sig):
        ctx = ctx_for(eps, sig)
        out = torch.zeros((N, len(probes)), dtype=torch.float32, device="cuda")
        ctx.fdtd_run(N, src, probes, out)
        o = out.double().cpu().numpy()
        ctx.close()
        return np.array([(o[:, 8 * k:8 * k + 8] ** 2).sum() for k in range(S)])

    def perturbed(cells, eps_d, sig_d):
        eps = [e.copy() for e in eps0]
        sig = [x.copy() for x in sig0]
        for k, (i, j) in enumerate(cells):
            eps[k][j, i] += eps_d[k]
            sig[k][j, i] += sig_d[k]
        return J_sims(eps, sig)

    rng = np.random.default_rng(1609071145)

    def random_cell(k):
        s = w["sims"][k]
        near = np.zeros((s["ny"], s["nx"]), bool)
        for (mi, i0, j0) in s["place"]:
            near[j0 - 2:j0 + 18, i0 - 2:i0 + 18] = True
        while True:
            i, j = int(rng.integers(2, s["nx"] - 2)), int(rng.integers(2, s["ny"] - 2))
            if not near[j, i]:
                return i, j

    rounds = {"random0": [random_cell(k) for k in range(S)], "random1": [random_cell(k) for k in range(S)],
              "ring": [(s["place"][k % 2][1] - 1, s["place"][k % 2][2] + 3 + k % 7) for k, s in enumerate(w["sims"])]}
    J0 = J_sims(eps0, sig0)
    hs = 0.04
    zero = [0.0] * S
    good_e = good_s = 0
    for name, cells in rounds.items():
        he = [0.1 * eps0[k][j, i] for k, (i, j) in enumerate(cells)]
        De = (perturbed(cells, he, zero) - perturbed(cells, [-h for h in he], zero)) / (2 * np.array(he))
        Ds = (-3 * J0 + 4 * perturbed(cells, zero, [hs] * S) - perturbed(cells, zero, [2 * hs] * S)) / (2 * hs)
        for k, (i, j) in enumerate(cells):
            g_e, g_s = ge[k][j, i], gs[k][j, i]
            assert abs(De[k] - g_e) <= 0.02 * abs(g_e) + 2e-5 * np.abs(ge[k]).max(), (name, k, De[k], g_e)
            assert abs(Ds[k] - g_s) <= 0.05 * abs(g_s) + 1e-4 * np.abs(gs[k]).max(), (name, k, Ds[k], g_s)
            if name != "ring":
                good_e += abs(De[k] - g_e) <= 0.01 * abs(g_e)
                good_s += abs(Ds[k] - g_s) <= 0.05 * abs(g_s)
    assert good_e >= 24 and good_s >= 20, (good_e, good_s)


def _adjoint16_case(wb, k, N):
    """Workload record of simulation k of the gradient configuration (for the
    oracle)."""
    s = wb["sims"][k]
    return dict(nx=s["nx"], ny=s["ny"], dx=wb["dx"], dy=wb["dy"], dt=wb["dt"], eps_r=s["eps_r"],
                sigma=s["sigma"], roms=[dict(wb["models"][mi], i0=i0, j0=j0) for (mi, i0, j0) in s["place"]],
                sources=[s["source"]], probes=list(s["probes"]), nsteps=N)


def test_scaled_gradient_configuration_matches_oracle_fields(monkeypatch):
    """The gradient configuration's recipe (two shared q = 120 models per
    simulation, vacuum rings, 8 probes, J = sum Hz^2, checkpoints every 500
    steps) on a scaled copy, 2 x 192^2 over 1500 steps, in the library's
    default launch configuration: the whole dJ/deps, dJ/dsigma fields and the
    source gradients against the FP64 oracle adjoint."""
    monkeypatch.delenv("FDTD_TB", raising=False)
    N = 1500
    wb = workloads.adjoint_16(N, nsim=2, n=192)
    ws = [_adjoint16_case(wb, k, N) for k in range(2)]
    J, ge, gs, gw, _ = gpu_grad(ws, N, 500)
    Jt = 0.0
    for k, w in enumerate(ws):
        Jo, deps, dsig, gsrc = adjoint.gradients(w, N)
        Jt += Jo
        assert np.abs(deps).max() > 0
        assert rel_l2(ge[k], deps) < GTOL
        assert rel_l2(gs[k], dsig) < GTOL
        assert rel_l2(gw[k], gsrc[0]) < GTOL
    assert abs(J - Jt) < 1e-4 * Jt
