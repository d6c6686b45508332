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
from paper_1609_07114_gb300.autograd import ProbeEnergy, ProbeEnergySpec
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


def test_autograd_function():
    w = grad_case(seed=64, nx=60, ny=50, nsteps=120)
    models = [(pg.rom_build(rd["a"], rd["b"], rd["r"], w["dx"], w["dy"], w["dt"], rd["eps_r"], rd["sigma"],
                            rd["q"], f0=rd["f0"]), rd["i0"], rd["j0"]) for rd in w["roms"]]
    spec = ProbeEnergySpec(w["dx"], w["dy"], w["dt"], 120,
                           [{k: v for k, v in s.items() if k != "wave"} for s in w["sources"]],
                           w["probes"], models, ckpt_every=40)
    eps = torch.tensor(w["eps_r"], requires_grad=True)
    sig = torch.tensor(w["sigma"], requires_grad=True)
    wav = torch.tensor(np.stack([s["wave"][:120] for s in w["sources"]]).astype(np.float32), requires_grad=True)
    J = ProbeEnergy.apply(eps, sig, wav, spec)
    (3.0 * J).backward()
    Jo, deps, dsig, gsrc = adjoint.gradients(w, 120)
    assert abs(float(J) - Jo) < 1e-4 * Jo
    assert rel_l2(eps.grad.numpy() / 3.0, deps) < GTOL
    assert rel_l2(sig.grad.numpy() / 3.0, dsig) < GTOL
    assert rel_l2(wav.grad.numpy()[0] / 3.0, gsrc[0]) < GTOL


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


def test_full_size_gradient_properties(monkeypatch):
    """The gradient configuration at full batch size (16 x 1024^2, two shared
    models each), in the benchmark's launch configuration (the library's
    default choice of one or two steps per launch for the forward and
    checkpoint passes), over 3000 steps with checkpoints every 500: J is
    quadratic in the sources, so J = 1/2 sum s . dJ/ds (Euler); and the eps
    gradient at the cell with the largest sensitivity matches a central
    difference of two forward runs."""
    monkeypatch.delenv("FDTD_TB", raising=False)
    N = 3000
    w = workloads.adjoint_16(N)
    models = [pg.rom_build(md["a"], md["b"], md["r"], w["dx"], w["dy"], w["dt"], md["eps_r"],
                           md["sigma"], md["q"], f0=md["f0"]) for md in w["models"]]

    def ctx_for(eps_list):
        ctx = pg.FdtdContext(w["dx"], w["dy"], w["dt"], [(e, s["sigma"]) for e, s in zip(eps_list, w["sims"])])
        for k, s in enumerate(w["sims"]):
            for (mi, i0, j0) in s["place"]:
                ctx.rom_embed(models[mi], k, i0, j0)
        return ctx

    waves = [torch.tensor(np.asarray(s["source"]["wave"], np.float32), device="cuda") for s in w["sims"]]
    src = [dict(s["source"], sim=k, wave=waves[k]) for k, s in enumerate(w["sims"])]
    probes = [(k, i, j) for k, s in enumerate(w["sims"]) for (i, j) in s["probes"]]
    eps0 = [s["eps_r"] for s in w["sims"]]
    J, ge, gs, gw = ctx_for(eps0).fdtd_grad(N, src, probes, 500)
    assert J > 0
    gw = gw.cpu().numpy()
    euler = 0.5 * sum(float(np.dot(np.asarray(s["source"]["wave"][:N], np.float64), gw[k]))
                      for k, s in enumerate(w["sims"]))
    assert abs(euler - J) < 1e-3 * J
    gmax = [float(g.abs().max()) for g in ge]
    k = int(np.argmax(gmax))
    gk = ge[k].cpu().numpy()
    j, i = np.unravel_index(np.argmax(np.abs(gk)), gk.shape)
    h = 1e-3 * eps0[k][j, i]

    def J_at(delta):
        eps = [e.copy() for e in eps0]
        eps[k][j, i] += delta
        ctx = ctx_for(eps)
        out = torch.zeros((N, len(probes)), dtype=torch.float32, device="cuda")
        ctx.fdtd_run(N, src, probes, out)
        return float((out.double() ** 2).sum())

    fd = (J_at(h) - J_at(-h)) / (2 * h)
    assert abs(fd - gk[j, i]) < 2e-2 * abs(gk[j, i])
