"""Convolutional PML layers on the device against the FP64 oracle's CPML,
their absorption, and the checks around them."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1609_07114_gb300 as pg
import workloads
import test_gpu_parity as tp
import test_oracle_cpml as oc

pytestmark = pytest.mark.gpu


def pml_workload(prof, n=8, nsteps=600):
    """Lossy 200 x 160 grid, two r = 2 models, a source 12 cells from the
    west layer, probes in, at and beside the layers."""
    w = workloads.random_grid(44, 200, 160, 2, 6, 2, 24, nsteps, n_probes=0, margin=n + 4)
    occ = np.zeros((w["ny"], w["nx"]), bool)
    for rd in w["roms"]:
        occ[rd["j0"] - 3:rd["j0"] + rd["b"] + 3, rd["i0"] - 3:rd["i0"] + rd["a"] + 3] = True
    i = n + 12
    j = next(j for j in range(70, 160) if not occ[j - 3:j + 4, i - 3:i + 4].any())
    w["sources"][0].update(i=i, j=j)
    w["probes"] = [(2, j), (n, j + 5), (n + 1, j - 20), (i + 7, j), (i, min(j + 30, 150)), (100, 3),
                   (190, 150)]
    w["pml"] = dict(n=n, sides=15, **prof)
    return w


def gpu_pml_context(w):
    ctx, models = tp.gpu_context([w])
    p = w["pml"]
    ctx.set_pml(0, p["sides"], p["n"], p.get("m", 3.0), p.get("sigma_max") or 0.0,
                p.get("kappa_max", 1.0), p.get("alpha_max", 0.0))
    return ctx, models


@pytest.mark.parametrize("prof", [dict(), dict(kappa_max=4.0, alpha_max=0.03, m=4.0)])
def test_pml_matches_oracle(prof):
    w = pml_workload(prof)
    ctx, _ = gpu_pml_context(w)
    g = tp.gpu_run(ctx, [w], 600)
    o, st = tp.oracle_run(w, 600)
    assert tp.rel_l2(g, o) < tp.TOL
    tp.check_fields(ctx, 0, st)


def test_pml_absorbs_on_device():
    """The oracle pin's pulse, on the device: 80^2 with 10-cell layers vs the
    400^2 PEC grid (also on the device)."""
    res = []
    for n, pml in ((400, None), (80, dict(n=10, sides=15))):
        w = oc.pulse_problem(n, pml)
        ctx = pg.FdtdContext(w["dx"], w["dy"], w["dt"], [(w["eps_r"], w["sigma"])])
        if pml:
            ctx.set_pml(0, 15, 10)
        res.append(tp.gpu_run(ctx, [w], oc.STEPS))
    assert oc.err(res[1], res[0]) < 1e-3


def test_pml_save_load_is_bit_identical():
    w = pml_workload(dict(), nsteps=300)
    full, _ = gpu_pml_context(w)
    g_full = tp.gpu_run(full, [w], 300)
    a, _ = gpu_pml_context(w)
    w1 = dict(w, sources=[dict(s, wave=s["wave"][:120]) for s in w["sources"]])
    g1 = tp.gpu_run(a, [w1], 120)
    blob = a.save_state()
    b, _ = gpu_pml_context(w)
    b.load_state(blob)
    w2 = dict(w, sources=[dict(s, wave=s["wave"][120:]) for s in w["sources"]])
    g2 = tp.gpu_run(b, [w2], 180)
    np.testing.assert_array_equal(np.concatenate([g1, g2]), g_full)


def test_pml_placement_checks():
    w = pml_workload(dict())
    ctx, models = gpu_pml_context(w)
    rd = w["roms"][0]
    with pytest.raises(pg.FdtdError):      # a model inside the layer's reach
        ctx.rom_embed(models[0], 0, 9, 9)
    bad = dict(w["sources"][0], i=5, j=80, wave=torch.zeros(10, device="cuda"))
    with pytest.raises(pg.FdtdError):      # a source on a layer edge
        ctx.fdtd_run(10, [dict(bad, sim=0)])
    c2, _ = tp.gpu_context([w])
    with pytest.raises(pg.FdtdError):      # layers reaching an embedded region
        c2.set_pml(0, 15, rd["i0"] - 1)
    with pytest.raises(pg.FdtdError):
        ctx.fdtd_grad(10, [], [(0, 50, 50)])
