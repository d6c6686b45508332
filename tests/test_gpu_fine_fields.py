"""Fine-region fields rebuilt from the model state on the device
(fdtd_fine_fields) against the oracle's V x~ after the same steps."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1609_07114_gb300 as pg
import workloads
import test_gpu_parity as tp
from oracle import problem, scheme

pytestmark = pytest.mark.gpu


def compare(ctx, models, w, nsteps, insts, order=None):
    _, _, grid, emb, _ = problem.run(w, nsteps, order=order)
    for k in insts:
        rd = w["roms"][k]
        ref = scheme.fine_fields(emb[k], rd["r"] * rd["a"], rd["r"] * rd["b"])
        got = ctx.fine_fields(k, models[k])
        torch.cuda.synchronize()
        for g, o in zip(got, ref):
            assert g.shape == o.shape
            assert tp.rel_l2(g.cpu().numpy(), o) < tp.TOL


def test_cavity_fine_fields():
    w = workloads.cavity_60(500)
    ctx, models = tp.gpu_context([w])
    tp.gpu_run(ctx, [w], 500)
    compare(ctx, models, w, 500, [0])


def test_fine_fields_with_cfl_extension():
    """dt = 1.9 x the fine CFL limit: the clamped (full-order) models'
    rebuilt fields."""
    w = workloads.random_grid(21, 120, 90, 2, 4, 2, 0, 300, dt_factor=1.9, n_probes=6)
    ctx, models = tp.gpu_context([w], order=0)
    assert all(m.report.n_clamped > 0 for m in models)
    tp.gpu_run(ctx, [w], 300)
    compare(ctx, models, w, 300, [0, 1], order=0)


def test_fine_fields_wrong_model_is_rejected():
    w = workloads.cavity_60(10)
    ctx, models = tp.gpu_context([w])
    rd = w["roms"][0]
    other = pg.rom_build(rd["a"], rd["b"], rd["r"], w["dx"], w["dy"], w["dt"], rd["eps_r"],
                         rd["sigma"], rd["q"], f0=rd["f0"])
    with pytest.raises(pg.FdtdError):
        ctx.fine_fields(0, other)
