"""Reduced models built on the device (rom_build_gpu) against the host build
and the FP64 oracle: same reduced space (principal angles), same coupled
map (Markov parameters), passivity, and a time march with the device-built
model against the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1609_07114_gb300 as pg
import workloads
import test_gpu_parity as tp
from oracle import problem, yee

pytestmark = pytest.mark.gpu


def markov(P, Q, ny, K=12):
    out, Pk = [], np.eye(P.shape[0])
    for _ in range(K):
        out.append((Pk @ Q)[:ny])
        Pk = P @ Pk
    return out


def both(w, rd):
    args = (rd["a"], rd["b"], rd["r"], w["dx"], w["dy"], w["dt"], rd["eps_r"], rd["sigma"], rd["q"])
    return pg.rom_build(*args, f0=rd["f0"]), pg.rom_build_gpu(*args, f0=rd["f0"])


def cases():
    lat = workloads.lattice_8192(10, n=768, pitch=256)
    big = next(rd for rd in lat["roms"] if rd["q"] == 400)
    g4 = workloads.grid_4096(10)
    return [(workloads.cavity_60(10), workloads.cavity_60(10)["roms"][0]),
            (g4, g4["roms"][0]),
            (lat, big)]


@pytest.mark.parametrize("k", [0, 1, 2])
def test_device_build_matches_host_build(k):
    w, rd = cases()[k]
    mh, mg = both(w, rd)
    assert (mg.qE, mg.qH) == (mh.qE, mh.qH)
    for Vg, Vh in zip(mg.basis(), mh.basis()):
        assert np.abs(Vg.T @ Vg - np.eye(Vg.shape[1])).max() < 1e-9
        cos = np.linalg.svd(Vg.T @ Vh, compute_uv=False)
        assert cos.min() > 1 - 1e-6
    assert mg.report.n_clamped == mh.report.n_clamped
    assert mg.report.min_eig_R > 0 and mg.report.cond3_residual < 1e-12
    grid = problem.make_grid(dict(w, roms=[dict(rd, i0=rd["i0"], j0=rd["j0"])]))
    itf = grid.interfaces[0]
    Ph, Qh = mh.couple(itf.eps_b / yee.EPS0, itf.sig_b)
    Pg, Qg = mg.couple(itf.eps_b / yee.EPS0, itf.sig_b)
    for a, b in zip(markov(Ph, Qh, itf.ny_), markov(Pg, Qg, itf.ny_)):
        assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(a)
    print(f"build seconds host {mh.report.seconds:.3f} device {mg.report.seconds:.3f} (q={rd['q']})")


def test_time_march_with_device_built_model():
    w = workloads.cavity_60(2000)
    rd = w["roms"][0]
    ctx = pg.FdtdContext(w["dx"], w["dy"], w["dt"], [(w["eps_r"], w["sigma"])])
    m = pg.rom_build_gpu(rd["a"], rd["b"], rd["r"], w["dx"], w["dy"], w["dt"], rd["eps_r"], rd["sigma"],
                         rd["q"], f0=rd["f0"])
    ctx.rom_embed(m, 0, rd["i0"], rd["j0"])
    g = tp.gpu_run(ctx, [w], 2000)
    o, st = tp.oracle_run(w, 2000)
    assert tp.rel_l2(g, o) < tp.TOL
