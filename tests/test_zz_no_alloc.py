"""fdtd_energy_noalloc: the storage function without any device allocation.

Some callers must not allocate GPU memory at the moment they ask for the
energy (another framework's caching allocator holds the free memory, a
time-critical loop cannot afford cudaMalloc's implicit synchronisation, or
the work is about to be recorded into a CUDA graph).  This entry point keeps
its partial sums in a fixed array inside the library instead.  The test calls
it twice in a row through the C ABI and checks each result against
fdtd_energy (which uses a context-owned buffer), in a fresh process or after
the other tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1609_07114_gb300 as pg
import workloads

pytestmark = pytest.mark.gpu


def test_noalloc_energy_matches_fdtd_energy_twice():
    ws = [workloads.random_grid(40 + k, nx, ny, 2, 6, 3, 40, 200, n_probes=1)
          for k, (nx, ny) in enumerate([(300, 120), (150, 260)])]
    ctx = pg.FdtdContext(ws[0]["dx"], ws[0]["dy"], ws[0]["dt"], [(w["eps_r"], w["sigma"]) for w in ws])
    models = []
    for s, w in enumerate(ws):
        for rd in w["roms"]:
            m = pg.rom_build(rd["a"], rd["b"], rd["r"], w["dx"], w["dy"], w["dt"], rd["eps_r"],
                             rd["sigma"], rd["q"], f0=rd["f0"])
            ctx.rom_embed(m, s, rd["i0"], rd["j0"])
            models.append(m)
    srcs = [dict(w["sources"][0], sim=s,
                 wave=torch.tensor(w["sources"][0]["wave"].astype(np.float32), device="cuda"))
            for s, w in enumerate(ws)]
    for n in (120, 80):
        ctx.fdtd_run(n, [dict(sr, wave=sr["wave"][:n]) for sr in srcs], [], None)
        ref = ctx.energy()
        got = ctx.energy_noalloc()
        assert np.all(ref > 0)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)


def test_noalloc_energy_rejects_contexts_beyond_its_capacity():
    """A context with more stencil tiles + models + simulations than the
    fixed array holds gets FDTD_EINVAL from the no-allocation entry point
    (and nothing is written); fdtd_energy still serves it."""
    n = pg.FDTD_ENERGY_STATIC_MAX // 2 + 16     # 2 x 2 simulations: one tile each
    rng = np.random.default_rng(7)
    sims = [(1.0 + rng.random((2, 2)), np.zeros((2, 2))) for _ in range(n)]
    dx = 1e-3
    ctx = pg.FdtdContext(dx, dx, 0.5 * pg.fdtd_cfl_limit(dx, dx), sims)
    out = np.full(n, -7.0)
    rc = pg.lib().fdtd_energy_noalloc(ctx._h, out.ctypes.data_as(pg._dp))
    assert rc == -1                              # FDTD_EINVAL
    assert b"static capacity" in pg.lib().fdtd_last_error(ctx._h)
    assert np.all(out == -7.0)
    assert np.all(ctx.energy() == 0.0)
