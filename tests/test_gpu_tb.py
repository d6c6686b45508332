"""The two-steps-per-pass path (FDTD_TB=1; chosen by default where the
model tiles take a small share of a wave) in both forms (the
row-marching kernel with model tiles, and FDTD_TB_SMEM=1 shared-memory
tiles): the parity cases of the one-step path rerun through it against the
FP64 oracle, and the paths against each other on the same inputs (the
row-marching form bit for bit: it uses the one-step kernel's operations).
The models' maps are stepped either inside their zone tiles (fused) or by the
zone chain (tile halves around a map launch: the default for maps shared by a
GEMM group, FDTD_TB_CHAIN=1 for every model); the map itself one row per warp
or as a GEMM over the simulations sharing it.  Every choice gives the same
bits."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1609_07114_gb300 as pg
import workloads
import test_gpu_parity as tp

pytestmark = pytest.mark.gpu


@pytest.fixture(params=["march", "smem"])
def tb_on(monkeypatch, request):
    monkeypatch.setenv("FDTD_TB", "1")
    monkeypatch.setenv("FDTD_TB_SMEM", "1" if request.param == "smem" else "0")


@pytest.mark.parametrize("case", [
    "test_cavity_60_full_length",
    "test_multi_tile_ragged_lossy_grid",
    "test_batch_of_uneven_grids",
    "test_cfl_extension_run",
    "test_split_runs_equal_one_run",
    "test_save_load_resume_is_bit_identical",
    "test_full_size_grid_sampled_outputs",
])
def test_parity_case_through_two_step_path(tb_on, case):
    getattr(tp, case)()


def test_full_batched_256_through_row_marching_form(monkeypatch):
    """The 256-simulation batch in the benchmark's launch configuration
    (two steps per launch, chosen automatically there), against the oracle."""
    monkeypatch.setenv("FDTD_TB", "1")
    monkeypatch.setenv("FDTD_TB_SMEM", "0")
    tp.test_full_batched_256_sampled_simulations()


def test_two_step_path_agrees_with_one_step_path(monkeypatch):
    monkeypatch.setenv("FDTD_TB_SMEM", "1")
    w = workloads.random_grid(7, 700, 150, 3, 6, 3, 40, 301, n_probes=12)
    for rd in w["roms"]:
        w["probes"] += [(rd["i0"] - 1, rd["j0"]), (rd["i0"] + rd["a"], rd["j0"] + rd["b"] - 1)]
    res = {}
    for tb in ("0", "1"):
        monkeypatch.setenv("FDTD_TB", tb)
        ctx, _ = tp.gpu_context([w])
        res[tb] = (tp.gpu_run(ctx, [w], 301), ctx.get_fields(0))   # odd count: a trailing single step
    assert tp.rel_l2(res["1"][0], res["0"][0]) < 1e-6
    for a, b in zip(res["1"][1], res["0"][1]):
        assert tp.rel_l2(a, b) < 1e-6


def _covered(w, i, j, pad=1):
    return any(rd["i0"] - pad <= i < rd["i0"] + rd["a"] + pad and rd["j0"] - pad <= j < rd["j0"] + rd["b"] + pad
               for rd in w["roms"])


def _boundary_workloads(nsteps):
    """Two grids (same r, so the same dt) with probes on both sides of the
    120-column strip and 480-column tile boundaries, a Jy line source along a
    strip boundary and an Ex point source, models placed at random (their
    zones straddle strips and tiles; 12 cells apart, so that no model is
    within reach of another's tile and the two-step path is taken)."""
    ws = [workloads.random_grid(21, 1000, 300, 5, 6, 3, 40, nsteps, n_probes=6, margin=12),
          workloads.random_grid(22, 250, 470, 3, 5, 3, 30, nsteps, n_probes=6, margin=12)]
    g = np.random.default_rng(5)
    for w in ws:
        for c0 in range(120, w["nx"] - 1, 120):
            for i in (c0 - 2, c0 - 1, c0, c0 + 1):
                j = int(g.integers(1, w["ny"] - 1))
                if 0 <= i < w["nx"] and not _covered(w, i, j):
                    w["probes"].append((i, j))
        wave = w["sources"][0]["wave"]
        for x in (480, 479, 240, 241, 120):
            if x < w["nx"] and not any(_covered(w, x, j) or _covered(w, x - 1, j) for j in range(w["ny"])):
                w["sources"].append(dict(comp=1, i=x, j=0, len=w["ny"], wave=0.5 * wave))
                break
        for (i, j) in ((361, 17), (100, 34), (479, 51)):
            if i < w["nx"] and j < w["ny"] and not (_covered(w, i, j) or _covered(w, i, j - 1)):
                w["sources"].append(dict(comp=0, i=i, j=j, len=1, wave=-0.25 * wave))
    return ws


@pytest.mark.parametrize("rows", ["17", "auto"])
def test_row_marching_form_is_bit_identical_to_one_step(monkeypatch, rows):
    """Probe series and final fields of the row-marching two-step form equal
    the one-step path bit for bit over an odd step count (a trailing single
    step), for many row tiles (17 rows) and the automatic plan."""
    n = 203
    ws = _boundary_workloads(n)
    res = {}
    for tb in ("0", "1"):
        monkeypatch.setenv("FDTD_TB", tb)
        monkeypatch.setenv("FDTD_TB_SMEM", "0")
        if rows == "auto":
            monkeypatch.delenv("FDTD_TB_ROWS", raising=False)
        else:
            monkeypatch.setenv("FDTD_TB_ROWS", rows)
        ctx, _ = tp.gpu_context(ws)
        out = tp.gpu_run(ctx, ws, n)
        res[tb] = (out, [ctx.get_fields(s) for s in range(len(ws))])
    assert np.abs(res["0"][0]).max() > 0
    assert np.array_equal(res["1"][0], res["0"][0])
    for fa, fb in zip(res["1"][1], res["0"][1]):
        for a, b in zip(fa, fb):
            assert np.array_equal(a, b)


def test_default_choice_of_the_two_step_path(monkeypatch):
    """Unset FDTD_TB: with every model in the zone chain (the default) the
    two-step path is taken at every size (the 4096^2 benchmark grid, a 128^2
    grid with one q = 400 model, the 64-model lattice at 2048^2); with the
    maps fused into their zone tiles (FDTD_TB_CHAIN=0) the small grid, where
    one CTA stepping the model twice outlasts two one-step launches, steps
    singly and the benchmark grid still in pairs; FDTD_TB=0 / 1 force the
    choice."""
    import test_gpu_lattice as tl
    monkeypatch.delenv("FDTD_TB", raising=False)
    monkeypatch.delenv("FDTD_TB_CHAIN", raising=False)
    w = workloads.grid_4096(10)
    ctx, _ = tp.gpu_context([w])
    assert ctx.steps_per_launch() == 2
    ctx.close()
    ws = workloads.random_grid(1, 128, 128, 1, 16, 4, 400, 10)
    assert tp.gpu_context([ws])[0].steps_per_launch() == 2
    wl = workloads.lattice_8192(10, n=2048, pitch=256)
    ctxl, _ = tl.lattice_context(wl)
    assert len(wl["roms"]) == 64 and ctxl.steps_per_launch() == 2
    ctxl.close()
    monkeypatch.setenv("FDTD_TB_CHAIN", "0")
    assert tp.gpu_context([ws])[0].steps_per_launch() == 1
    ctx, _ = tp.gpu_context([w])
    assert ctx.steps_per_launch() == 2
    ctx.close()
    monkeypatch.delenv("FDTD_TB_CHAIN", raising=False)
    monkeypatch.setenv("FDTD_TB", "0")
    assert tp.gpu_context([w])[0].steps_per_launch() == 1
    monkeypatch.setenv("FDTD_TB", "1")
    monkeypatch.setenv("FDTD_TB_CHAIN", "0")
    assert tp.gpu_context([ws])[0].steps_per_launch() == 2


_BATCHED_MODELS = {}


def batched_context(ws):
    """Context of _batched_small workloads: the four shared models are built
    once per process and embedded in every simulation."""
    w0 = ws[0]
    if not _BATCHED_MODELS:
        for k, md in enumerate(w0["models"]):
            _BATCHED_MODELS[k] = pg.rom_build(md["a"], md["b"], md["r"], w0["dx"], w0["dy"], w0["dt"], md["eps_r"],
                                              md["sigma"], md["q"], f0=md["f0"])
    ctx = pg.FdtdContext(w0["dx"], w0["dy"], w0["dt"], [(w["eps_r"], w["sigma"]) for w in ws])
    for s, w in enumerate(ws):
        for (k, i0, j0) in w["place"]:
            ctx.rom_embed(_BATCHED_MODELS[k], s, i0, j0)
    return ctx, list(_BATCHED_MODELS.values())


def _batched_small(N, per_size=40):
    """40 grids of 128^2 sharing the four batched-layout models (vacuum
    rings): two GEMM column blocks per map (32 + 8 columns)."""
    wb = workloads.batched_256(N, per_size=per_size, sizes=(128,))
    ws = []
    for s in wb["sims"]:
        probes = [s["probe"]] + [(i0 - 1, j0 + 2) for (_, i0, j0) in s["place"]]   # some inside zones
        ws.append(dict(nx=s["nx"], ny=s["ny"], dx=wb["dx"], dy=wb["dy"], dt=wb["dt"], eps_r=s["eps_r"],
                       sigma=s["sigma"], roms=[dict(wb["models"][k], i0=i0, j0=j0) for (k, i0, j0) in s["place"]],
                       sources=[s["source"]], probes=probes, nsteps=N, place=s["place"], models=wb["models"],
                       make=batched_context))
    return ws


def context_for(ws):
    """The workloads' own context builder (shared models) or one model per
    region."""
    return ws[0]["make"](ws) if "make" in ws[0] else tp.gpu_context(ws)


def _run_forms(monkeypatch, ws, n, settings):
    res = {}
    for name, env in settings.items():
        for k, v in env.items():
            monkeypatch.setenv(k, v)
        ctx, _ = context_for(ws)
        out = tp.gpu_run(ctx, ws, n)
        res[name] = (out, [ctx.get_fields(s) for s in range(len(ws))], ctx.steps_per_launch())
        ctx.close()
    return res


def _assert_same_bits(res, ref):
    assert np.abs(res[ref][0]).max() > 0
    for name, (out, fields, _) in res.items():
        assert np.array_equal(out, res[ref][0]), name
        for fa, fb in zip(fields, res[ref][1]):
            for a, b in zip(fa, fb):
                assert np.array_equal(a, b), name


def test_gemm_and_row_forms_are_bit_identical(monkeypatch):
    """One step per launch: the shared maps stepped one row per warp, or as a
    GEMM over the 40 simulations sharing each (both CTA shapes)."""
    ws = _batched_small(121)
    res = _run_forms(monkeypatch, ws, 121, {
        "row": {"FDTD_TB": "0", "FDTD_ROM_GEMM_MIN": "1000"},
        "gemm1": {"FDTD_TB": "0", "FDTD_ROM_GEMM_MIN": "1", "FDTD_GEMM_RPW": "1"},
        "gemm2": {"FDTD_TB": "0", "FDTD_ROM_GEMM_MIN": "1", "FDTD_GEMM_RPW": "2"},
    })
    _assert_same_bits(res, "row")


def test_zone_chain_is_bit_identical(monkeypatch):
    """Two steps per launch with the shared maps as GEMMs in the zone chain
    (the default for shared maps), with every model in the chain one row per
    warp, and with the maps inside fused model tiles, against one step per
    launch; odd step count (a trailing single step)."""
    ws = _batched_small(121)
    monkeypatch.setenv("FDTD_TB_SMEM", "0")
    res = _run_forms(monkeypatch, ws, 121, {
        "one": {"FDTD_TB": "0", "FDTD_ROM_GEMM_MIN": "1"},
        "chain_gemm": {"FDTD_TB": "1", "FDTD_ROM_GEMM_MIN": "1", "FDTD_TB_CHAIN": "1"},
        "chain_rows": {"FDTD_TB": "1", "FDTD_ROM_GEMM_MIN": "1000", "FDTD_TB_CHAIN": "1"},
        "fused": {"FDTD_TB": "1", "FDTD_ROM_GEMM_MIN": "1", "FDTD_TB_CHAIN": "0"},
    })
    assert [res[k][2] for k in ("one", "chain_gemm", "chain_rows", "fused")] == [1, 2, 2, 2]
    _assert_same_bits(res, "one")


@pytest.mark.parametrize("rows", ["17", "auto"])
def test_zone_chain_on_tile_boundaries_is_bit_identical(monkeypatch, rows):
    """Every model (their maps not shared) in the zone chain, with probes and
    sources on strip and tile boundaries and inside zones, against one step
    per launch."""
    n = 203
    ws = _boundary_workloads(n)
    for w in ws:
        for rd in w["roms"]:
            w["probes"] += [(rd["i0"] - 2, rd["j0"] + 1), (rd["i0"] + rd["a"] + 1, rd["j0"])]
    monkeypatch.setenv("FDTD_TB_SMEM", "0")
    if rows == "auto":
        monkeypatch.delenv("FDTD_TB_ROWS", raising=False)
    else:
        monkeypatch.setenv("FDTD_TB_ROWS", rows)
    res = _run_forms(monkeypatch, ws, n, {
        "one": {"FDTD_TB": "0"},
        "chain": {"FDTD_TB": "1", "FDTD_TB_CHAIN": "1"},
    })
    assert res["chain"][2] == 2
    _assert_same_bits(res, "one")


def test_three_cta_form_is_bit_identical(monkeypatch):
    """The row-marching kernel built for 3 resident CTAs per SM (FDTD_TB_MB=3,
    an autotuner candidate: more registers per thread) against the 4-CTA
    form and one step per launch."""
    n = 203
    ws = _boundary_workloads(n)
    monkeypatch.setenv("FDTD_TB_SMEM", "0")
    monkeypatch.delenv("FDTD_TB_ROWS", raising=False)
    res = _run_forms(monkeypatch, ws, n, {
        "one": {"FDTD_TB": "0"},
        "four": {"FDTD_TB": "1", "FDTD_TB_RING": "0"},
        "three": {"FDTD_TB": "1", "FDTD_TB_MB": "3"},
    })
    assert res["three"][2] == 2
    _assert_same_bits(res, "one")


@pytest.mark.parametrize("ring", ["2", "3", "4"])
def test_staged_rows_are_bit_identical(monkeypatch, ring):
    """The row-marching kernel with its loads staged 1-3 rows ahead through
    shared memory (FDTD_TB_RING) against its register form, 17-row tiles
    (many tile starts and ends) and the automatic plan's."""
    n = 203
    ws = _boundary_workloads(n)
    monkeypatch.setenv("FDTD_TB_SMEM", "0")
    for rows in ("17", None):
        if rows:
            monkeypatch.setenv("FDTD_TB_ROWS", rows)
        else:
            monkeypatch.delenv("FDTD_TB_ROWS", raising=False)
        res = _run_forms(monkeypatch, ws, n, {
            "regs": {"FDTD_TB": "1", "FDTD_TB_RING": "0"},
            "ring": {"FDTD_TB": "1", "FDTD_TB_RING": ring},
        })
        _assert_same_bits(res, "regs")
