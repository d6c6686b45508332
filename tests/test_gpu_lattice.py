"""Many embedded models on a vacuum grid with sparse scatterers and line
sources, stepped beyond the fine-mesh CFL limit (dt = 2 x): against the FP64
oracle on a scaled lattice, at full size (8192^2, 64 models) on the windows
the oracle can recompute, and the sparse-material stencil against the dense
one bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1609_07114_gb300 as pg
import workloads
import test_gpu_parity as tp

pytestmark = pytest.mark.gpu


def lattice_context(w):
    """One model per fine-region type, embedded at every region of that type."""
    ctx = pg.FdtdContext(w["dx"], w["dy"], w["dt"], [(w["eps_r"], w["sigma"])])
    built = {}
    for rd in w["roms"]:
        key = id(rd["eps_r"])
        if key not in built:
            built[key] = pg.rom_build(rd["a"], rd["b"], rd["r"], w["dx"], w["dy"], w["dt"],
                                      rd["eps_r"], rd["sigma"], rd["q"], rule=pg.FDTD_RULE_DUAL,
                                      f0=rd["f0"])
        ctx.rom_embed(built[key], 0, rd["i0"], rd["j0"])
    return ctx, list(built.values())


def small_lattice(nsteps):
    w = workloads.lattice_8192(nsteps, n=768, pitch=256)
    for rd in w["roms"][:4]:
        w["probes"] += [(rd["i0"] - 1, rd["j0"] + 1), (rd["i0"] + rd["a"], rd["j0"] + rd["b"] - 2)]
    return w


def test_scaled_lattice_matches_oracle():
    """768^2, nine models of three types (CFL extension active), 1% lossy
    scatterers, four full-column line sources, 300 steps."""
    N = 300
    w = small_lattice(N)
    ctx, models = lattice_context(w)
    assert any(m.report.n_clamped > 0 for m in models)
    g = tp.gpu_run(ctx, [w], N)
    o, st = tp.oracle_run(w, N)
    assert tp.rel_l2(g, o) < tp.TOL
    tp.check_fields(ctx, 0, st)


def test_sparse_material_path_equals_dense_path(monkeypatch):
    N = 200
    w = small_lattice(N)
    res = {}
    for dense in ("0", "1"):
        monkeypatch.setenv("FDTD_MAT_DENSE", dense)
        ctx, _ = lattice_context(w)
        res[dense] = (tp.gpu_run(ctx, [w], N), ctx.get_fields(0))
    np.testing.assert_array_equal(res["0"][0], res["1"][0])
    for a, b in zip(res["0"][1], res["1"][1]):
        np.testing.assert_array_equal(a, b)


def test_two_step_sparse_march_equals_one_step(monkeypatch):
    """The two-step march skips the materials of background-only strip rows
    as the one-step kernel does: two steps per launch (register loads, staged
    rows, the models' maps in their tiles or in the zone chain) against one
    step per launch and against the dense-material form, bit for bit."""
    N = 201
    w = small_lattice(N)
    settings = {
        "one": {"FDTD_TB": "0"},
        "two": {"FDTD_TB": "1", "FDTD_TB_RING": "0", "FDTD_TB_CHAIN": "0"},
        "two_ring": {"FDTD_TB": "1", "FDTD_TB_RING": "3", "FDTD_TB_CHAIN": "0"},
        "two_chain": {"FDTD_TB": "1", "FDTD_TB_RING": "0", "FDTD_TB_CHAIN": "1"},
        "two_dense": {"FDTD_TB": "1", "FDTD_TB_RING": "0", "FDTD_TB_CHAIN": "0", "FDTD_MAT_DENSE": "1"},
    }
    res = {}
    for name, env in settings.items():
        for k, v in env.items():
            monkeypatch.setenv(k, v)
        ctx, _ = lattice_context(w)
        assert ctx.steps_per_launch() == (1 if name == "one" else 2)
        res[name] = (tp.gpu_run(ctx, [w], N), ctx.get_fields(0))
        monkeypatch.delenv("FDTD_MAT_DENSE", raising=False)
    assert np.abs(res["one"][0]).max() > 0
    for name in settings:
        np.testing.assert_array_equal(res[name][0], res["one"][0])
        for a, b in zip(res[name][1], res["one"][1]):
            np.testing.assert_array_equal(a, b)


def test_full_size_lattice_sampled_windows(monkeypatch):
    """8192^2 with 64 models, in the launch configuration the benchmark
    times (the library's default choice).  After N steps from rest only
    columns within N of a line source can be nonzero; the oracle recomputes
    each full-height band (with every model inside it) and probes and band
    fields are compared."""
    monkeypatch.delenv("FDTD_TB", raising=False)
    N = 40
    w = workloads.lattice_8192(N)
    # A model couples its whole interface within one step, so a band that
    # reaches a model grows by the model's width on both sides (an upper
    # bound on how far the wave can get through it).
    bands = []
    for src in w["sources"]:
        lo, hi = src["i"] - N - 3, src["i"] + N + 4
        taken = set()
        changed = True
        while changed:
            changed = False
            for k, rd in enumerate(w["roms"]):
                if k not in taken and rd["i0"] - 3 < hi and rd["i0"] + rd["a"] + 3 > lo:
                    taken.add(k)
                    lo, hi = min(lo, rd["i0"] - 3) - rd["a"] - 3, max(hi, rd["i0"] + rd["a"] + 3) + rd["a"] + 3
                    changed = True
        bands.append([max(lo, 0), min(hi, w["nx"])])
    bands.sort()
    merged = []
    for b in bands:
        if merged and b[0] <= merged[-1][1]:
            merged[-1][1] = max(merged[-1][1], b[1])
        else:
            merged.append(b)
    probes = []
    for lo, hi in merged:
        probes += [(lo + (hi - lo) // 3, 100), ((lo + hi) // 2, 4000), (hi - 5, 8000)]
    w["probes"] = probes
    ctx, _ = lattice_context(w)
    g = tp.gpu_run(ctx, [w], N)
    Ex, Ey, Hz = ctx.get_fields(0)
    mask = np.ones_like(Hz, dtype=bool)
    for lo, hi in merged:
        sub = dict(w, nx=hi - lo, eps_r=w["eps_r"][:, lo:hi], sigma=w["sigma"][:, lo:hi],
                   roms=[dict(rd, i0=rd["i0"] - lo) for rd in w["roms"] if lo < rd["i0"] and rd["i0"] + rd["a"] < hi],
                   sources=[dict(s, i=s["i"] - lo) for s in w["sources"] if lo < s["i"] < hi],
                   probes=[(i - lo, j) for (i, j) in probes if lo <= i < hi])
        o, st = tp.oracle_run(sub, N)
        sel = [k for k, (i, j) in enumerate(probes) if lo <= i < hi]
        assert tp.rel_l2(g[:, sel], o) < tp.TOL
        assert tp.rel_l2(Hz[:, lo:hi], st.Hz) < tp.TOL
        assert tp.rel_l2(Ey[:, lo + 1:hi], st.Ey[:, 1:-1]) < tp.TOL
        mask[:, lo:hi] = False
    assert np.abs(Hz[mask]).max() == 0.0
