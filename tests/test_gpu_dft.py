"""Running DFT monitors of Hz (frequency responses) against the oracle's DFT
of the oracle's own probe samples."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1609_07114_gb300 as pg
import workloads
import test_gpu_parity as tp
from oracle import dft

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_cavity_response_over_split_runs():
    """60^2 cavity with its q = 60 model, 2000 steps taken as 700 + 600 + 700
    (accumulation carries across runs, time from the context's step count);
    48 frequencies 1-60 GHz at the two probes and one more cell."""
    w = workloads.cavity_60(2000)
    mons = list(w["probes"]) + [(20, 20)]
    freqs = np.linspace(1e9, 60e9, 48)
    ctx, _ = tp.gpu_context([w])
    ctx.dft_set(mons, freqs)
    wave = torch.tensor(np.asarray(w["sources"][0]["wave"], np.float32), device="cuda")
    k = 0
    for n in (700, 600, 700):
        ctx.fdtd_run(n, [dict(w["sources"][0], sim=0, wave=wave[k:k + n])])
        k += n
    X = ctx.dft_get()
    wo = dict(w, probes=mons)
    o, _ = tp.oracle_run(wo, 2000)
    ref = dft.dft(o, w["dt"], freqs)
    assert rel(X, ref) < 1e-4
    for m in range(len(mons)):
        assert rel(X[m], ref[m]) < 1e-4


def test_monitors_in_a_batch_and_resume():
    """Two simulations of a batch, monitors in both; a run of 150 steps, then
    save / fresh context / load with the accumulators handed over, 150 more:
    equals one context running 300 steps with its monitors."""
    ws = [workloads.random_grid(90 + k, 140 + 30 * k, 110, 2, 5, 3, 30, 300, n_probes=3) for k in range(2)]
    mons = [(s, i, j) for s, w in enumerate(ws) for (i, j) in w["probes"]]
    freqs = np.array([5e9, 17.5e9, 30e9, 42e9])

    def run(ctx, k0, n):
        srcs = []
        for s, w in enumerate(ws):
            t = torch.tensor(np.asarray(w["sources"][0]["wave"][k0:k0 + n], np.float32), device="cuda")
            srcs.append(dict(w["sources"][0], sim=s, wave=t))
            run.keep.append(t)
        ctx.fdtd_run(n, srcs)
        torch.cuda.synchronize()
    run.keep = []

    full, _ = tp.gpu_context(ws)
    full.dft_set(mons, freqs)
    run(full, 0, 300)
    X_full = full.dft_get()

    a, _ = tp.gpu_context(ws)
    a.dft_set(mons, freqs)
    run(a, 0, 150)
    blob = a.save_state()
    X_half = a.dft_get()
    b, _ = tp.gpu_context(ws)
    b.load_state(blob)
    b.dft_set(mons, freqs, init=X_half)
    run(b, 150, 150)
    X_res = b.dft_get()
    assert rel(X_res, X_full) < 1e-12
    # against the oracle, per simulation
    for s, w in enumerate(ws):
        o, _ = tp.oracle_run(w, 300)
        ref = dft.dft(o, w["dt"], freqs)
        sel = [k for k, m in enumerate(mons) if m[0] == s]
        assert rel(X_full[sel], ref) < 1e-4


def test_bad_monitor_is_rejected():
    w = workloads.cavity_60(10)
    ctx, _ = tp.gpu_context([w])
    with pytest.raises(pg.FdtdError):
        ctx.dft_set([(60, 3)], [1e9])
    with pytest.raises(pg.FdtdError):
        ctx.dft_set([(3, 3)], [-1.0])
    ctx.dft_set([], [])
    assert ctx.dft_get().shape == (0, 0)
