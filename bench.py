#!/usr/bin/env python
"""Throughput benchmark of the Yee + embedded-ROM forward time march on GB300.

Workload (the large single-run configuration): a 4096 x 4096 coarse grid at
dx = 1 mm with per-cell eps_r ~ U[1,4] and sigma ~ U[0,0.02] S/m, eight
16 x 16-cell regions refined r = 4 with seeded lossy inclusions, each
replaced by a q = 200 reduced model, one differentiated-Gaussian Jy point
source and 16 Hz probes, dt = 0.95 x the fine-mesh CFL limit.  One benchmark
step = one fdtd_run of --tsteps time steps (default 2000, so the ten timed
steps cover the configuration's 20000 time steps).

Metric: Gcell-steps/s = coarse cells x time steps / device time (CUDA events
on the library's stream), reduced-model build excluded.  Multi-GPU runs are
independent replicas (the path has no exchange step): value = cells x steps
summed over ranks / max time over ranks.

--impl reference times the FP64 oracle on the host cores (the method's
reference implementation in this repository) on a bounded sample of the same
workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# the CPU oracle timings run on one host core, as they report (numpy's BLAS
# would otherwise thread the small model products); set before numpy loads
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

METRIC = "Yee+ROM Gcell-steps/s"
UNIT = "Gcell-steps/s"
BYTES_PER_CELL_STEP = 32   # read Ex, Ey, Hz, eps, sigma; write Ex, Ey, Hz (FP32)
FALLBACK_HBM_GBS = 6800.0
WORKLOAD = ("grid_4096: 4096x4096 coarse cells (dx=1mm, eps_r~U[1,4], sigma~U[0,0.02]), "
            "8 regions 16x16 r=4 with lossy inclusions, ROM q=200 (dual rule), 1 Jy source, "
            "16 Hz probes, dt=0.95 fine CFL")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    return ws, int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(el_ms, dist, device):
    """The slowest rank's time: the job's time (replicas run independently;
    this timing reduction is the only collective)."""
    if not dist:
        return el_ms
    import torch
    t = torch.tensor([el_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(cells, tsteps, steps, ranks, el_ms):
    """Whole-job Gcell-steps/s: every rank advanced `cells` cells by
    tsteps x steps time steps in at most el_ms."""
    return cells * tsteps * steps * ranks / (el_ms / 1e3) / 1e9


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


PROFILE_OF = {"yee_step_kernel": "yee_step_grid4096.md", "yee_tb2m_kernel": "yee_tb2m_grid4096.md"}


def profile_traffic(kernel="yee_step_kernel"):
    """DRAM bytes per launch of `kernel` on the 4096^2 workload from the
    committed ncu summary, if it was taken on the current kernel source."""
    summ = os.path.join(ROOT, "profiles", PROFILE_OF[kernel])
    if not os.path.exists(summ):
        return None
    sha = stencil_source_sha() if kernel == "yee_step_kernel" else march_source_sha()
    txt = open(summ).read()
    m_sha = re.search(r"kernel source sha256\[:16\]:\s*([0-9a-f]+)", txt)
    m_b = re.search(r"dram bytes per full-size launch:\s*([0-9.eE+]+)", txt)
    if m_sha and m_b and m_sha.group(1) == sha:
        return float(m_b.group(1))
    return None


def _code_only(text):
    """Source text without // comments and blank lines (so that a comment
    edit does not void a profile taken on the same code)."""
    lines = (re.sub(r"//.*", "", ln).rstrip() for ln in text.splitlines())
    return "\n".join(ln for ln in lines if ln.strip())


def stencil_source_sha():
    """Hash of the stencil kernel's code: the grid and tile structures of
    kernels.cuh (up to the reduced-model structures) plus the part of fdtd.cu
    from the edge-coefficient helper up to the reduced-model kernel, comments
    removed."""
    d = os.path.join(ROOT, "paper_1609_07114_gb300", "csrc")
    cu = open(os.path.join(d, "fdtd.cu")).read()
    a = cu.index("// E-edge coefficients from the two adjacent cells")
    b = cu.index("// Eq. (23) for every embedded model")
    kh = open(os.path.join(d, "kernels.cuh")).read()
    kh = kh[:kh.index("struct RomInstDev")]
    h = hashlib.sha256(_code_only(kh).encode() + _code_only(cu[a:b]).encode())
    return h.hexdigest()[:16]


def march_source_sha():
    """Hash of the row-marching two-step kernel's code: the structures of
    kernels.cuh, fdtd.cu's edge-coefficient helper and tb_march.cuh,
    comments removed."""
    d = os.path.join(ROOT, "paper_1609_07114_gb300", "csrc")
    cu = open(os.path.join(d, "fdtd.cu")).read()
    a = cu.index("// E-edge coefficients from the two adjacent cells")
    b = cu.index("// Fused coarse H and E half steps over one tile")
    kh = open(os.path.join(d, "kernels.cuh")).read()
    kh = kh[:kh.index("struct RomInstDev")]
    tm = open(os.path.join(d, "tb_march.cuh")).read()
    return hashlib.sha256(_code_only(kh).encode() + _code_only(cu[a:b]).encode()
                          + _code_only(tm).encode()).hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.p = None

    def __enter__(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.p = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        rows = [r.split(",") for r in getattr(self, "out", "").strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = sorted(float(r[1]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].strip() == "Active"})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows)}


def build_problem(nsteps_total, grid=4096):
    import workloads
    if grid == 4096:
        return workloads.grid_4096(nsteps_total)
    # same recipe at another size (profiling captures of a smaller case)
    return workloads.random_grid(1, grid, grid, 8, 16, 4, 200, nsteps_total, dt_factor=0.95)


def cpu_sample(w, steps):
    """Times the FP64 oracle (as it stands) stepping the full grid with all
    its embedded models; the models are built first, untimed, as for the
    GPU metric."""
    from oracle import problem, scheme
    grid, emb, _ = problem.build(w)
    st = scheme.State(*grid.zeros())
    out = [[0.0] * len(w["probes"])] * steps
    import numpy as np
    out = np.zeros((steps, len(w["probes"])))
    t0 = time.perf_counter()
    for n in range(steps):
        scheme.step(grid, st, emb, w["sources"], n, w["probes"], out)
    dt = time.perf_counter() - t0
    cells = w["nx"] * w["ny"]
    return {"value": cells * steps / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{steps} time steps of the full 4096x4096 grid with its 8 models (numpy FP64, "
                      f"{dt:.1f} s; model build untimed)"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    args.cpu_sample_steps = min(args.cpu_sample_steps, 3)   # bounded: the run ends in ~1 min
    w = build_problem(args.cpu_sample_steps * (args.steps + args.warmup) + 1)
    from oracle import problem, scheme
    import numpy as np
    grid, emb, _ = problem.build(w)
    st = scheme.State(*grid.zeros())
    out = np.zeros((args.cpu_sample_steps * (args.steps + args.warmup), len(w["probes"])))
    n = 0
    for _ in range(args.warmup):
        for _ in range(args.cpu_sample_steps):
            scheme.step(grid, st, emb, w["sources"], n, w["probes"], out)
            n += 1
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for _ in range(args.cpu_sample_steps):
            scheme.step(grid, st, emb, w["sources"], n, w["probes"], out)
            n += 1
    el = time.perf_counter() - t0
    cells = w["nx"] * w["ny"]
    value = cells * args.cpu_sample_steps * args.steps / el / 1e9
    sample = (f"each step = {args.cpu_sample_steps} time steps of the full 4096x4096 grid with its 8 "
              f"models, FP64 numpy on 1 host core")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "time_steps_per_step": args.cpu_sample_steps},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def run_batched(args):
    """Batched vs plain: 256 simulations (64 each of 128^2, 256^2, 512^2,
    1024^2) sharing four reduced models, advanced together in one launch per
    step, against the same simulations run one context and one fdtd_run at a
    time."""
    import numpy as np
    import torch
    import paper_1609_07114_gb300 as pg
    from paper_1609_07114_gb300 import build as pbuild
    import workloads
    pbuild.build()
    K, W, T = args.steps, args.warmup, args.tsteps
    Tp = max(T // 5, 32)      # time steps of each one-at-a-time run (two runs per simulation)
    w = workloads.batched_256(max((W + K) * T, 2 * Tp))
    models = [pg.rom_build(md["a"], md["b"], md["r"], w["dx"], w["dy"], w["dt"], md["eps_r"],
                           md["sigma"], md["q"], f0=md["f0"]) for md in w["models"]]
    sims = w["sims"]

    def make_ctx(group):
        ctx = pg.FdtdContext(w["dx"], w["dy"], w["dt"], [(s["eps_r"], s["sigma"]) for s in group])
        for k, s in enumerate(group):
            for (mi, i0, j0) in s["place"]:
                ctx.rom_embed(models[mi], k, i0, j0)
        waves = [torch.tensor(s["source"]["wave"].astype(np.float32), device="cuda") for s in group]
        probes = [(k, s["probe"][0], s["probe"][1]) for k, s in enumerate(group)]
        return ctx, waves, probes

    def step(ctx, group, waves, probes, k0, n, out):
        src = [dict(s["source"], sim=k, wave=waves[k][k0:k0 + n]) for k, s in enumerate(group)]
        ctx.fdtd_run(n, src, probes, out)

    cells = sum(s["nx"] * s["ny"] for s in sims)
    ctx, waves, probes = make_ctx(sims)
    out = torch.zeros((T, len(probes)), dtype=torch.float32, device="cuda")
    for k in range(W):
        step(ctx, sims, waves, probes, k * T, T, out)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with ClockSampler() as clk:
        e0.record(stream)
        for k in range(W, W + K):
            step(ctx, sims, waves, probes, k * T, T, out)
        e1.record(stream)
        torch.cuda.synchronize()
    el_b = e0.elapsed_time(e1) / 1e3
    batched = cells * T * K / el_b / 1e9
    ctx.set_timing(True)
    step(ctx, sims, waves, probes, 0, T, out)
    yee_ms, n_yee, post_ms, n_post = ctx.kernel_times()
    spl = ctx.steps_per_launch()
    ctx.close()
    # plain: one context and one fdtd_run at a time, Tp steps each
    el_p = 0.0
    outp = torch.zeros((Tp, 1), dtype=torch.float32, device="cuda")
    for s in sims:
        c1, wv, pr = make_ctx([s])
        step(c1, [s], wv, pr, 0, Tp, outp)                  # warm (graph capture)
        torch.cuda.synchronize()
        e0.record(stream)
        step(c1, [s], wv, pr, Tp, Tp, outp)
        e1.record(stream)
        torch.cuda.synchronize()
        el_p += e0.elapsed_time(e1) / 1e3
        c1.close()
    plain = cells * Tp / el_p / 1e9
    hbm, kind = peaks()
    achieved = BYTES_PER_CELL_STEP * cells / (yee_ms / n_yee / 1e3) / 1e9
    print(json.dumps({
        "metric": "batched " + METRIC, "value": batched, "unit": UNIT, "n_gpus": 1, "steps": K,
        "warmup": W, "ms_per_step": el_b / K * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batched_256: 64 each of 128^2, 256^2, 512^2, 1024^2 coarse grids, "
                               "4 shared ROMs r=3 q=40/80/160/320, every simulation in each launch",
                   "time_steps_per_step": T, "cells": cells,
                   "plain_value": plain, "plain_time_steps_per_sim": Tp,
                   "batched_over_plain": batched / plain},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": None, "peak_kind": kind,
                     "kernel": "yee_tb2m_kernel" if spl == 2 else "yee_step_kernel",
                     "kernel_avg_ms": yee_ms / n_yee, "steps_per_launch": spl,
                     "rom_post_avg_ms": post_ms / n_post if n_post else None},
        # per step: stencil + model/probe kernel, or per pair of steps: model
        # tiles + row-marching kernel; one counter advance per 16 steps
        "gpu_launches": K * ((T // 2) * 2 + 2 * (T % 2) if spl == 2 else 2 * T) + K * (T // 16),
        "clocks": clk.summary()}))


def run_adjoint(args):
    """Adjoint/forward time ratio: 16 simulations of 1024^2 cells with two
    shared q = 120 models each, J = sum of Hz^2 at 8 probes per simulation
    over --tsteps steps (default 10000), checkpoints every 500 steps."""
    import numpy as np
    import torch
    import paper_1609_07114_gb300 as pg
    from paper_1609_07114_gb300 import build as pbuild
    import workloads
    pbuild.build()
    N = args.tsteps if args.tsteps != 2000 else 10000
    w = workloads.adjoint_16(N, nsim=args.adj_nsim)
    models = [pg.rom_build(md["a"], md["b"], md["r"], w["dx"], w["dy"], w["dt"], md["eps_r"],
                           md["sigma"], md["q"], f0=md["f0"]) for md in w["models"]]

    def make_ctx():
        ctx = pg.FdtdContext(w["dx"], w["dy"], w["dt"], [(s["eps_r"], s["sigma"]) for s in w["sims"]])
        for k, s in enumerate(w["sims"]):
            for (mi, i0, j0) in s["place"]:
                ctx.rom_embed(models[mi], k, i0, j0)
        return ctx

    waves = [torch.tensor(s["source"]["wave"].astype(np.float32), device="cuda") for s in w["sims"]]
    src = [dict(s["source"], sim=k, wave=waves[k]) for k, s in enumerate(w["sims"])]
    probes = [(k, i, j) for k, s in enumerate(w["sims"]) for (i, j) in s["probes"]]
    cells = sum(s["nx"] * s["ny"] for s in w["sims"])
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fwd, adj = [], []
    out = torch.zeros((N, len(probes)), dtype=torch.float32, device="cuda")
    with ClockSampler() as clk:
        for rep in range(args.warmup + args.steps):
            ctx = make_ctx()
            torch.cuda.synchronize()
            e0.record(stream)
            ctx.fdtd_run(N, src, probes, out)
            e1.record(stream)
            torch.cuda.synchronize()
            tf = e0.elapsed_time(e1) / 1e3
            ctx.close()
            ctx = make_ctx()
            torch.cuda.synchronize()
            e0.record(stream)
            J, ge, gs, gw = ctx.fdtd_grad(N, src, probes, 500)
            e1.record(stream)
            torch.cuda.synchronize()
            ta = e0.elapsed_time(e1) / 1e3
            ctx.close()
            if rep >= args.warmup:
                fwd.append(tf)
                adj.append(ta)
    tf, ta = float(np.median(fwd)), float(np.median(adj))
    print(json.dumps({
        "metric": "adjoint/forward time ratio", "value": ta / tf, "unit": "x", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ta * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"adjoint_16: {args.adj_nsim} x 1024^2 coarse grids, 2 shared ROMs r=3 q=120 each, "
                               "8 probes per simulation, J = sum Hz^2, checkpoints every 500 steps",
                   "time_steps": N, "cells": cells, "forward_s": tf, "adjoint_s": ta,
                   "forward_gcell_steps_per_s": cells * N / tf / 1e9,
                   "gradient_gcell_steps_per_s": cells * N / ta / 1e9, "J": J},
        "clocks": clk.summary()}))


def run_lattice(args):
    """Many heterogeneous models with CFL extension: an 8192^2 vacuum grid
    with 1% lossy scatterers, 64 embedded models of three types (r = 5, q =
    60/180/400) at dt = 2 x the fine-mesh CFL limit, four full-column line
    sources, 16 probes.  One benchmark step = --tsteps time steps (default
    1000, so ten timed steps are the configuration's 10000).  --lossless
    runs the sigma = 0 variant; --energy-every E then also records the
    storage function every E steps over --tsteps x (warmup + steps) steps and
    reports its drift after the pulse has left the sources."""
    import numpy as np
    import torch
    import paper_1609_07114_gb300 as pg
    from paper_1609_07114_gb300 import build as pbuild
    import workloads
    pbuild.build()
    K, W, T = args.steps, args.warmup, args.tsteps
    total = (W + K) * T
    n = args.lattice_n
    w = workloads.lattice_8192(min(total, 20000), n=n, pitch=n // 8, lossless=args.lossless)
    ctx = pg.FdtdContext(w["dx"], w["dy"], w["dt"], [(w["eps_r"], w["sigma"])])
    t0 = time.perf_counter()
    built = {}
    for rd in w["roms"]:
        key = id(rd["eps_r"])
        if key not in built:
            built[key] = pg.rom_build(rd["a"], rd["b"], rd["r"], w["dx"], w["dy"], w["dt"], rd["eps_r"],
                                      rd["sigma"], rd["q"], f0=rd["f0"])
        ctx.rom_embed(built[key], 0, rd["i0"], rd["j0"])
    rom_seconds = time.perf_counter() - t0
    t0 = time.perf_counter()   # the same three models built on the device (not used below)
    for rd in {id(rd["eps_r"]): rd for rd in w["roms"]}.values():
        pg.rom_build_gpu(rd["a"], rd["b"], rd["r"], w["dx"], w["dy"], w["dt"], rd["eps_r"], rd["sigma"],
                         rd["q"], f0=rd["f0"])
    torch.cuda.synchronize()
    rom_gpu_seconds = time.perf_counter() - t0
    nwave = len(w["sources"][0]["wave"])
    wave = torch.zeros(total + T, dtype=torch.float32, device="cuda")
    wave[:nwave] = torch.tensor(w["sources"][0]["wave"].astype(np.float32), device="cuda")
    probes = [(0, i, j) for (i, j) in w["probes"]]
    out = torch.zeros((T, len(probes)), dtype=torch.float32, device="cuda")

    def one_step(k):
        src = [dict(s, sim=0, wave=wave[k * T:(k + 1) * T]) for s in w["sources"]]
        ctx.fdtd_run(T, src, probes, out)

    energy = []
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if args.energy_every:
        E = args.energy_every
        assert T % E == 0
        src_all = [dict(s, sim=0, wave=wave) for s in w["sources"]]
        t_run = 0.0
        with ClockSampler() as clk:
            for k in range(total // E):
                src = [dict(s, wave=s["wave"][k * E:(k + 1) * E]) for s in src_all]
                torch.cuda.synchronize()
                e0.record(stream)
                ctx.fdtd_run(E, src, probes, out[:E] if E <= T else None)
                e1.record(stream)
                torch.cuda.synchronize()
                t_run += e0.elapsed_time(e1) / 1e3
                energy.append(float(ctx.energy()[0]))
        el_s = t_run
        nsteps_timed = total
    else:
        for k in range(W):
            one_step(k)
        torch.cuda.synchronize()
        with ClockSampler() as clk:
            e0.record(stream)
            for k in range(W, W + K):
                one_step(k)
            e1.record(stream)
            torch.cuda.synchronize()
        el_s = e0.elapsed_time(e1) / 1e3
        nsteps_timed = K * T
    cells = w["nx"] * w["ny"]
    value = cells * nsteps_timed / el_s / 1e9
    ctx.set_timing(True)
    for k in range(2):
        one_step(k)
    yee_ms, n_yee, post_ms, n_post = ctx.kernel_times()
    ctx.set_timing(False)
    spl = ctx.steps_per_launch()
    f_nb = float(np.mean((w["eps_r"] != 1.0) | (w["sigma"] != 0.0)))
    # fields + the materials of non-background cells (the two-step kernel
    # reads every material)
    bpc = 32.0 if spl == 2 else 24.0 + 8.0 * f_nb
    hbm, kind = peaks()
    achieved = bpc * cells / (yee_ms / n_yee / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": K, "warmup": W,
        "ms_per_step": el_s / max(nsteps_timed // T, 1) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"lattice_{n}: {n}^2 vacuum grid, {100 * f_nb:.2f}% "
                               f"{'lossless' if args.lossless else 'lossy'} scatterer cells, 64 ROMs of 3 "
                               "types (r=5, q=60/180/400) at dt=2x fine CFL, 4 full-column Jy line "
                               "sources, 16 Hz probes",
                   "time_steps_per_step": T, "nx": w["nx"], "ny": w["ny"], "roms": len(w["roms"]),
                   "rom_q": sorted({m.q for m in built.values()}),
                   "rom_clamped": [m.report.n_clamped for m in built.values()],
                   "rom_build_s": round(rom_seconds, 3), "rom_build_gpu_s": round(rom_gpu_seconds, 3),
                   "l2": f"inputs larger than L2: {24 * n * n / 1e9:.2f} GB of fields per time step (L2 129 MB)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": None, "peak_kind": kind,
                     "kernel": "yee_tb2m_kernel" if spl == 2 else "yee_step_kernel",
                     "kernel_avg_ms": yee_ms / n_yee, "steps_per_launch": spl,
                     "alg_bytes_per_cell_step": bpc, "rom_post_avg_ms": post_ms / max(n_post, 1)},
        "gpu_launches": (nsteps_timed // T) * (2 * T + T // 16),
        "clocks": clk.summary(),
    }
    if energy:
        E = args.energy_every
        wv = np.abs(w["sources"][0]["wave"])
        n_quiet = int(np.nonzero(wv > 1e-12 * wv.max())[0][-1]) + 1   # sources silent from here on
        k0 = min(len(energy) - 1, (n_quiet + E - 1) // E)
        ref = energy[k0]
        tail = np.array(energy[k0:])
        x = np.arange(len(tail)) * E
        slope = float(np.polyfit(x, tail / ref, 1)[0]) if len(tail) > 2 else 0.0
        line["energy"] = {"every": E, "samples": len(energy), "from_step": k0 * E, "W_ref": ref,
                          "max_rel_dev": float(np.abs(tail / ref - 1).max()),
                          "final_rel_dev": float(tail[-1] / ref - 1),
                          "slope_per_1e6_steps": slope * 1e6}
    print(json.dumps(line))
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tsteps", type=int, default=2000, help="time steps per benchmark step")
    ap.add_argument("--cpu-sample-steps", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--grid", type=int, default=4096, help="coarse grid size (4096 = the benchmark)")
    ap.add_argument("--workload", default="grid", choices=["grid", "batched", "adjoint", "lattice"])
    ap.add_argument("--lossless", action="store_true", help="lattice: sigma = 0 everywhere")
    ap.add_argument("--adj-nsim", type=int, default=16,
                    help="adjoint: simulations in the batch (16 = the configuration)")
    ap.add_argument("--lattice-n", type=int, default=8192,
                    help="lattice: grid size (8192 = the configuration; 64 models at pitch n/8)")
    ap.add_argument("--energy-every", type=int, default=0,
                    help="lattice: record the storage function every E steps")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "adjoint":
        if args.steps == 10:
            args.steps = 3
        args.warmup = 1 if args.warmup == 3 else args.warmup
        run_adjoint(args)
        return
    if args.workload == "lattice":
        if args.tsteps == 2000:
            args.tsteps = 1000         # 10 timed steps = the configuration's 10000 time steps
        run_lattice(args)
        return
    if args.workload == "batched":
        if args.tsteps == 2000:
            args.tsteps = 500          # 10 timed steps = the batch's 5000 time steps
        run_batched(args)
        return

    import numpy as np
    import torch
    import paper_1609_07114_gb300 as pg
    from paper_1609_07114_gb300 import build as pbuild

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        pbuild.build()
    if dist:
        dist.barrier()

    K, W, T = args.steps, args.warmup, args.tsteps
    total = (W + K) * T
    w = build_problem(total, args.grid)
    ctx = pg.FdtdContext(w["dx"], w["dy"], w["dt"], [(w["eps_r"], w["sigma"])])
    models = []
    t0 = time.perf_counter()
    for rd in w["roms"]:
        m = pg.rom_build(rd["a"], rd["b"], rd["r"], w["dx"], w["dy"], w["dt"], rd["eps_r"],
                         rd["sigma"], rd["q"], f0=rd["f0"])
        ctx.rom_embed(m, 0, rd["i0"], rd["j0"])
        models.append(m)
    rom_seconds = time.perf_counter() - t0
    wave = torch.tensor(w["sources"][0]["wave"].astype(np.float32), device="cuda")
    probes = [(0, i, j) for (i, j) in w["probes"]]
    out = torch.zeros((T, len(probes)), dtype=torch.float32, device="cuda")
    src0 = w["sources"][0]

    def one_step(k):
        src = [dict(src0, sim=0, wave=wave[k * T:(k + 1) * T])]
        ctx.fdtd_run(T, src, probes, out)

    for k in range(W):
        one_step(k)
    torch.cuda.synchronize()
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        uuid = None
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(uuid) as clk:
        e0.record(stream)
        for k in range(W, W + K):
            one_step(k)
        e1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    el_ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    cells = w["nx"] * w["ny"]
    value = replica_throughput(cells, T, K, ws, el_ms)

    # Per-kernel device time of the dominant (stencil) kernel, CUDA events on
    # the launching stream, over a second pass of the same K steps.
    # On the two-steps-per-launch path a launch is the row-marching kernel
    # (with the model tiles beside it): one read and one write pass over the
    # fields and materials for two steps, so the algorithmic bytes per launch
    # are the same 32 B per cell.
    spl = ctx.steps_per_launch()
    kernel = "yee_tb2m_kernel" if spl == 2 else "yee_step_kernel"
    ctx.set_timing(True)
    for k in range(K):
        one_step(k)
    yee_ms, n_yee, post_ms, n_post = ctx.kernel_times()
    ctx.set_timing(False)
    yee_avg_s = yee_ms / n_yee / 1e3
    alg_bytes = BYTES_PER_CELL_STEP * cells
    hbm, kind = peaks()
    achieved = alg_bytes / yee_avg_s / 1e9
    traffic = profile_traffic(kernel)

    # End to end through the host-buffer entry point: H2D of the step's
    # source samples from pinned memory, D2H of its probe samples.
    hw = torch.empty(T, dtype=torch.float32, pin_memory=True)
    hw.copy_(torch.tensor(src0["wave"][:T].astype(np.float32)))
    hwn = hw.numpy()
    ctx.fdtd_run_host(T, [dict(src0, sim=0, wave=hwn)], probes)   # warm the host path
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(K):
        ctx.fdtd_run_host(T, [dict(src0, sim=0, wave=hwn)], probes)
    e2e_s = time.perf_counter() - t0
    e2e = {"value": cells * T * K * ws / e2e_s / 1e9, "unit": UNIT,
           "h2d_bytes_per_step": 4 * T, "d2h_bytes_per_step": 4 * T * len(probes)}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_sample(build_problem(args.cpu_sample_steps + 1), args.cpu_sample_steps)

    if spl == 2:   # per pair: the model tiles (if any) and the row-marching kernel
        launches_per_run = (T // 2) * (2 if models else 1) + (2 if T % 2 else 0) + T // 16
    else:
        launches_per_run = 2 * T + T // 16
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W,
        "ms_per_step": el_ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if args.grid == 4096 else f"grid {args.grid}^2, same recipe",
                   "time_steps_per_step": T, "nx": w["nx"], "ny": w["ny"],
                   "roms": len(w["roms"]), "rom_q": [m.q for m in models],
                   "rom_build_s": round(rom_seconds, 3),
                   "l2": "inputs larger than L2: 0.47 GB of fields+materials per time step (L2 129 MB)",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic, "peak_kind": kind,
                     "kernel": kernel, "kernel_avg_ms": yee_avg_s * 1e3, "steps_per_launch": spl,
                     "alg_bytes_per_launch": alg_bytes,
                     "rom_post_avg_ms": post_ms / n_post if n_post else None},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": K * launches_per_run,
        "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
