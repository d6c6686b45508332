#!/usr/bin/env python
"""Throughput benchmark of the Yee + embedded-ROM time march on GB300.

Headline workload (the large single-run configuration): a 4096 x 4096 coarse
grid at dx = 1 mm with per-cell eps_r ~ U[1,4] and sigma ~ U[0,0.02] S/m,
eight 16 x 16-cell regions refined r = 4 with seeded lossy inclusions, each
replaced by a q = 200 reduced model, one differentiated-Gaussian Jy point
source and 16 Hz probes, dt = 0.95 x the fine-mesh CFL limit.  One benchmark
step = one fdtd_run of --tsteps time steps (default 2000, so ten timed steps
cover the configuration's 20000 time steps).

Metric: Gcell-steps/s = coarse cells x time steps / device time (CUDA events
on the library's stream), reduced-model build excluded.  Multi-GPU runs are
independent replicas (the path has no exchange step): value = cells x steps
summed over ranks / max time over ranks.

The default single-GPU line also carries the other three parts of the
metric, each measured on its own workload with its own timed region:
  "batched"  256 uneven grids sharing four models in every launch, against the
             same simulations run one context and one fdtd_run at a time;
  "adjoint"  the gradient / forward time ratio of 16 x 1024^2 grids;
  "lattice"  the 8192^2 grid with 64 models of three types at dt = 2 x the
             fine-mesh CFL limit.
Each carries a roofline record of its stencil kernel.  Kernel times come from
graph replays of that kernel alone (fdtd_time_stencil: no per-kernel events),
so a launch never looks longer than the step it belongs to.

The CPU baseline runs the FP64 oracle as it stands on every usable host core:
the problem is built once, then one forked process per core steps its own copy
of the fields (independent replicas of the same sample; started before any
CUDA call).  --impl reference times the same way on the same configuration.
"""
from __future__ import annotations

import argparse
import atexit
import hashlib
import json
import os
import re
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# each oracle process runs on one host core (numpy's BLAS would otherwise
# thread the small model products); set before numpy loads
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

METRIC = "Yee+ROM Gcell-steps/s"
UNIT = "Gcell-steps/s"
BYTES_PER_CELL_STEP = 32   # one step: read Ex, Ey, Hz, eps, sigma; write Ex, Ey, Hz (FP32)
FALLBACK_HBM_GBS = 6800.0
WORKLOAD = ("grid_4096: 4096x4096 coarse cells (dx=1mm, eps_r~U[1,4], sigma~U[0,0.02]), "
            "8 regions 16x16 r=4 with lossy inclusions, ROM q=200 (dual rule), 1 Jy source, "
            "16 Hz probes, dt=0.95 fine CFL")
# autotuner results of this run (contexts of the same shape reuse them)
TUNE_CACHE = os.path.join("/tmp", f"fdtd_tune_{os.getpid()}.txt")
TUNE = [True]   # --no-tune: the fixed rule (and the FDTD_* environment) instead


def autotune(ctx):
    return ctx.autotune(TUNE_CACHE) if TUNE[0] else dict(ctx.plan(), fixed_rule=True)
atexit.register(lambda: os.path.exists(TUNE_CACHE) and os.remove(TUNE_CACHE))
CONFIG = {"workload": WORKLOAD, "nx": 4096, "ny": 4096, "roms": 8, "rom_q": 200,
          "l2": "inputs larger than L2: 0.47 GB of fields+materials per time step (L2 129 MB)"}


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


def launches_per_run(T, spl, ninst, nchain):
    """This library's kernel launches in one fdtd_run of T steps: per pair of
    steps the row-marching kernel, the fused model tiles (if any) and the four
    kernels of the zone chain (if any); per single step the stencil and the
    model/probe kernel; one counter advance per 16-step graph."""
    if spl == 2:
        per_pair = 1 + (1 if ninst > nchain else 0) + (4 if nchain else 0)
        return (T // 2) * per_pair + (2 if T % 2 else 0) + T // 16
    return 2 * T + T // 16


def roofline(alg_bytes_per_launch, kernel_ms, kernel, spl, value=None, bpc=BYTES_PER_CELL_STEP, traffic=None):
    """Roofline record of a stencil kernel: algorithmic bytes of one launch
    over its device time (graph replay of the kernel alone), against the
    measured copy bandwidth; and, for the whole path, the one-step
    convention (bpc bytes per cell-step at the measured throughput), which
    exceeds 1 when a launch advances two steps per pass over the fields."""
    hbm, kind = peaks()
    achieved = alg_bytes_per_launch / (kernel_ms / 1e3) / 1e9
    r = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
         "traffic": traffic, "peak_kind": kind, "kernel": kernel, "kernel_avg_ms": kernel_ms,
         "kernel_timing": "graph replay of the stencil kernel alone (no per-kernel events)",
         "steps_per_launch": spl, "alg_bytes_per_launch": alg_bytes_per_launch}
    if value is not None:
        r["one_step_convention"] = {"alg_bytes_per_cell_step": bpc, "achieved": value * bpc,
                                    "frac": value * bpc / hbm}
    return r


# ---------------------------------------------------------------- CPU oracle

def _usable_cores():
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def _available_bytes():
    """Host memory this process may still use: MemAvailable, capped by a
    cgroup limit when one is set."""
    avail = None
    try:
        for ln in open("/proc/meminfo"):
            if ln.startswith("MemAvailable:"):
                avail = int(ln.split()[1]) * 1024
    except OSError:
        pass
    for lim_p, use_p in (("/sys/fs/cgroup/memory.max", "/sys/fs/cgroup/memory.current"),
                         ("/sys/fs/cgroup/memory/memory.limit_in_bytes",
                          "/sys/fs/cgroup/memory/memory.usage_in_bytes")):
        try:
            lim = open(lim_p).read().strip()
            if lim != "max" and int(lim) < (1 << 60):
                room = int(lim) - int(open(use_p).read().strip())
                avail = room if avail is None else min(avail, room)
        except (OSError, ValueError):
            pass
    return avail if avail is not None else 8 << 30


_ORACLE = {}


def _oracle_replica(bar, q, warm, timed):
    """One forked process: steps its own fields of the shared problem (the
    oracle's step as it stands); the timed steps lie between two barriers."""
    import numpy as np
    from oracle import scheme
    grid, emb, w = _ORACLE["grid"], _ORACLE["emb"], _ORACLE["w"]
    st = scheme.State(*grid.zeros())
    out = np.zeros((warm + timed, len(w["probes"])))
    for n in range(warm):
        scheme.step(grid, st, emb, w["sources"], n, w["probes"], out)
    bar.wait()
    t0 = time.perf_counter()
    for n in range(warm, warm + timed):
        scheme.step(grid, st, emb, w["sources"], n, w["probes"], out)
    t1 = time.perf_counter()
    q.put((t0, t1))
    bar.wait()


def oracle_procs(cells, max_procs=None):
    """Processes for the oracle: one per usable host core, fewer if host
    memory is short (half of what is available, ~96 B per cell each)."""
    P = max(1, min(_usable_cores(), int(0.5 * _available_bytes() / (96 * cells))))
    return min(P, max_procs) if max_procs else P


def oracle_replicas(P, warm, timed):
    """Runs the prepared oracle problem in P forked processes, each stepping
    warm + timed time steps of its own copy of the fields.  Returns
    (cell-steps/s over the timed region of all processes, wall seconds of that
    region).  Must run before any CUDA call in this process."""
    import multiprocessing as mp
    w = _ORACLE["w"]
    cells = w["nx"] * w["ny"]
    ctx = mp.get_context("fork")
    bar, q = ctx.Barrier(P), ctx.Queue()
    ps = [ctx.Process(target=_oracle_replica, args=(bar, q, warm, timed)) for _ in range(P)]
    for p in ps:
        p.start()
    spans = [q.get() for _ in range(P)]
    for p in ps:
        p.join()
    wall = max(b for _, b in spans) - min(a for a, _ in spans)
    return cells * timed * P / wall, wall


def prepare_oracle(nsteps):
    """Builds the oracle's 4096^2 problem (its own FP64 model builds) once."""
    from oracle import problem
    w = build_problem(nsteps + 1)
    grid, emb, _ = problem.build(w)
    _ORACLE.update(grid=grid, emb=emb, w=w)
    return w["nx"] * w["ny"]


def host_cpu():
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part", "hardware")):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_baseline(timed=4):
    """The oracle on every usable host core (independent replicas), and on one
    core, each over `timed` time steps of the full 4096^2 grid with its 8
    models after one warm-up step; model build untimed."""
    cells = prepare_oracle(timed + 1)
    P = oracle_procs(cells)
    v, wall = oracle_replicas(P, 1, timed)
    v1, _ = oracle_replicas(1, 1, timed)
    _ORACLE.clear()
    return {"value": v / 1e9, "unit": UNIT, "cores": P, "kind": "oracle",
            "sample": f"{timed} time steps (after 1 warm-up step) of the full 4096x4096 grid with its 8 "
                      f"models, numpy FP64, in each of {P} forked processes (one per usable host core: "
                      f"independent replicas of the same problem, {wall:.1f} s); model build untimed",
            "value_1core": v1 / 1e9, "host": {"usable_cores": _usable_cores(), "cpu": host_cpu()}}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    s = 1     # time steps per benchmark step in each process: the run ends in about a minute
    W, K = args.warmup, args.steps
    cells = prepare_oracle(s * (W + K))
    P = oracle_procs(cells)
    value, el = oracle_replicas(P, s * W, s * K)
    value /= 1e9
    _ORACLE.clear()
    sample = (f"each step = {s} time step of the full 4096x4096 grid with its 8 models in each of {P} "
              f"forked processes (one per usable host core, independent replicas), FP64 numpy")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": K, "warmup": W, "ms_per_step": el / K * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": dict(CONFIG, parallelism="single"),
        "time_steps_per_step": s, "replicas": P,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": P, "kind": "oracle", "sample": sample,
                         "host": {"usable_cores": _usable_cores(), "cpu": host_cpu()}},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


# ---------------------------------------------------------------- GPU parts

def measure_batched(K, W, T, plain_per_size=16, per_size=64):
    """Batched vs plain: 256 simulations (64 each of 128^2, 256^2, 512^2,
    1024^2) sharing four reduced models, advanced together in one launch per
    step (K timed steps of T time steps), against simulations run one context
    and one fdtd_run at a time (plain_per_size of each size, each timed over
    Tp graph-replayed steps; the plain rate is cells x steps over the summed
    times of those runs, which stand for all 64 of their size)."""
    import numpy as np
    import torch
    import paper_1609_07114_gb300 as pg
    import workloads
    Tp = max(T // 5, 32)
    w = workloads.batched_256(max((W + K) * T, 2 * Tp), per_size=per_size)
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
        if k == 0:   # tuned with the run's sources and probes in place
            tune = autotune(ctx)
    spl = ctx.steps_per_launch()
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
    kms = ctx.time_stencil(8, 4)
    ctx.close()
    # plain: one context and one fdtd_run at a time
    el_p, cells_p = 0.0, 0
    outp = torch.zeros((Tp, 1), dtype=torch.float32, device="cuda")
    by_size = {}
    for s in sims:
        by_size.setdefault(s["nx"], []).append(s)
    for group in by_size.values():
        for s in group[:plain_per_size]:
            c1, wv, pr = make_ctx([s])
            step(c1, [s], wv, pr, 0, Tp, outp)              # warm (the run's sources and probes in place)
            autotune(c1)                                    # the first of each size is timed, the rest cached
            step(c1, [s], wv, pr, 0, Tp, outp)              # warm (graph capture)
            torch.cuda.synchronize()
            e0.record(stream)
            step(c1, [s], wv, pr, Tp, Tp, outp)
            e1.record(stream)
            torch.cuda.synchronize()
            el_p += e0.elapsed_time(e1) / 1e3
            cells_p += s["nx"] * s["ny"]
            c1.close()
    plain = cells_p * Tp / el_p / 1e9
    return {
        "metric": "batched " + METRIC, "value": batched, "unit": UNIT, "steps": K, "warmup": W,
        "ms_per_step": el_b / K * 1e3, "time_steps_per_step": T, "higher_is_better": True,
        "workload": f"batched_256: {per_size} each of 128^2, 256^2, 512^2, 1024^2 coarse grids, 4 shared ROMs "
                    "r=3 q=40/80/160/320, every simulation in each launch",
        "cells": cells, "plain_value": plain, "batched_over_plain": batched / plain,
        "plain": f"{plain_per_size} simulations of each size, each alone in its own autotuned context, {Tp} "
                 f"time steps per run (graph-replayed after a warm run of {Tp})",
        "tune": tune,
        "roofline": roofline(BYTES_PER_CELL_STEP * cells, kms, "yee_tb2m_kernel" if spl == 2 else "yee_step_kernel",
                             spl, batched),
        "gpu_launches": K * launches_per_run(T, spl, 4 * len(sims), tune["chained_models"]),
        "clocks": clk.summary()}


def measure_adjoint(K, W, N, nsim=16):
    """Adjoint/forward time ratio: nsim simulations of 1024^2 cells with two
    shared q = 120 models each, J = sum of Hz^2 at 8 probes per simulation
    over N steps, checkpoints every 500 steps; W untimed and K timed
    repetitions of one forward run and one gradient run (medians)."""
    import numpy as np
    import torch
    import paper_1609_07114_gb300 as pg
    import workloads
    w = workloads.adjoint_16(N, nsim=nsim)
    models = [pg.rom_build(md["a"], md["b"], md["r"], w["dx"], w["dy"], w["dt"], md["eps_r"],
                           md["sigma"], md["q"], f0=md["f0"]) for md in w["models"]]

    tunes = []

    def make_ctx():
        ctx = pg.FdtdContext(w["dx"], w["dy"], w["dt"], [(s["eps_r"], s["sigma"]) for s in w["sims"]])
        for k, s in enumerate(w["sims"]):
            for (mi, i0, j0) in s["place"]:
                ctx.rom_embed(models[mi], k, i0, j0)
        tunes.append(autotune(ctx))
        return ctx

    waves = [torch.tensor(s["source"]["wave"].astype(np.float32), device="cuda") for s in w["sims"]]
    src = [dict(s["source"], sim=k, wave=waves[k]) for k, s in enumerate(w["sims"])]
    probes = [(k, i, j) for k, s in enumerate(w["sims"]) for (i, j) in s["probes"]]
    cells = sum(s["nx"] * s["ny"] for s in w["sims"])
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fwd, adj = [], []
    out = torch.zeros((N, len(probes)), dtype=torch.float32, device="cuda")
    J = None
    with ClockSampler() as clk:
        for rep in range(W + K):
            ctx = make_ctx()
            torch.cuda.synchronize()
            e0.record(stream)
            ctx.fdtd_run(N, src, probes, out)
            e1.record(stream)
            torch.cuda.synchronize()
            tf = e0.elapsed_time(e1) / 1e3
            spl = ctx.steps_per_launch()
            ctx.close()
            ctx = make_ctx()
            torch.cuda.synchronize()
            e0.record(stream)
            J, ge, gs, gw = ctx.fdtd_grad(N, src, probes, 500)
            e1.record(stream)
            torch.cuda.synchronize()
            ta = e0.elapsed_time(e1) / 1e3
            ctx.close()
            if rep >= W:
                fwd.append(tf)
                adj.append(ta)
    tf, ta = float(np.median(fwd)), float(np.median(adj))
    return {
        "metric": "adjoint/forward time ratio", "value": ta / tf, "unit": "x", "steps": K, "warmup": W,
        "higher_is_better": False,
        "workload": f"adjoint_16: {nsim} x 1024^2 coarse grids, 2 shared ROMs r=3 q=120 each, 8 probes per "
                    "simulation, J = sum Hz^2, checkpoints every 500 steps",
        "time_steps": N, "cells": cells, "forward_s": tf, "gradient_s": ta, "forward_steps_per_launch": spl,
        "forward_gcell_steps_per_s": cells * N / tf / 1e9,
        "gradient_gcell_steps_per_s": cells * N / ta / 1e9, "J": J, "tune": tunes[0], "clocks": clk.summary()}


def measure_lattice(K, W, T, n=8192, lossless=False, energy_every=0):
    """Many heterogeneous models with CFL extension: an n^2 vacuum grid with
    1% lossy scatterers, 64 embedded models of three types (r = 5, q =
    60/180/400) at dt = 2 x the fine-mesh CFL limit, four full-column line
    sources, 16 probes; K timed steps of T time steps.  lossless: the
    sigma = 0 variant; energy_every E: the storage function every E steps over
    (W + K) T steps, with its drift after the pulse has left the sources."""
    import numpy as np
    import torch
    import paper_1609_07114_gb300 as pg
    import workloads
    total = (W + K) * T
    w = workloads.lattice_8192(min(total, 20000), n=n, pitch=n // 8, lossless=lossless)
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
    if energy_every:
        tune = autotune(ctx)
        E = energy_every
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
            if k == 0:   # tuned with the run's sources and probes in place
                tune = autotune(ctx)
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
    spl = ctx.steps_per_launch()
    kms = ctx.time_stencil(8, 4)
    f_nb = float(np.mean((w["eps_r"] != 1.0) | (w["sigma"] != 0.0)))
    # per launch (one or two steps): the fields and the materials of the
    # non-background cells (both kernels skip background-only strip rows)
    bpc = 24.0 + 8.0 * f_nb
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "steps": K, "warmup": W,
        "ms_per_step": el_s / max(nsteps_timed // T, 1) * 1e3, "time_steps_per_step": T,
        "higher_is_better": True,
        "workload": f"lattice_{n}: {n}^2 vacuum grid, {100 * f_nb:.2f}% "
                    f"{'lossless' if lossless else 'lossy'} scatterer cells, 64 ROMs of 3 "
                    "types (r=5, q=60/180/400) at dt=2x fine CFL, 4 full-column Jy line sources, 16 Hz probes",
        "nx": w["nx"], "ny": w["ny"], "roms": len(w["roms"]),
        "rom_q": sorted({m.q for m in built.values()}),
        "rom_clamped": [m.report.n_clamped for m in built.values()],
        "rom_build_s": round(rom_seconds, 3), "rom_build_gpu_s": round(rom_gpu_seconds, 3), "tune": tune,
        "l2": f"inputs larger than L2: {24 * n * n / 1e9:.2f} GB of fields per time step (L2 129 MB)",
        "roofline": roofline(bpc * cells, kms, "yee_tb2m_kernel" if spl == 2 else "yee_step_kernel", spl,
                             value, bpc=24.0 + 8.0 * f_nb),
        "gpu_launches": (nsteps_timed // T) * launches_per_run(T, spl, len(w["roms"]), tune["chained_models"]),
        "clocks": clk.summary(),
    }
    if energy:
        E = energy_every
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
    ctx.close()
    return line


def measure_grid(args, ws, rank, local, dist):
    """The headline: K timed steps of T time steps of the 4096^2 workload
    (per rank), then the stencil kernel alone and the host-buffer run."""
    import numpy as np
    import torch
    import paper_1609_07114_gb300 as pg

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
        if k == 0:   # tuned with the run's sources and probes in place
            t0 = time.perf_counter()
            tune = autotune(ctx)
            tune["seconds"] = round(time.perf_counter() - t0, 3)
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

    # The stencil kernel alone (graph replay, no per-kernel events).  On the
    # two-steps-per-launch path a launch is one read and one write pass over
    # the fields and materials for two steps: 32 B per cell per launch.
    spl = ctx.steps_per_launch()
    kernel = "yee_tb2m_kernel" if spl == 2 else "yee_step_kernel"
    kms = ctx.time_stencil(16, 8)
    alg_bytes = BYTES_PER_CELL_STEP * cells

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

    cfg = dict(CONFIG) if args.grid == 4096 else {"workload": f"grid {args.grid}^2, same recipe"}
    cfg["parallelism"] = "replicas" if ws > 1 else "single"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W,
        "ms_per_step": el_ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
        "time_steps_per_step": T, "rom_build_s": round(rom_seconds, 3), "tune": tune,
        "roofline": roofline(alg_bytes, kms, kernel, spl, value, traffic=profile_traffic(kernel)),
        "e2e": e2e,
        "gpu_launches": K * launches_per_run(T, spl, len(models), tune["chained_models"]),
        "clocks": clk.summary(),
    }
    ctx.close()
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tsteps", type=int, default=2000, help="time steps per benchmark step")
    ap.add_argument("--cpu-sample-steps", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--headline-only", action="store_true",
                    help="the 4096^2 line without the batched, adjoint and lattice records")
    ap.add_argument("--grid", type=int, default=4096, help="coarse grid size (4096 = the benchmark)")
    ap.add_argument("--workload", default="grid", choices=["grid", "batched", "adjoint", "lattice"])
    ap.add_argument("--lossless", action="store_true", help="lattice: sigma = 0 everywhere")
    ap.add_argument("--adj-nsim", type=int, default=16,
                    help="adjoint: simulations in the batch (16 = the configuration)")
    ap.add_argument("--lattice-n", type=int, default=8192,
                    help="lattice: grid size (8192 = the configuration; 64 models at pitch n/8)")
    ap.add_argument("--energy-every", type=int, default=0,
                    help="lattice: record the storage function every E steps")
    ap.add_argument("--plain-per-size", type=int, default=16,
                    help="batched: simulations of each size run one at a time for the plain rate")
    ap.add_argument("--batch-per-size", type=int, default=64,
                    help="batched: simulations of each size in the batch (64 = the configuration)")
    ap.add_argument("--no-tune", action="store_true", help="the fixed rule instead of the autotuner's choice")
    args = ap.parse_args()
    TUNE[0] = not args.no_tune
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return
    ws, rank, local = dist_env()
    single = args.workload != "grid"
    if single:
        import torch
        from paper_1609_07114_gb300 import build as pbuild
        pbuild.build()
        torch.cuda.set_device(local)
        if args.workload == "adjoint":
            K = 3 if args.steps == 10 else args.steps
            W = 1 if args.warmup == 3 else args.warmup
            N = args.tsteps if args.tsteps != 2000 else 10000
            line = measure_adjoint(K, W, N, args.adj_nsim)
        elif args.workload == "lattice":
            T = 1000 if args.tsteps == 2000 else args.tsteps   # 10 timed steps = the configuration's 10000
            line = measure_lattice(args.steps, args.warmup, T, args.lattice_n, args.lossless, args.energy_every)
        else:
            T = 500 if args.tsteps == 2000 else args.tsteps    # 10 timed steps = the batch's 5000
            line = measure_batched(args.steps, args.warmup, T, args.plain_per_size, args.batch_per_size)
        line.update({"n_gpus": 1, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic"})
        print(json.dumps(line))
        return

    # The CPU oracle first: its processes are forked, so before any CUDA call.
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_sample_steps)

    import torch
    from paper_1609_07114_gb300 import build as pbuild
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        pbuild.build()
    if dist:
        dist.barrier()
    line = measure_grid(args, ws, rank, local, dist)
    line["cpu_baseline"] = cpu
    if ws == 1 and not args.headline_only and args.grid == 4096:
        # the other parts of the metric, each on its own workload and timed region
        line["batched"] = measure_batched(4, 3, 500, args.plain_per_size)
        line["adjoint"] = measure_adjoint(2, 1, 10000, 16)
        line["lattice"] = measure_lattice(5, 3, 1000)
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
