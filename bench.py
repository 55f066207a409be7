"""Throughput of the CRBM proposal + Metropolis-Hastings step on GB300.

Default workload ("ising-batch"): 2D Ising, L in {16, 32, 64, 128}, 4096 chains
per L over 32 temperatures in [1.5, 3.5], CRBM with K = 4 filters 5 x 5, all
four lattice sizes in ONE batched launch; mixed precision (FP32 with certified
margins and FP64 recompute).  One bench step = one launch running S_STEP
proposals of every chain.  value = chain-proposals per second over all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload ising-batch|ising-small|kitaev-small] [--precision mixed|fp64]

--impl reference times the CPU oracle (the plain FP64 numpy restatement of
the method) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import crbm_workloads as wl  # noqa: E402

METRIC = "CRBM-MH proposals/s (Ising, Kitaev) vs plain FP64 path; serving p50/p99 latency"
SEED = wl.BASE_SEED


def workload(name):
    """(kind, [(L, n_chains)], T-ladder fn, J, model params, S_STEP, description)."""
    if name == "ising-batch":
        W, hb, vb = _ising_batch_model()
        return dict(kind=0, jobs=[(L, 4096) for L in (16, 32, 64, 128)], T=lambda n: wl.ising_ladder(n, 32),
                    J=(1.0,), model=(W, hb, vb), S=10,
                    desc="2D Ising L in {16,32,64,128} x 4096 chains, 32 T in [1.5,3.5], K=4 5x5 CRBM")
    if name == "ising-small":
        W, hb, vb = wl.gaussian_crbm(2, 3, 0.1)
        return dict(kind=0, jobs=[(8, 16)], T=lambda n: np.full(n, 2.269), J=(1.0,), model=(W, hb, vb), S=100,
                    desc="2D Ising L=8, 16 chains, T=2.269, K=2 3x3 CRBM N(0,0.1)")
    if name == "kitaev-small":
        W, hb, vb = wl.gaussian_crbm(4, 3, 0.05)
        return dict(kind=1, jobs=[(6, 1024)], T=lambda n: wl.kitaev_ladder(n, 24), J=(1.0, 1.0, 1.0),
                    model=(W, hb, vb), S=2,
                    desc="Kitaev L=6 (72 sites), J=1, 1024 chains, 24 T log-spaced in [0.005,1], K=4 3x3 CRBM")
    if name == "kitaev-batch":
        W, hb, vb = wl.gaussian_crbm(4, 3, 0.05)
        return dict(kind=1, jobs=[(8, 683), (10, 683), (12, 682)], T=lambda n: wl.kitaev_ladder(n, 24),
                    J=(1.0, 1.0, 1.0), model=(W, hb, vb), S=1,
                    desc="Kitaev L in {8,10,12} (2048 chains split by L) in one launch, 24 T log-spaced "
                         "in [0.005,1], K=4 3x3 CRBM")
    raise SystemExit(f"unknown workload {name}")


def _ising_batch_model():
    path = os.path.join(ROOT, "paper_2008_05401_gb300", "data", "ising_cd1_L16_K4_k5.npz")
    if os.path.exists(path):
        d = np.load(path)
        return d["W"], d["hb"], float(d["vb"])
    return wl.gaussian_crbm(4, 5, 0.1)


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p:
            time.sleep(0.25)
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# FP32 / FP64 FMA peaks measured on this device by the library's probe (filled in main)
PROBED = {"fp32": None, "fp64": None}


def fp64_peak():
    """(TFLOP/s, source) of the FP64 pipe: the probe's measurement, else GB300's nominal figure."""
    if PROBED["fp64"]:
        return PROBED["fp64"], "measured FP64 FMA probe (crbm_probe_peaks)"
    return 1.25, "nominal GB300 FP64"


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


# DRAM bytes (read + write) of one full-size launch of the persistent
# tensor-core kernel on the batch Ising workload (the timed step after three
# warm-up steps, L2 flushed before it), from an ncu capture: 14,549,248 B read,
# 60,416 B written (the lattices and state written back stay in the 129 MB L2
# until after the launch).
BATCH_ISING_TC_TRAFFIC_BYTES = 14_549_248 + 60_416


def _sm_mhz(clocks):
    return (clocks or {}).get("sm_mhz") or peaks().get("clocks_under_load", {}).get("sm_mhz_median") or 1462.0


def roofline(kernel_ms, clocks, K, k, n_sites, traffic=None):
    """ALU roofline of an Ising proposal kernel with the algorithmic count of
    the method: per site and proposal the hidden and visible convolutions,
    2 K k^2 multiply-adds = 4 K k^2 flops (400 at K = 4, k = 5; the free
    energy's pre-activations are the next proposal's hidden ones when v' is
    kept, so a proposal needs two convolution passes), against the FP32 FMA
    peak from unit counts (152 SMs x 128 lanes x 2 flops) at the SM clock
    sampled during the run.  The other pipes the method needs bound it no
    tighter: (4K + 2) special-function operations per site at 16 per SM and
    clock, and (K + 1) / 4 Philox blocks of about 80 integer operations at 64
    per SM and clock (the same 1.56 clocks per site as the FMA count).  The
    kernels compute all three convolutions (the F pass recomputed, 6 K k^2
    flops per site): that executed count is reported beside, labelled."""
    mhz = _sm_mhz(clocks)
    peak = 152 * 128 * 2 * mhz * 1e6 / 1e12
    flops = 4.0 * K * k * k * n_sites
    achieved = flops / (kernel_ms * 1e-3) / 1e12
    executed = 6.0 * K * k * k * n_sites / (kernel_ms * 1e-3) / 1e12
    clk_site = {"fma": 2 * K * k * k / 128.0, "sfu": (4 * K + 2) / 16.0, "int_philox": (K + 1) / 4.0 * 80 / 64.0}
    return {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 3), "unit": "TFLOP/s",
            "frac": round(achieved / peak, 4), "traffic": traffic,
            "peak_source": f"FP32 FMA from unit counts x sampled SM clock {mhz:.0f} MHz",
            "algorithmic_flops_per_site": 4 * K * k * k,
            "pipe_clk_per_site_per_sm": clk_site,
            "measured_clk_per_site_per_sm": round(kernel_ms * 1e-3 * mhz * 1e6 * 152 / n_sites, 3),
            "executed_3pass": {"flops_per_site": 6 * K * k * k, "achieved": round(executed, 3),
                               "frac": round(executed / peak, 4),
                               "note": "direct-FP32-equivalent of the three convolutions the kernel computes"}}


# FP32 instructions of one double-FP32 multiply-add with one normalisation
# (df_fma: two_prod 2, two cross-term FMAs and an add, two_sum 6, an add,
# fast_two_sum 3; the rank-2 update's a - (x1 y1 + x2 y2) takes 27 for two):
# the mixed Kitaev path emulates each FP64 multiply-add of the reduction with
# them on the FP32 pipe
DF64_FP32_OPS_PER_FMA = 15


def kitaev_roofline(spec, ms, steps, prec, clocks):
    """Eigen-stage roofline with the survey's algorithmic count, (8/3) N^3
    flops per proposal ((4/3) N^3 multiply-adds: a Golub-Kahan
    bidiagonalisation of M, values only).  FP64 path: against the FP64 FMA
    peak the library's probe measures.  Mixed path: those multiply-adds run as
    double-FP32 on the FP32 pipe, 15 FP32 instructions each, against the FP32
    pipe's instruction rate from unit counts (152 SMs x 128 lanes) at the
    sampled SM clock."""
    fmas = sum(n * (4.0 / 3.0) * (L * L) ** 3 for L, n in spec["jobs"]) * spec["S"] * steps
    if prec == 0:
        pk, src = fp64_peak()
        achieved = 2 * fmas / (ms * 1e-3) / 1e12
        return {"bound": "fp64", "achieved": round(achieved, 4), "peak": round(pk, 4), "unit": "TFLOP/s",
                "frac": round(achieved / pk, 4), "traffic": None,
                "peak_source": src + "; flops = (8/3) N^3 per proposal"}
    mhz = _sm_mhz(clocks)
    peak = 152 * 128 * mhz * 1e6 / 1e12                     # FP32 instructions per second, 1e12
    achieved = fmas * DF64_FP32_OPS_PER_FMA / (ms * 1e-3) / 1e12
    return {"bound": "alu", "achieved": round(achieved, 4), "peak": round(peak, 4), "unit": "TFP32-inst/s",
            "frac": round(achieved / peak, 4), "traffic": None,
            "peak_source": f"FP32 pipe from unit counts x SM clock {mhz:.0f} MHz; (4/3) N^3 FP64 multiply-adds "
                           f"per proposal x {DF64_FP32_OPS_PER_FMA} FP32 instructions each (double-FP32)"}


def _oracle_worker(args):
    """One process of the all-core oracle timing: `chains` chains of side L
    (chain ids from `base`) step for about budget_s seconds."""
    name, L, base, chains, budget_s = args
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    from oracle import chain
    spec = workload(name)
    W, hb, vb = spec["model"]
    ch = chain.make_chains(spec["kind"], W, hb, vb, L, spec["T"](base + chains)[base:], spec["J"], SEED,
                           np.arange(base, base + chains))
    t0 = time.perf_counter()
    s = 0
    while s == 0 or time.perf_counter() - t0 < budget_s:
        chain.step(ch)
        s += 1
    return chains * s, time.perf_counter() - t0


def cpu_baseline_run(spec, name, budget_s=15.0, cores=None):
    """The oracle (numpy FP64, one BLAS thread per process) on a bounded sample
    of the workload: for every lattice size of the mix, `cores` processes
    (spawned: no fork of a process that holds a CUDA context) each step their
    own chains for about budget_s / n_sizes seconds; the per-size rates give
    the proposals/s of the workload's mix (its chains per L).  cores = 1 gives
    the single-core figure."""
    import multiprocessing as mp
    cores = cores or os.cpu_count() or 1
    per = 64 if spec["kind"] == 0 else 32
    sizes = spec["jobs"]
    t_each = budget_s / len(sizes)
    tasks = [(name, L, w * per, per, t_each) for L, _ in sizes for w in range(cores)]
    if cores == 1:
        res = [_oracle_worker(t) for t in tasks]
    else:
        with mp.get_context("spawn").Pool(cores) as pool:
            res = pool.map(_oracle_worker, tasks, chunksize=1)
    secs_per_mix, samples = 0.0, []
    for i, (L, n) in enumerate(sizes):
        part = res[i * cores:(i + 1) * cores]
        props = sum(p for p, _ in part)
        dt = max(t for _, t in part)
        secs_per_mix += n / (props / dt)          # time for this size's share of one mix proposal round
        samples.append(f"L={L}: {cores} x {per} chains, {props} proposals in {dt:.1f}s")
    rate = sum(n for _, n in sizes) / secs_per_mix
    return {"value": rate, "unit": "proposals/s", "cores": cores, "kind": "oracle",
            "sample": "; ".join(samples) + " (rates combined over the workload's chains per L)"}


def bench_config(spec, args, world):
    """The workload description shared by both arms' JSON lines."""
    return {"workload": spec["desc"], "proposals_per_step": spec["S"], "chains": sum(n for _, n in spec["jobs"]),
            "precision": args.precision, "l2": "flushed between timed steps (256 MiB write)",
            "parallelism": f"chains x{world}"}


def run_reference(args, spec):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cb = cpu_baseline_run(spec, args.workload, budget_s=max(8.0, 1.0 * args.steps))
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "proposals/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(spec, args, world), "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "proposals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_jobs(ctx, jobs, S, prec, steps, warmup, stream, dev, flush, graph=False):
    """Device time (ms) of `steps` batched launches (or, with graph, replays of
    one captured batched run), L2 flushed before each."""
    import torch
    g = ctx.graph(jobs, S, precision=prec) if graph else None
    step = (lambda: g.launch(stream)) if graph else (lambda: ctx.run_batch(jobs, S, precision=prec, stream=stream))
    for _ in range(warmup):
        step()
    torch.cuda.synchronize(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    if g is not None:
        g.destroy()
    return sum(a.elapsed_time(b) for a, b in ev)


def secondary(ctx_cls, name, prec, steps, dev, stream, flush, graph=False, clocks=None, tune=None):
    """Proposals/s of another workload or precision (no e2e, no clocks); graph:
    replay a captured CUDA graph of the batched run; tune (default: with the
    graph): autotuned tiles first."""
    from paper_2008_05401_gb300 import MIXED
    spec = workload(name)
    ctx = ctx_cls(dev)
    W, hb, vb = spec["model"]
    mid = ctx.load_model(spec["kind"], W, vb, hb)
    jobs, base = [], 0
    for L, n in spec["jobs"]:
        jobs.append(ctx.new_job(mid, spec["kind"], L, spec["T"](n), spec["J"], SEED, base,
                                wl.pack_bits(wl.random_lattices(n, L, seed=SEED + L)), prec))
        base += n
    if graph if tune is None else tune:
        for L, _ in spec["jobs"]:
            ctx.tune(mid, L, prec)            # autotuned tiles (Kitaev: chains, i.e. thread groups, per CTA)
    ms = time_jobs(ctx, jobs, spec["S"], prec, steps, 1, stream, dev, flush, graph=graph)
    n_chains = sum(n for _, n in spec["jobs"])
    sums = [j.observables() for j in jobs]
    acc = sum(int(a.sum()) for _, a, _ in sums) / (n_chains * spec["S"] * (steps + 1))
    rec = [sum(int(r[:, 0].sum()) for _, _, r in sums), sum(int(r[:, 1].sum()) for _, _, r in sums)]
    ctx.close()
    out = {"workload": spec["desc"] + (", captured CUDA graph replayed" if graph else ""),
           "precision": "mixed" if prec == MIXED else "fp64",
           "value": n_chains * spec["S"] * steps / (ms * 1e-3), "unit": "proposals/s",
           "ms_per_step": ms / steps, "proposals_per_step": spec["S"], "acceptance": acc,
           "fp64_recomputes": rec}
    if spec["kind"] == 1:
        out["roofline"] = kitaev_roofline(spec, ms, steps, prec, clocks)
    return out


def _oracle_rate(fn, budget_s):
    """Calls of fn() per second over about budget_s seconds (at least one call), one BLAS thread."""
    try:
        from threadpoolctl import threadpool_limits
        lim = threadpool_limits(1)
    except Exception:  # noqa: BLE001
        lim = None
    t0, n = time.perf_counter(), 0
    while n == 0 or time.perf_counter() - t0 < budget_s:
        fn()
        n += 1
    dt = time.perf_counter() - t0
    if lim is not None and hasattr(lim, "unregister"):
        lim.unregister()
    return n / dt, n, dt


def tempering_run(ctx_cls, name, prec, cycles, dev, stream, flush, oracle_s=3.0, clocks=None, g=1, L_n=None):
    """Parallel-tempering exchange correction (App. B.2) on a workload's first
    lattice size (or L_n = (L, chains)): the workload's chains are the physical
    ladder, as many RBM chains run beside them.  value = chain-cycles/s (one RBM
    proposal of g Gibbs steps, one swap decision and one temperature-exchange
    decision per pair and cycle)."""
    import torch
    from paper_2008_05401_gb300 import MIXED
    spec = workload(name)
    L, n = L_n or spec["jobs"][0]
    ctx = ctx_cls(dev)
    W, hb, vb = spec["model"]
    mid = ctx.load_model(spec["kind"], W, vb, hb)
    T = spec["T"](n)
    x = ctx.new_job(mid, spec["kind"], L, T, spec["J"], SEED, 0,
                    wl.pack_bits(wl.random_lattices(n, L, seed=SEED + L)), prec)
    y = ctx.new_job(mid, spec["kind"], L, T, spec["J"], SEED + 1, n,
                    wl.pack_bits(wl.random_lattices(n, L, seed=SEED + L + 1)), prec)
    ctx.pt_run(x, y, 2, g=g, precision=prec, stream=stream)
    torch.cuda.synchronize(dev)
    flush.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.pt_run(x, y, cycles, g=g, precision=prec, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    _, acc, _ = x.observables()
    ctx.close()
    model = "2D Ising" if spec["kind"] == 0 else "Kitaev"
    out = {"workload": f"parallel tempering, {model} L={L}, {n} physical + {n} RBM chains, one proposal "
                       f"(g={g}) per RBM chain and cycle, the workload's T ladder",
           "precision": "mixed" if prec == MIXED else "fp64", "value": n * cycles / (ms * 1e-3),
           "unit": "chain-cycles/s", "ms_per_cycle": ms / cycles, "cycles": cycles,
           "swap_rate": float(acc.sum()) / (n * (cycles + 2))}
    if spec["kind"] == 0:
        # the RBM proposal (mode-2 kernel) dominates: the headline's conv-flop count per site
        K, k = W.shape[0], W.shape[1]
        out["roofline"] = roofline(ms / cycles, clocks or {}, K, k, n * L * L)
    if oracle_s > 0:
        from oracle import chain, tempering
        nc = 32
        px = chain.make_chains(spec["kind"], W, hb, vb, L, T[:nc], spec["J"], SEED, np.arange(nc))
        py = chain.make_chains(spec["kind"], W, hb, vb, L, T[:nc], spec["J"], SEED + 1, np.arange(nc, 2 * nc))
        rate, c, dt = _oracle_rate(lambda: tempering.cycle(px, py, g), oracle_s)
        out["cpu_baseline"] = {"value": rate * nc, "unit": "chain-cycles/s", "cores": 1, "kind": "oracle",
                               "sample": f"{nc} + {nc} chains x {c} cycles in {dt:.1f}s"}
    return out


def tau_run(ctx_cls, L, n, T, steps, dev, stream, warm=200, oracle_s=2.0):
    """The paper's sampler comparison (Sec. III): integrated autocorrelation
    time of the energy for CRBM proposals (the batch workload's CD-1 filters,
    mixed precision, MH-corrected) and for checkerboard single-spin Metropolis
    sweeps, from E traces of `steps` steps of n chains at one temperature;
    tau from crbm_autocorr (mean over chains), time per step from CUDA events."""
    import torch
    from paper_2008_05401_gb300 import FP64, ISING, MIXED
    W, hb, vb = _ising_batch_model()
    ctx = ctx_cls(dev)
    mid = ctx.load_model(ISING, W, vb, hb)
    out = {"workload": f"2D Ising L={L}, {n} chains, T={T}, E traces of {steps} steps after {warm} of warm-up"}
    for name, prec in (("crbm", MIXED), ("metropolis", FP64)):
        job = ctx.new_job(mid, ISING, L, np.full(n, T), (1.0,), SEED, 0,
                          wl.pack_bits(wl.random_lattices(n, L, seed=SEED + L)), prec)
        step = (lambda k: job.run(k, precision=MIXED, stream=stream)) if name == "crbm" else \
            (lambda k: job.local_run(k, stream=stream))
        step(warm)
        torch.cuda.synchronize(dev)
        buf = job.set_trace(steps)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(steps)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        tau, win = ctx.autocorr(buf, stream=stream)
        _, acc, _ = job.observables()
        t = float(np.mean(tau))
        out[name] = {"tau_E_steps": t, "tau_E_median": float(np.median(tau)), "window_median": int(np.median(win)),
                     "ms_per_step": ms, "independent_samples_per_s": n / (2.0 * t * ms * 1e-3),
                     "acceptance": float(acc.sum()) / (n * (steps + warm) * (1 if name == "crbm" else L * L))}
        job.set_trace(None)
        job.release()
    ctx.close()
    out["crbm_over_metropolis_independent_samples"] = (out["crbm"]["independent_samples_per_s"]
                                                       / out["metropolis"]["independent_samples_per_s"])
    out["metropolis"]["chain_sweeps_per_s"] = n / (out["metropolis"]["ms_per_step"] * 1e-3)
    if oracle_s > 0:
        from oracle import chain, metropolis
        nc = 64
        och = chain.make_chains(chain.ISING, W, hb, vb, L, np.full(nc, T), (1.0,), SEED, np.arange(nc))
        rate, c, dt = _oracle_rate(lambda: metropolis.sweep(och), oracle_s)
        out["metropolis"]["cpu_baseline"] = {"value": rate * nc, "unit": "chain-sweeps/s", "cores": 1,
                                             "kind": "oracle", "sample": f"{nc} chains x {c} sweeps in {dt:.1f}s"}
    return out


def train_run(ctx_cls, dev, stream, n_problems=24, L=8, K=2, k=5, n=10_000, batch=20, oracle_s=2.0):
    """The paper's trainer (Algorithm 1's epoch, App. D sizes): one CRBM of
    K x k x k filters per temperature, n samples of L x L each, minibatches of
    `batch`, ADAM; one epoch of all problems is one launch.  value = sample
    gradients/s; flops counted as a direct forward and weight-gradient
    convolution, 4 K k^2 L^2 per sample."""
    import torch
    from paper_2008_05401_gb300 import FP64, ISING, trainer
    ctx = ctx_cls(dev)
    mid = ctx.load_model(ISING, np.zeros((K, k, k)), 0.0, np.zeros(K))
    probs, xs, ts, os_ = [], [], [], []
    for i in range(n_problems):
        bits = wl.pack_bits(wl.random_lattices(n, L, seed=SEED + i))
        job = ctx.new_job(mid, ISING, L, np.full(n, 1.5 + i * 0.05), (1.0,), SEED, 0, bits, FP64)
        lp, _, _ = job.energies()
        job.release()
        xs.append(torch.tensor(bits.view(np.int32), device=f"cuda:{dev}"))
        ts.append(torch.tensor(-lp, device=f"cuda:{dev}"))
        os_.append(torch.tensor(wl.epoch_order(n, SEED, i), device=f"cuda:{dev}"))
        probs.append(trainer.Problem.new(ctx, K, k, L, wl.init_train_params(K, k, seed=SEED + i)))
    trainer.train_epochs(ctx, probs, xs, ts, os_, batch, stream=stream)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    losses = trainer.train_epochs(ctx, probs, xs, ts, os_, batch, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    ctx.close()
    flops = 4.0 * K * k * k * L * L * n * n_problems
    achieved = flops / (ms * 1e-3) / 1e12
    out = {"workload": f"trainer epoch: {n_problems} problems (one per temperature), K={K} {k}x{k} filters, "
                       f"L={L}, {n} samples each, minibatch {batch}, ADAM, FP64",
           "value": n * n_problems / (ms * 1e-3), "unit": "sample-gradients/s", "ms_per_epoch": ms,
           "adam_steps_per_s": n_problems * ((n + batch - 1) // batch) / (ms * 1e-3),
           "mean_loss_epoch2": float(np.mean([float(x.mean()) for x in losses])),
           "roofline": {"bound": "fp64", "achieved": round(achieved, 4), "peak": round(fp64_peak()[0], 4),
                        "unit": "TFLOP/s", "frac": round(achieved / fp64_peak()[0], 4), "traffic": None,
                        "peak_source": fp64_peak()[1] + "; flops = direct forward + weight-gradient "
                                                        "convolutions, 4 K k^2 L^2 per sample"}}
    if oracle_s > 0:
        from oracle import train
        v = wl.random_lattices(2000, L, seed=SEED)
        tt = np.random.default_rng(1).normal(size=2000)
        st = train.Adam.zeros(K * k * k + 1 + K)
        th = wl.init_train_params(K, k)
        rate, c, dt = _oracle_rate(lambda: train.epoch(th, st, v, tt, np.arange(2000), K, k, M=batch), oracle_s)
        out["cpu_baseline"] = {"value": rate * 2000, "unit": "sample-gradients/s", "cores": 1, "kind": "oracle",
                               "sample": f"{c} epochs of 2000 samples in {dt:.1f}s"}
    return out


def lcrbm_run(ctx_cls, dev, stream, L=8, n=1024, S=2, edge=3, K=2, k=5, oracle_s=2.0):
    """Open-boundary Kitaev model with the locally connected CRBM (Sec. IV):
    the paper's three unshared edge kernels per side and 2x5x5 kernels, the
    small Kitaev workload's temperature ladder, FP64 (the LCRBM's only
    precision).  value = proposals/s."""
    import torch
    from paper_2008_05401_gb300 import FP64, KITAEV
    g = wl.rng(SEED + 4)
    W = g.normal(0.0, 0.05, (2 * edge + 1, K, k, k))
    hb, vb = g.normal(0.0, 0.05, K), float(g.normal(0.0, 0.05))
    T = wl.kitaev_ladder(n, 24)
    bits = wl.pack_bits(wl.random_lattices(n, L, seed=SEED + L))
    ctx = ctx_cls(dev)
    mid = ctx.load_lcrbm(KITAEV, W, vb, hb)
    job = ctx.new_job(mid, KITAEV, L, T, (1.0, 1.0, 1.0), SEED, 0, bits, FP64)
    job.run(1, precision=FP64, stream=stream)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    job.run(S, precision=FP64, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    _, acc, _ = job.observables()
    ctx.close()
    out = {"workload": f"open-boundary Kitaev L={L} with an LCRBM ({edge} edge kernels per side, K={K} "
                       f"{k}x{k}), {n} chains, 24 T log-spaced in [0.005,1]",
           "precision": "fp64", "value": n * S / (ms * 1e-3), "unit": "proposals/s", "ms_per_step": ms,
           "acceptance": float(acc.sum()) / (n * (S + 1))}
    if oracle_s > 0:
        from oracle import chain
        nc = 16
        och = chain.make_chains(chain.KITAEV, W, hb, vb, L, T[:nc], (1.0, 1.0, 1.0), SEED, np.arange(nc),
                                edge=edge)
        rate, c, dt = _oracle_rate(lambda: chain.step(och), oracle_s)
        out["cpu_baseline"] = {"value": rate * nc, "unit": "proposals/s", "cores": 1, "kind": "oracle",
                               "sample": f"{nc} chains x {c} proposals in {dt:.1f}s"}
    return out


def serving_run(dev, n=32, rate=200.0, max_proposals=10_000):
    """Continuous batching of a Poisson request stream: mixed Ising (L in
    {16,..,256}) / Kitaev (L in 4..12) jobs, 1-64 chains, 10^3-max_proposals
    proposals each (log-uniform; the serving workload's range is 10^3-10^5,
    where one Kitaev L = 12 chain alone needs about 4 minutes for 10^5
    proposals, so the default run takes one decade less), mixed precision, HBM
    budget 8 GiB, n requests.  p50/p99 latency, aggregate proposals/s, and the
    offered load: chain-proposals per second the arrival process asks for."""
    from paper_2008_05401_gb300 import MIXED
    from paper_2008_05401_gb300.serving import Server, synthetic_requests
    reqs = synthetic_requests(n, rate_hz=rate, min_proposals=1000, max_proposals=max_proposals, precision=MIXED)
    span = max(r.arrival for r in reqs)
    offered = sum(r.S * len(r.T) for r in reqs) / max(span, 1e-9)
    srv = Server(device=dev, hbm_budget_bytes=8 << 30, quantum=256)
    t0 = time.perf_counter()
    srv.run(reqs, realtime=True, timeout_s=900.0)
    st = srv.stats(t_start=t0)
    iv = srv.launch_intervals()
    srv.close()
    busy = sum(b - a for _, _, a, b in iv)
    st.update({"arrivals": f"Poisson {rate:g}/s, {n} requests over {span:.3f} s",
               "offered_chain_proposals_per_s": offered,
               "launch_time_over_wall": busy / max(st.get("wall_s") or 1e-9, 1e-9),
               "jobs": f"Ising L in {{16..256}} or Kitaev L in 4..12, 1-64 chains, 1e3-{max_proposals:.0e} proposals "
                       "(log-uniform), mixed precision, HBM budget 8 GiB"})
    return st


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ising-batch")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--chains", type=int, default=0, help="override chains per lattice size (profiling)")
    ap.add_argument("--Ls", default="", help="comma list restricting the lattice sizes (profiling)")
    ap.add_argument("--no-secondary", action="store_true", help="skip the FP64-path and Kitaev lines")
    ap.add_argument("--serving-only", action="store_true",
                    help="run only the serving measurement (with --serving-requests, --serving-max-proposals)")
    ap.add_argument("--serving-requests", type=int, default=32)
    ap.add_argument("--serving-max-proposals", type=int, default=10_000)
    args = ap.parse_args()
    if args.serving_only:
        import __graft_entry__
        __graft_entry__.build()
        print(json.dumps({"serving": serving_run(0, n=args.serving_requests,
                                                  max_proposals=args.serving_max_proposals)}), flush=True)
        return
    spec = workload(args.workload)
    if args.Ls:
        keep = {int(x) for x in args.Ls.split(",")}
        spec["jobs"] = [(L, n) for L, n in spec["jobs"] if L in keep]
    if args.chains:
        spec["jobs"] = [(L, args.chains) for L, _ in spec["jobs"]]
    if args.impl == "reference":
        return run_reference(args, spec)

    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = local if world > 1 else 0
    import __graft_entry__
    __graft_entry__.build()
    from paper_2008_05401_gb300 import FP64, MIXED, Context, binding
    prec = MIXED if args.precision == "mixed" else FP64
    ctx = Context(dev)
    W, hb, vb = spec["model"]
    mid = ctx.load_model(spec["kind"], W, vb, hb)
    jobs = []
    base = 0
    for L, n in spec["jobs"]:
        init = wl.pack_bits(wl.random_lattices(n, L, seed=SEED + L))
        # weak scaling: each rank owns its own chain-id range
        jobs.append(ctx.new_job(mid, spec["kind"], L, spec["T"](n), spec["J"], SEED,
                                rank * 10_000_000 + base, init, prec))
        base += n
    S = spec["S"]
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=f"cuda:{dev}")
    for _ in range(args.warmup):
        ctx.run_batch(jobs, S, precision=prec, stream=stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with Clocks(dev) as ck:
        torch.cuda.synchronize(dev)
        for i in range(args.steps):
            flush.zero_()                      # L2 flush between timed steps (untimed)
            ev[i][0].record(stream)
            ctx.run_batch(jobs, S, precision=prec, stream=stream)
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device=f"cuda:{dev}")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    n_chains = sum(n for _, n in spec["jobs"])
    props = n_chains * S * args.steps * world
    value = props / (total_ms * 1e-3)
    clocks = ck.summary()

    # end to end through the C ABI with host buffers: upload lattices (pinned)
    # and re-evaluate the chains (crbm_write_states), run, read lattices and
    # observable sums back (crbm_read_states)
    host_bits = []
    for j in jobs:
        b = torch.empty(j.state()[0].shape, dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
        b[:] = j.state()[0]
        host_bits.append(b)
    out_bits = [torch.empty(b.shape, dtype=torch.int32, pin_memory=True).numpy().view(np.uint32) for b in host_bits]
    out_sums = [torch.empty((j.n, 4), dtype=torch.float64, pin_memory=True).numpy() for j in jobs]
    e2e_steps = 0 if args.no_e2e else max(2, min(args.steps, 5))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    h2d = d2h = 0
    for _ in range(e2e_steps):
        ctx.write_states(jobs, host_bits, [j.step for j in jobs], prec)      # one evaluation launch
        h2d += sum(hbits.nbytes for hbits in host_bits)
        ctx.run_batch(jobs, S, precision=prec, stream=stream)
        ctx.read_states(jobs, out_bits, out_sums)                           # one synchronisation
        d2h += sum(b.nbytes + x.nbytes for b, x in zip(out_bits, out_sums))
    e2e_s = time.perf_counter() - t0
    e2e = None if not e2e_steps else {
        "value": n_chains * S * e2e_steps * world / e2e_s, "unit": "proposals/s",
        "h2d_bytes_per_step": h2d // e2e_steps, "d2h_bytes_per_step": d2h // e2e_steps}

    K, k = W.shape[0], W.shape[1]
    sites = sum(n * L * L for L, n in spec["jobs"]) * S
    # the dominant kernel alone, on this stream, CUDA events around each launch
    # (after the timed region): in the mixed Ising path the persistent
    # tensor-core kernel, one launch for the jobs of every side it serves; else
    # the largest lattice's jobs on the table kernel
    tc_L = (128, 64, 32, 16) if prec == MIXED and spec["kind"] == 0 and K <= 4 and k <= 5 else ()
    dom = [(L, n, j) for (L, n), j in zip(spec["jobs"], jobs) if L in tc_L]
    dom_name = "crbm_tc_kernel (persistent, every side in one launch)"
    if not dom:
        dom = [(L, n, j) for (L, n), j in zip(spec["jobs"], jobs) if L == max(Lj for Lj, _ in spec["jobs"])]
        dom_name = "crbm_step_kernel"
    dom_jobs = [j for _, _, j in dom]
    dev_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(3)]
    ctx.run_batch(dom_jobs, S, precision=prec, stream=stream)
    for a, b in dev_ev:
        flush.zero_()
        a.record(stream)
        ctx.run_batch(dom_jobs, S, precision=prec, stream=stream)
        b.record(stream)
    torch.cuda.synchronize(dev)
    dom_ms = sum(a.elapsed_time(b) for a, b in dev_ev) / len(dev_ev)
    dom_sites = sum(n * L * L for L, n, _ in dom) * S
    # kernels per step: a proposal kernel and its step-counter update per part
    # of the batch (the tensor-core jobs form one part; table-kernel jobs one
    # per CTA size)
    n_parts = int(bool(tc_L and any(L in tc_L for L, _ in spec["jobs"]))) + \
        len({L for L, _ in spec["jobs"] if L not in tc_L})
    line = {"metric": METRIC, "value": value, "unit": "proposals/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if prec == MIXED else "f64", "data": "synthetic",
            "config": bench_config(spec, args, world),
            "roofline": roofline(dom_ms, clocks, K, k, dom_sites,
                                 traffic=(BATCH_ISING_TC_TRAFFIC_BYTES if args.workload == "ising-batch" and
                                          dom_name.startswith("crbm_tc") and not args.chains and not args.Ls
                                          else None)),
            "e2e": e2e, "gpu_launches": args.steps * 2 * n_parts, "clocks": clocks}
    line["roofline"]["kernel"] = (f"{dom_name}: L = {sorted({L for L, _, _ in dom}, reverse=True)} "
                                  f"({sum(n for _, n, _ in dom)} chains x {S} proposals), {dom_ms:.3f} ms per launch")
    step_rf = roofline(total_ms / args.steps, clocks, K, k, sites)
    line["roofline"]["whole_step"] = {"achieved": step_rf["achieved"], "frac": step_rf["frac"],
                                      "note": "every lattice size and kernel of the timed step"}
    sums = [j.observables() for j in jobs]
    props_done = max(1, n_chains * jobs[0].step)
    line["stats"] = {
        "acceptance": sum(int(a.sum()) for _, a, _ in sums) / props_done,
        "fp64_recomputes_per_proposal": {
            "bernoulli": sum(int(r[:, 0].sum()) for _, _, r in sums) / props_done,
            "mh": sum(int(r[:, 1].sum()) for _, _, r in sums) / props_done,
            "mh_by_L": {str(L): int(r[:, 1].sum()) / max(1, len(r) * j.step)
                        for (L, _), j, (_, _, r) in zip(spec["jobs"], jobs, sums)}},
        "acceptance_by_L": {str(L): int(a.sum()) / max(1, len(a) * j.step)
                            for (L, _), j, (_, a, _) in zip(spec["jobs"], jobs, sums)}}
    if rank == 0 and not args.no_secondary:
        # measured FMA peaks of this device (outside every timed region)
        PROBED["fp32"], PROBED["fp64"] = binding.crbm_probe_peaks(ctx.h)
        line["roofline"]["measured_fp32_fma_tflops"] = round(PROBED["fp32"], 2)
        line["roofline"]["frac_of_measured_fp32"] = round(line["roofline"]["achieved"] / PROBED["fp32"], 4)
        line["measured_fp64_fma_tflops"] = round(PROBED["fp64"], 3)
    if rank == 0 and not args.no_secondary and args.workload == "ising-batch":
        line["secondary"] = [
            secondary(Context, "ising-batch", FP64, 2, dev, stream, flush),
            # the persistent tensor-core launch of the whole batch, replayed from a captured graph
            secondary(Context, "ising-batch", MIXED, 3, dev, stream, flush, graph=True, clocks=clocks, tune=False),
            secondary(Context, "kitaev-small", FP64, 3, dev, stream, flush),
            secondary(Context, "kitaev-small", MIXED, 3, dev, stream, flush, clocks=clocks),
            secondary(Context, "kitaev-batch", FP64, 2, dev, stream, flush),
            secondary(Context, "kitaev-batch", MIXED, 2, dev, stream, flush, clocks=clocks),
            secondary(Context, "kitaev-batch", MIXED, 2, dev, stream, flush, graph=True, clocks=clocks),
            tempering_run(Context, "ising-batch", MIXED, 20, dev, stream, flush, clocks=clocks,
                          oracle_s=0.0 if args.no_cpu_baseline else 3.0),
            tempering_run(Context, "kitaev-small", MIXED, 4, dev, stream, flush,
                          oracle_s=0.0 if args.no_cpu_baseline else 2.0),
            # the paper's Kitaev protocol at L = 8: k = 4 Gibbs steps per correction (Table II)
            tempering_run(Context, "kitaev-small", MIXED, 4, dev, stream, flush,
                          oracle_s=0.0 if args.no_cpu_baseline else 2.0, g=4, L_n=(8, 1024))]
        line["stats"]["mixed_vs_fp64_path"] = value / line["secondary"][0]["value"]
        line["serving"] = serving_run(dev, n=args.serving_requests, max_proposals=args.serving_max_proposals)
        ob = 0.0 if args.no_cpu_baseline else 2.0
        line["train"] = train_run(Context, dev, stream, oracle_s=ob)
        line["lcrbm"] = lcrbm_run(Context, dev, stream, oracle_s=ob)
        line["tau"] = [tau_run(Context, 16, 1024, 2.269, 2000, dev, stream, oracle_s=ob),
                       tau_run(Context, 64, 512, 2.269, 2000, dev, stream, oracle_s=ob)]
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_run(spec, args.workload)
        line["cpu_baseline"]["single_core"] = {
            k_: v_ for k_, v_ in cpu_baseline_run(spec, args.workload, budget_s=8.0, cores=1).items()
            if k_ in ("value", "cores", "sample")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
