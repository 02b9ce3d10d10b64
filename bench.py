#!/usr/bin/env python
"""Benchmark of the GB300 Gibbs sampler on the paper-scale workload.

Workload: the RNA-seq model of Landau & Niemi (arXiv 1606.06659) on synthetic
Poisson-lognormal counts with N=16 samples (4 varieties x 4 libraries, the
paper's 16 x 5 design), G=40000 genes, L=5, theta=(4,0,0,0,0),
sigma=(2,.5,.3,.2,.2), tau=0.1, nu=3; priors c=s=10, a=b=1, d=10; run length
20000 iterations with 10000 burn-in and thin 10.

Forms: "f64" (the plain method in FP64: gamma_g, tau, sigma_l^2 drawn exactly),
"f64_all_slice" (the ablation that slice-samples gamma_g, tau and sigma_l as well,
as the paper does), "f32" (FP32 slice log densities, FP64
reductions and hyperparameters, Kahan-compensated FP32 moments) and "learned"
(the f32 form plus the learned beta_g proposal: 2e6 training pairs drawn by the
plain sampler during burn-in, trained on the GPU, then an eta-preserving
Metropolis-Hastings move before the slice updates of beta_g).  `--form` picks
the form of the headline line (default: learned); the configured job runs for
every form unless --forms headline, so that the line carries each form's
iterations/s and ESS/s next to the plain FP64 form's.

Metric: Gibbs iterations per second (value, device-timed) and min ESS per
second over all G*L beta.  A "step" is `--sweeps-per-step` consecutive Gibbs
sweeps (one fbs_run call replaying the captured CUDA graph); L2 is flushed
(a 256 MiB write) before every timed step.

Lines printed by rank 0 (one JSON object):
  --impl ours       the CUDA library through its C ABI
  --impl reference  the CPU oracle on this host's cores, on gene samples of the
                    same workload, scaled to the full G (there is no runnable
                    reference implementation of the paper)
With torchrun (N>1 ranks) every rank runs an independent chain on its own GPU
(chains are replicas; nothing is exchanged) and value = all ranks' sweeps /
the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gibbs iters/sec and min ESS/sec over beta at N=16,G=40000 vs plain FP64 form"
CFG = 1
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--form", choices=("f64", "f64_all_slice", "f32", "learned", "learned_a02",
                                       "learned_cfg4"),
                    default="learned")
    ap.add_argument("--forms", choices=("all", "headline"), default="all",
                    help="run the configured job (ESS) for every form or only the headline one")
    ap.add_argument("--block", type=int, default=0, help="threads per block of the gene kernel")
    ap.add_argument("--workload", choices=("paper", "batch"), default="paper",
                    help="paper: N=16 G=40000 L=5 (the metric's workload); batch: 64 datasets "
                         "of uneven N, G, L in one set of launches")
    ap.add_argument("--sweeps-per-step", type=int, default=100)
    ap.add_argument("--profile-run", type=int, default=0,
                    help="set up the timed sampler (tuning, and for a learned form training and "
                         "calibration), run this many sweeps as direct launches inside the NVTX "
                         "range 'profile_sweeps' and exit (for ncu captures)")
    ap.add_argument("--chains", type=int, default=4,
                    help="chains of the concurrent multi-chain job (the paper runs 4); 1: skip")
    ap.add_argument("--no-ess", action="store_true", help="skip the 20000-iteration ESS jobs")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--train-epochs", type=int, default=20,
                    help="training epochs of the learned proposal (2e6 pairs per epoch)")
    ap.add_argument("--tune-sweeps", type=int, default=2000,
                    help="burn-in sweeps that tune the slice widths before the timed steps")
    return ap.parse_args()


# --------------------------------------------------------------------------- helpers
# FP64 floating-point operations per slice log-density evaluation of the FP64
# sweep kernels k_eps_f64 + k_gb_f64 (DFMA counted as 2, DADD and DMUL as 1),
# from one ncu capture of each in a sampling sweep at config 1 (bench.py --form
# f64 --profile-run 2): 1.339e8 (eps) + 1.000e8 (gb) flop per sweep over the
# 6.141e6 log-density evaluations the device counted per sweep = 38.1.  The slice
# comparisons are decided in FP32 (0.35% fall back to FP64), so this covers the
# FP64 work that remains per evaluation on average (rates at accepted points,
# log-rates, class sums and rate updates, gamma draws, interval arithmetic,
# moments).  Re-measure when the kernels change.
FP64_FLOP_PER_EVAL = 38.1
FP64_TRAFFIC_BYTES = 44.1e6   # dram read+write of both kernels per sweep, same captures
# FP32 forms: warp instructions issued per sweep (smsp__inst_executed.sum) by the
# eps kernel and the gamma/beta kernel (k_gb_f32; with the learned proposal
# k_gb_net_f32, which includes the network pass, in a sampling sweep after
# calibration) and their dram read+write (writes stay in L2), from ncu captures
# at config 1 (bench.py --profile-run)
FP32_WARP_INST = {"f32": 21.01e6 + 9.12e6, "learned": 21.01e6 + 19.08e6}
FP32_TRAFFIC_BYTES = {"f32": 19.7e6 + 13.24e6, "learned": 19.7e6 + 15.49e6}
# issue peak: 152 SMs x 4 schedulers x 1 warp instruction per clock x 2.07 GHz
ISSUE_PEAK_WARP_INST_S = 152 * 4 * 2.07e9
# the proposal network's own flops per gene (2 x (F*64 + 64*64 + 64*K), F = 21,
# K = 20) and the tensor-core flops its split-BF16 GEMMs issue per gene
NET_FLOP_PER_GENE = 2 * (21 * 64 + 64 * 64 + 64 * 20)
MMA_FLOP_PER_GENE = 2 * 3 * (32 * 64 + 64 * 64 + 64 * 32)
# One training row (L = 5: F = 21 features, K = 20 outputs, hidden 64): the
# forward products, the two backward products that carry the gradient to the
# hidden layers, and the three weight-gradient products; and what the tensor
# cores execute for it (three split-BF16 products each, padded shapes: 22 -> 32
# input columns with the column of ones, 20 -> 32 outputs, the weight-gradient
# products as one of 128 x (64 + 32 + 32) and one of 128 x 64 over the rows)
TRAIN_FLOP_PER_ROW = 2 * (21 * 64 + 64 * 64 + 64 * 20) + 2 * (20 * 64 + 64 * 64) + \
    2 * (64 * 21 + 64 * 64 + 20 * 64)
TRAIN_MMA_FLOP_PER_ROW = 2 * 3 * ((32 * 64 + 64 * 64 + 64 * 32) + (32 * 64 + 64 * 64) +
                                  128 * 128 + 128 * 64)
# FP64 peak from unit counts and clock: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


# Algorithmic arithmetic per log-density evaluation of the FP32 slice updates,
# counted from EpsDensityF and BetaDensityFT (csrc/fbs_gene_f32.cu): an eps
# evaluation is 19 FP32 operations (the difference to x0, the e^z - 1 - z series
# of 8 FMA and 2 multiplies, the rate carried to the point, the quadratic prior
# term, the comparison with the level); a beta evaluation is 6 plus 13 per value
# class of its column (z = v d, the series, the class's two terms).  Every slice
# update adds one lg2 (the level log U) and the Philox blocks of its uniforms:
# 20 multiply-high per block (2 per round, 10 rounds), one block per 4 uniforms,
# 3 uniforms plus one per shrinkage proposal (bounded here by one per evaluation).
F32_OPS_EPS_EVAL = 19
F32_OPS_BETA_EVAL_BASE, F32_OPS_BETA_EVAL_PER_CLASS = 6, 13


def class_counts(X):
    """Distinct non-zero values of every column of X (the beta update's classes)."""
    X = np.asarray(X)
    return [len(set(v for v in X[:, l] if v != 0.0)) for l in range(X.shape[1])]


def alu_roofline(evals, N, G, L, X, ms_gene, peaks, precision):
    """Arithmetic roofline of the per-gene kernels of one sweep: the device-counted
    evaluations of the sweep times the algorithmic operations per evaluation,
    over the kernels' time inside the replayed graph, against each pipe's
    throughput measured by fbs_measure_peaks.  The bound is the pipe with the
    largest fraction."""
    t = ms_gene / 1e3
    if precision == "f64":
        flop = (evals["evals_eps"] + evals["evals_beta"] + evals["evals_gam"]) * FP64_FLOP_PER_EVAL
        peak = 2.0 * peaks["dfma"]
        return {"bound": "alu", "pipe": "fp64", "achieved": flop / t / 1e12,
                "peak": peak / 1e12, "unit": "TFLOP/s (FP64)", "frac": flop / t / peak,
                "flop_per_eval": FP64_FLOP_PER_EVAL,
                "peak_source": "measured (fbs_measure_peaks, FP64 FMA x 2)"}
    cls = class_counts(X)
    beta_ops = F32_OPS_BETA_EVAL_BASE + F32_OPS_BETA_EVAL_PER_CLASS * float(np.mean(cls))
    updates = (N + L) * G
    ev = evals["evals_eps"] + evals["evals_beta"]
    pipes = {
        "fp32": (F32_OPS_EPS_EVAL * evals["evals_eps"] + beta_ops * evals["evals_beta"],
                 peaks["ffma"]),
        "mufu": (float(updates), peaks["lg2"]),
        "imul_hi": (5.0 * (3.0 * updates + ev), peaks["imulhi"]),
    }
    out = {k: {"ops_per_sweep": ops, "achieved_per_s": ops / t, "peak_per_s": pk,
               "frac": ops / t / pk} for k, (ops, pk) in pipes.items()}
    top = max(out, key=lambda k: out[k]["frac"])
    return {"bound": "alu", "pipe": top, "achieved": out[top]["achieved_per_s"] / 1e12,
            "peak": out[top]["peak_per_s"] / 1e12, "unit": "Tops/s", "frac": out[top]["frac"],
            "pipes": out, "peak_source": "measured (fbs_measure_peaks)",
            "ops_per_eval": {"eps": F32_OPS_EPS_EVAL, "beta": beta_ops}}


def bytes_per_gene(N, L, precision="f64"):
    """Algorithmic HBM bytes of one gene in one post-burn-in sweep of the per-gene
    kernel.  FP64: reads y (4N), eps, w_eps (8N each), beta, w_beta, T (8L each),
    gamma (8); read+write of the eps/beta/gamma running mean and mean square
    (32 per parameter); writes eps (8N), beta (8L), gamma (8).  FP32: reads y
    (4N), eps, w_eps (4N each), beta, w_beta (4L each), gamma (4); read+write of
    four FP32 moment planes per parameter (32); writes eps (4N), beta (4L), gamma (4)."""
    if precision == "f32":
        return 48 * N + 44 * L + 40
    return 60 * N + 64 * L + 48


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples taken every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu, self.proc, self.lines = gpu_index, None, []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def host_cpu():
    """Core count (the threads this process may use) and CPU model of this host."""
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() in ("Model name", "Model"):
                model = ln.split(":", 1)[1].strip()
                if ln.startswith("Model name"):
                    break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for ln in f:
                    if ln.lower().startswith(("model name", "cpu part")):
                        model = ln.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    import platform
    return cores, f"{model or 'unknown'} ({platform.machine()})"


def oracle_sweep_rate(data, seconds, threads, G_s=None, min_sweeps=2):
    """Sweeps per second of the CPU oracle as it stands on `threads` host threads
    (its per-gene loops under OpenMP), over the full workload or its first G_s
    genes, burn-in sweeps for about `seconds` (at least min_sweeps)."""
    import oracle
    y = data["y"] if G_s is None else data["y"][:G_s]
    old = oracle.set_threads(threads)
    try:
        ch = oracle.Chain(y, data["X"], data["h"], data["priors"], seed=7, burnin=10000,
                          tune_start=5000).init_default()
        ch.sweep()   # first touch of the state
        n, t0 = 0, time.perf_counter()
        while True:
            ch.sweep()
            n += 1
            el = time.perf_counter() - t0
            if el >= seconds and n >= min_sweeps:
                break
    finally:
        oracle.set_threads(old)
    return n / el, n, el


def cpu_baseline(data, seconds, G_full):
    """The CPU oracle as it stands on this host's cores: single-threaded on a
    gene sample (one sweep costs O(G), so the rate is scaled to the full G) and
    on every core over the full workload (OpenMP over genes), iterations/s each.
    `value` is the all-core rate."""
    cores, model = host_cpu()
    G_s = 2000
    r1, n1, t1 = oracle_sweep_rate(data, seconds / 2, 1, G_s=G_s)
    r1 *= G_s / G_full
    rn, nn, tn = oracle_sweep_rate(data, seconds / 2, cores)
    return {"value": rn, "unit": "iters/s", "cores": cores, "kind": "oracle", "cpu": model,
            "single_thread": r1, "all_cores": rn,
            "sample": f"all cores: {nn} full oracle sweeps of G={G_full} ({tn:.1f} s of burn-in "
                      f"sweeps); one core: {n1} sweeps over the first {G_s} genes ({t1:.1f} s), "
                      f"scaled by G/{G_s}"}


# --------------------------------------------------------------------------- reference arm
def job_rate(units_per_rank, seconds, world, device):
    """Whole-job throughput of `world` replicas: every rank processed
    units_per_rank units in `seconds`; the job takes as long as its slowest rank
    (MAX all-reduce of the times), so value = all ranks' units / that time."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([seconds], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        seconds = float(t.item())
    return units_per_rank * world / seconds, seconds


def run_reference(args, rank):
    """The oracle as it stands, on every host core, timed over real full-size
    sweeps of the paper-scale workload: each step is one sweep of all G genes."""
    if rank != 0:
        return
    from paper_1606_06659_gb300 import synthetic
    import oracle
    data = synthetic.make_config(CFG)
    G = data["spec"]["G"]
    cores, model = host_cpu()
    old = oracle.set_threads(cores)
    try:
        ch = oracle.Chain(data["y"], data["X"], data["h"], data["priors"], seed=7,
                          burnin=10000, tune_start=5000).init_default()
        for _ in range(args.warmup):
            ch.sweep()
        times = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            ch.sweep()
            times.append(time.perf_counter() - t0)
    finally:
        oracle.set_threads(old)
    per_sweep = statistics.mean(times)
    value = 1.0 / per_sweep
    sample = (f"{args.steps} timed full sweeps (G={G}) after {args.warmup} warm-up sweeps, "
              f"{cores} threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": per_sweep * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "RNA-seq Gibbs sweep N=16 G=40000 L=5 (paper design)",
                       "N": 16, "G": G, "L": 5, "step": "one full oracle sweep"},
            "cpu_baseline": {"value": value, "unit": "iters/s", "cores": cores, "kind": "oracle",
                             "cpu": model, "sample": sample},
            "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- batch workload
def run_batch(args):
    """64 datasets (N uniform on 4..32, G log-uniform on [1e3, 1e5], L in {2, 5})
    swept together in the FP32 form; the schedule comes from the autotuner."""
    import torch
    import paper_1606_06659_gb300 as fbs
    from paper_1606_06659_gb300 import synthetic
    sets = synthetic.make_batch(64)
    genes = sum(d["y"].shape[0] for d in sets)
    cells = sum(d["y"].size for d in sets)
    b = fbs.BatchSampler(sets, seeds=[20160621 + i for i in range(len(sets))])
    eb, gb, ms_tune = b.autotune(sweeps=5, burnin=5000)
    S = args.sweeps_per_step
    b.run(1000, burnin=5000)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for i in range(args.warmup):
        flush.fill_(i & 0xFF)
        b.run(S, burnin=5000)
    torch.cuda.synchronize()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    for i, (a, e) in enumerate(evs):
        flush.fill_((i + 3) & 0xFF)
        a.record(stream)
        b.run(S, burnin=5000)
        e.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    b.sync()
    step_ms = [a.elapsed_time(e) for a, e in evs]
    sweeps_per_s = args.steps * S / (sum(step_ms) / 1e3)
    line = {"metric": "batched Gibbs sweeps/sec (64 datasets per sweep)", "value": sweeps_per_s,
            "unit": "batch sweeps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.mean(step_ms), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "64 datasets, N uniform on 4..32, G log-uniform on "
                                   "[1e3, 1e5], L in {2,5}", "genes": genes, "cells": cells,
                       "schedule": {"eps_block": eb, "gb_block": gb,
                                    "autotune_ms_per_sweep": ms_tune},
                       "sweeps_per_step": S},
            "gene_sweeps_per_s": sweeps_per_s * genes, "cell_sweeps_per_s": sweeps_per_s * cells,
            "gpu_launches": args.steps * (3 * S + 2), "clocks": clk}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- our arm
FORM_TEXT = {
    "f64": "plain method, FP64",
    "f64_all_slice": "plain method, FP64, with gamma_g, tau and sigma_l slice-sampled "
                     "(each with its own tuned width) instead of drawn exactly",
    "f32": "FP32 slice log densities; FP64 reductions and hyperparameters; "
           "Kahan-compensated FP32 moments",
    "learned": "the f32 form plus the learned beta_g proposal (eta-preserving MH move "
               "before the slice updates of beta_g)",
    "learned_a02": "as learned, with the calibration threshold 0.2 of configuration 4",
    "learned_cfg4": "configuration 4 as written: the learned move replaces the slice updates "
                    "of beta_g; genes below 0.2 acceptance keep the slice sampler",
}
PAIR_SWEEPS = 50          # x thin 2 x G = 2e6 training pairs at G = 40000
TRAIN = {"epochs": 20, "batch": 8192, "lr": 3e-3}
CALIBRATE_SWEEPS = 100
# Calibration threshold of the learned move.  The headline form adds the move to
# the slice updates of beta_g (mode 1), so the slice sampler always runs and the
# threshold only decides whether a gene also makes the move: any gene whose
# better proposal accepts 1% of the time gains from it (each accepted move is a
# nearly independent draw of beta_g given the log-rates).  The 0.2 of the
# configured fallback applies where the move replaces the slice updates (mode 2).
MIN_ACCEPT = 0.01
# The learned forms of the job: (calibration threshold, mode).  "learned" is the
# headline; "learned_a02" takes configuration 4's threshold 0.2 with the move
# added to the slice updates; "learned_cfg4" is configuration 4 as written: the
# move replaces the slice updates of beta_g, and genes whose acceptance stays
# below 0.2 fall back to the slice sampler.
LEARNED_FORMS = {"learned": (MIN_ACCEPT, 1), "learned_a02": (0.2, 1), "learned_cfg4": (0.2, 2)}


def new_sampler(fbs, data, y, form, seed, chain, block, **kw):
    prec = fbs.FBS_F64 if form.startswith("f64") else fbs.FBS_F32
    return fbs.Sampler(y, data["X"], data["h"], data["priors"], seed=seed, chain=chain,
                       precision=prec, block=block, all_slice=int(form == "f64_all_slice"),
                       **kw)


def geyer_ess(tr):
    """Effective sample size of every column of a [rows][S] host trace (Geyer's
    initial monotone sequence; the device kernel behind fbs_beta_ess does the same
    for beta).  Used for the few hyperparameter columns."""
    tr = np.asarray(tr, np.float64)
    n = tr.shape[0]
    out = []
    for x in tr.T:
        x = x - x.mean()
        c0 = float(x @ x) / n
        if not c0 > 0:
            out.append(float(n))
            continue
        ac = np.correlate(x, x, "full")[n - 1:] / n / c0
        s, prev = 0.0, np.inf
        for j in range(0, n // 2):
            if 2 * j + 1 >= n:
                break
            pair = ac[2 * j] + ac[2 * j + 1]
            if not pair > 0:
                break
            pair = min(pair, prev)
            s += pair
            prev = pair
        out.append(n / max(-1.0 + 2.0 * s, 1.0 / n))
    return np.array(out)


def ess_job(fbs, torch, data, y_host, form, seed, chain, block, S, train_epochs):
    """The configured job (20000 iterations, burn-in 10000, thin 10) through the
    public API with pinned host counts: init upload, the sweeps in fbs_run calls of
    S iterations with phi read back after each, moments read back at the end.  For
    the learned form the job also collects the training pairs (after half the
    burn-in), trains the network and calibrates, all inside the timed job."""
    spec = data["spec"]
    iters, burnin, thin = spec["iters"], spec["burnin"], spec["thin"]
    rows = (iters - burnin) // thin
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    smp = new_sampler(fbs, data, y_host, form, seed, chain, block, trace_cap=rows, trace_beta=1)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    done, phi_reads, extra = 0, 0, {}

    def advance(upto):
        nonlocal done, phi_reads
        while done < upto:
            n = min(S, upto - done)
            smp.run(n, burnin=burnin, thin=thin)
            smp.phi()
            phi_reads += 1
            done += n

    if form in LEARNED_FORMS:
        min_accept, mode = LEARNED_FORMS[form]
        advance(burnin // 2)
        tt = time.perf_counter()
        smp.proposal_collect(PAIR_SWEEPS, burnin=burnin, thin=2)
        done += 2 * PAIR_SWEEPS
        t_tr = time.perf_counter()   # proposal_collect returns with the stream synchronised
        loss = smp.proposal_train(seed=seed, **dict(TRAIN, epochs=train_epochs))
        t_tr = time.perf_counter() - t_tr   # and proposal_train too
        smp.proposal_calibrate(CALIBRATE_SWEEPS, burnin=burnin, min_accept=min_accept)
        smp.proposal_mode(mode)
        done += CALIBRATE_SWEEPS
        st0 = smp.proposal_stats()
        n_pairs = PAIR_SWEEPS * data["y"].shape[0]
        extra = {"train_pairs": n_pairs, "train_loss": loss, "train_s": t_tr,
                 "train_steps": train_epochs * ((n_pairs + TRAIN["batch"] - 1) // TRAIN["batch"]),
                 "collect_train_calibrate_s": time.perf_counter() - tt,
                 "mh_genes": st0["mh_genes"], "prior_genes": st0["prior_genes"],
                 "min_accept": min_accept, "mode": mode}
    advance(iters)
    ev1.record(stream)
    mom = smp.moments()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    dev_s = ev0.elapsed_time(ev1) / 1e3
    e = smp.beta_ess()
    ess_phi = geyer_ess(smp.trace()["phi"])
    if form in LEARNED_FORMS:
        st = smp.proposal_stats()
        extra["accept_rate"] = st["accepted"] / max(1, st["tried"])
        extra["params"] = smp.proposal_params()
    h2d = y_host.nbytes + data["X"].nbytes + data["h"].nbytes
    d2h = phi_reads * 8 * (2 * spec["L"] + 2) + sum(np.asarray(v).nbytes for k, v in mom.items()
                                                     if k != "count")
    smp.close()
    del smp
    torch.cuda.empty_cache()
    out = {"iters_per_s_e2e": iters / wall, "iters_per_s_job_device": iters / dev_s,
           "job_wall_s": wall, "min_ess": float(e.min()), "p05_ess": float(np.percentile(e, 5)),
           "median_ess": float(np.median(e)), "ess_rows": rows,
           "min_ess_per_s": float(e.min()) / wall, "p05_ess_per_s": float(np.percentile(e, 5)) / wall,
           "median_ess_per_s": float(np.median(e)) / wall,
           "phi_ess": [round(float(v), 1) for v in ess_phi],
           "min_phi_ess_per_s": float(ess_phi.min()) / wall,
           "h2d_bytes_per_step": h2d / phi_reads, "d2h_bytes_per_step": d2h / phi_reads}
    out.update(extra)
    return out


def chains_job(fbs, torch, data, y_host, form, seed, C, block, S, train_epochs):
    """The paper's job shape (§5 runs 4 chains): C independent chains of the
    configured job (20000 iterations, burn-in 10000, thin 10), each a handle on
    its own CUDA stream so that the chains run concurrently on the one GPU, end to
    end through the public API with pinned host counts.  For a learned form chain
    0 collects the training pairs and trains the network inside the job; every
    chain then calibrates.  Pooled ESS of a beta_gl = the sum of its chains'
    Geyer ESS; convergence from the chains' running moments (fbs_rhat, §3.1)."""
    spec = data["spec"]
    iters, burnin, thin = spec["iters"], spec["burnin"], spec["thin"]
    rows = (iters - burnin) // thin
    main = torch.cuda.current_stream()
    streams = [torch.cuda.Stream() for _ in range(C)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    smps = []
    for c in range(C):
        with torch.cuda.stream(streams[c]):
            smps.append(new_sampler(fbs, data, y_host, form, seed, c, block, trace_cap=rows,
                                    trace_beta=1))
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(main)
    for st in streams:
        st.wait_event(ev0)
    done, phi_reads = 0, 0

    def advance(upto):
        nonlocal done, phi_reads
        while done < upto:
            n = min(S, upto - done)
            for c in range(C):
                with torch.cuda.stream(streams[c]):
                    smps[c].run(n, burnin=burnin, thin=thin)
            for c in range(C):
                smps[c].phi()
                phi_reads += 1
            done += n

    extra = {}
    if form in LEARNED_FORMS:
        min_accept, mode = LEARNED_FORMS[form]
        advance(burnin // 2)
        tt = time.perf_counter()
        with torch.cuda.stream(streams[0]):
            smps[0].proposal_collect(PAIR_SWEEPS, burnin=burnin, thin=2)
            smps[0].proposal_train(seed=seed, **dict(TRAIN, epochs=train_epochs))
        params = smps[0].proposal_params()
        for c in range(C):
            with torch.cuda.stream(streams[c]):
                if c > 0:  # the same sweeps as chain 0's collection, without collecting
                    smps[c].run(2 * PAIR_SWEEPS, burnin=burnin, thin=thin)
                    smps[c].proposal_params(set_to=params)
                smps[c].proposal_calibrate(CALIBRATE_SWEEPS, burnin=burnin, min_accept=min_accept)
                smps[c].proposal_mode(mode)
        done += 2 * PAIR_SWEEPS + CALIBRATE_SWEEPS
        extra = {"collect_train_calibrate_s": time.perf_counter() - tt, "min_accept": min_accept,
                 "mode": mode, "trained_on": "chain 0's pairs"}
    advance(iters)
    for st in streams:
        main.wait_stream(st)
    ev1.record(main)
    moms = [s.moments() for s in smps]
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    dev_s = ev0.elapsed_time(ev1) / 1e3
    ess = sum(s.beta_ess() for s in smps)
    phi_ess = sum(geyer_ess(s.trace()["phi"]) for s in smps)
    rh = fbs.rhat(smps)
    if form in LEARNED_FORMS:
        sts = [s.proposal_stats() for s in smps]
        extra["accept_rate"] = sum(x["accepted"] for x in sts) / max(1, sum(x["tried"] for x in sts))
    h2d = C * (y_host.nbytes + data["X"].nbytes + data["h"].nbytes)
    d2h = phi_reads * 8 * (2 * spec["L"] + 2) + sum(
        np.asarray(v).nbytes for m in moms for k, v in m.items() if k != "count")
    for s in smps:
        s.close()
    torch.cuda.empty_cache()
    out = {"chains": C, "iters_per_s_e2e": C * iters / wall, "iters_per_s_job_device": C * iters / dev_s,
           "job_wall_s": wall, "pooled_min_ess": float(ess.min()),
           "pooled_p05_ess": float(np.percentile(ess, 5)), "pooled_median_ess": float(np.median(ess)),
           "min_ess_per_s": float(ess.min()) / wall,
           "p05_ess_per_s": float(np.percentile(ess, 5)) / wall,
           "median_ess_per_s": float(np.median(ess)) / wall,
           "min_phi_ess_per_s": float(phi_ess.min()) / wall,
           "rhat_phi_max": float(np.nanmax(rh["phi"])),
           "rhat_beta_frac_above_1_1": float(np.mean(rh["beta"] > 1.1)),
           "h2d_bytes_per_step": h2d / max(1, phi_reads // C),
           "d2h_bytes_per_step": d2h / max(1, phi_reads // C)}
    out.update(extra)
    return out


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.workload == "batch":
        run_batch(args)
        return

    import torch
    import torch.distributed as dist

    import paper_1606_06659_gb300 as fbs
    from paper_1606_06659_gb300 import synthetic

    if not os.path.exists(fbs.LIB_PATH):
        from paper_1606_06659_gb300 import build as fbs_build
        fbs_build.build()
    assert torch.cuda.is_available(), "bench.py needs a GPU"
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    data = synthetic.make_config(CFG)
    spec = data["spec"]
    N, G, L = spec["N"], spec["G"], spec["L"]
    S = args.sweeps_per_step
    seed = 20160621
    form = args.form
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- the configured job of each form, end to end with host buffers
    y_pinned = torch.from_numpy(np.ascontiguousarray(data["y"])).pin_memory()
    y_host = y_pinned.numpy()
    burnin, thin = spec["burnin"], spec["thin"]
    forms = {}
    if not args.no_ess:
        order = (["f64", "f64_all_slice", "f32", "learned", "learned_a02", "learned_cfg4"]
                 if args.forms == "all" else [form])
        for f in order:
            barrier()
            forms[f] = ess_job(fbs, torch, data, y_host, f, seed, rank, args.block, S,
                               args.train_epochs)
    jobs_c = {}
    if not args.no_ess and args.chains > 1:
        for f in ("f64", "learned") if args.forms == "all" else (form,):
            barrier()
            jobs_c[f] = chains_job(fbs, torch, data, y_host, f, seed + 100, args.chains,
                                   args.block, S, args.train_epochs)
    params = forms.get("learned", {}).pop("params", None)
    for f in ("learned_a02", "learned_cfg4"):
        forms.get(f, {}).pop("params", None)

    # ---- device-timed throughput: W warm-up + K timed steps of S sweeps
    train_timed = None
    if form in forms and "train_s" in forms[form]:
        train_timed = {"s": forms[form]["train_s"], "steps": forms[form]["train_steps"]}
    smp = new_sampler(fbs, data, data["y"], form, seed + 1, rank, args.block)
    tb = args.tune_sweeps // 2
    smp.run(args.tune_sweeps, burnin=tb, thin=thin)   # tune the slice widths (burn-in)
    learned = form in LEARNED_FORMS
    if learned:
        if params is None:
            smp.proposal_collect(PAIR_SWEEPS, burnin=tb, thin=2)
            torch.cuda.synchronize()
            t_tr = time.perf_counter()
            smp.proposal_train(seed=seed, **dict(TRAIN, epochs=args.train_epochs))
            t_tr = time.perf_counter() - t_tr
            n_pairs = PAIR_SWEEPS * data["y"].shape[0]
            train_timed = {"s": t_tr, "steps": args.train_epochs *
                           ((n_pairs + TRAIN["batch"] - 1) // TRAIN["batch"])}
        else:
            smp.proposal_params(set_to=params)
        min_accept, mode = LEARNED_FORMS[form]
        smp.proposal_calibrate(CALIBRATE_SWEEPS, burnin=tb, min_accept=min_accept)
        smp.proposal_mode(mode)
    if args.profile_run > 0:
        torch.cuda.synchronize()
        k0 = smp.counters()
        torch.cuda.nvtx.range_push("profile_sweeps")
        for _ in range(args.profile_run):
            smp.run(1, burnin=tb, thin=thin)   # one sweep: its kernels as direct launches
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        k1 = smp.counters()
        smp.close()
        print(json.dumps({"profile_run": args.profile_run, "form": form,
                          "evals_per_sweep": {k: (k1[k] - k0[k]) / args.profile_run
                                              for k in ("evals_eps", "evals_beta", "evals_nu",
                                                        "evals_gam")}}), flush=True)
        return
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    for i in range(args.warmup):
        flush.fill_(i & 0xFF)
        smp.run(S, burnin=tb, thin=thin)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    c0 = smp.counters()
    torch.cuda.nvtx.range_push("timed_steps")
    for i, (a, b) in enumerate(evs):
        flush.fill_((i + 7) & 0xFF)
        a.record(stream)
        smp.run(S, burnin=tb, thin=thin)
        b.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    c1 = smp.counters()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_s = sum(step_ms) / 1e3
    value, total_s = job_rate(args.steps * S, total_s, world, "cuda")
    barrier()

    # ---- rooflines of the per-gene kernels, timed inside a replayed graph laid
    #      out like the sweep's (fbs_profile: event-record nodes around each
    #      kernel, on the kernel's own stream)
    ms_k1, ms_k2, ms_hyper, ms_prop, ms_replay = smp.profile(S, burnin=tb, thin=thin)
    ms_gene = ms_k1 + ms_k2
    peak, peak_kind = measured_peaks()
    prec_name = "f64" if form.startswith("f64") else "f32"
    bpg = bytes_per_gene(N, L, prec_name)
    achieved = bpg * G / (ms_gene / 1e3) / 1e9
    evals = {k: (c1[k] - c0[k]) / (args.steps * S) for k in ("evals_eps", "evals_beta",
                                                               "evals_nu", "evals_gam",
                                                               "evals_hyp")}
    ev_launch = evals["evals_eps"] + evals["evals_beta"] + evals["evals_gam"]
    pipe_peaks = fbs.measure_peaks()
    if prec_name == "f64":
        kern = "k_eps_f64 + k_gb_f64"
        traffic = FP64_TRAFFIC_BYTES
    else:
        kern = "k_eps_f32 + " + ("k_gb_net_f32" if learned else "k_gb_f32")
        traffic = FP32_TRAFFIC_BYTES["learned" if learned else "f32"]
    # primary: the algorithmic bytes of one sweep's per-gene work (bytes_per_gene
    # x G) over the two per-gene kernels' time, against the measured HBM copy rate
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": kern,
                "kernel_ms": ms_gene, "eps_kernel_ms": ms_k1, "gb_kernel_ms": ms_k2,
                "hyper_kernel_ms": ms_hyper, "critical_path_ms": ms_k2 + max(ms_k1, ms_hyper),
                "sweep_ms": statistics.mean(step_ms) / S, "profiled_sweep_ms": ms_replay,
                "bytes_per_gene": bpg,
                "genes_per_launch": G, "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)",
                "timing": "span from the first block's start to the last block's end of each "
                          "kernel (device global timer) inside a replayed graph segment laid "
                          "out as fbs_run's (fbs_profile), mean over one segment",
                "evals_per_launch": ev_launch}
    roofline["alu"] = alu_roofline(evals, N, G, L, data["X"], ms_gene, pipe_peaks, prec_name)
    roofline["pipe_peaks_per_s"] = pipe_peaks
    if prec_name == "f32":
        inst = FP32_WARP_INST["learned" if learned else "f32"]
        rate = inst / (ms_gene / 1e3)
        roofline["issue"] = {"achieved": rate, "peak": ISSUE_PEAK_WARP_INST_S,
                             "unit": "warp-instructions/s", "frac": rate / ISSUE_PEAK_WARP_INST_S,
                             "warp_instructions_per_sweep": inst,
                             "peak_source": "152 SMs x 4 schedulers x 1 warp instruction/clk "
                                            "x 2.07 GHz (ncu-counted issued instructions)"}
    if learned:
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                bf16, src = float(json.load(f)["bf16_tflops_sustained"]), "measured"
        except (OSError, KeyError, ValueError):
            bf16, src = 1700.0, "fallback"
        tf = NET_FLOP_PER_GENE * G / (ms_prop / 1e3) / 1e12
        roofline["proposal"] = {
            "kernel": "k_proposal_tc", "bound": "tensor", "kernel_ms": ms_prop,
            "achieved": tf, "peak": bf16, "unit": "TFLOP/s", "frac": tf / bf16,
            "flop_per_launch": NET_FLOP_PER_GENE * G,
            "mma_flop_per_launch": MMA_FLOP_PER_GENE * G,
            "peak_source": src + " bf16 sustained"}
        if train_timed is not None:
            step_s = train_timed["s"] / train_timed["steps"]
            rows = TRAIN["batch"]
            tft = TRAIN_FLOP_PER_ROW * rows / step_s / 1e12
            roofline["training"] = {
                "kernels": "k_mlp_tc + k_reduce_adam per step (one graph replay per 8 steps)",
                "bound": "tensor", "step_us": step_s * 1e6, "rows_per_step": rows,
                "achieved": tft, "peak": bf16, "unit": "TFLOP/s", "frac": tft / bf16,
                "flop_per_step": TRAIN_FLOP_PER_ROW * rows,
                "mma_flop_per_step": TRAIN_MMA_FLOP_PER_ROW * rows,
                "mma_tflops": TRAIN_MMA_FLOP_PER_ROW * rows / step_s / 1e12,
                "timing": "host-timed fbs_proposal_train call of the job (20 epochs of the "
                          "2e6 pairs; device synchronised on both sides; column statistics, "
                          "folding and graph instantiation included) / its steps",
                "peak_source": src + " bf16 sustained"}
    st = smp.proposal_stats() if learned else None
    smp.close()

    # ---- the plain FP32 sweep as a graph of separate launches against the
    #      persistent form (one cooperative launch per segment), device-timed
    persist = {}
    for pers in (0, 1):
        p2 = new_sampler(fbs, data, data["y"], "f32", seed + 2, rank, args.block, persistent=pers)
        p2.run(args.tune_sweeps, burnin=tb, thin=thin)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(pers)
        e0.record(stream)
        p2.run(args.steps * S, burnin=tb, thin=thin)
        e1.record(stream)
        torch.cuda.synchronize()
        persist["persistent" if pers else "graph"] = e0.elapsed_time(e1) / (args.steps * S)
        p2.close()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    # eps, gamma/beta (with the learned proposal it runs the network too) and
    # hyperparameter kernels per sweep, plus the segment snapshot per step
    launches_per_sweep = 3
    line = {
        "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.mean(step_ms), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": prec_name, "data": "synthetic",
        "config": {"workload": "RNA-seq Gibbs sweep N=16 G=40000 L=5 (paper design), "
                               "one chain per GPU",
                   "form": form, "form_text": FORM_TEXT[form],
                   "N": N, "G": G, "L": L, "sweeps_per_step": S,
                   "l2": "256 MiB write before every timed step; state (~40 MB) stays "
                         "L2-resident within a step",
                   "job": f"{spec['iters']} iterations, burn-in {burnin}, thin {thin}",
                   "parallelism": f"{world} independent chain(s)"},
        "gpu_launches": args.steps * (launches_per_sweep * S + 1),
        "clocks": clk,
        "roofline": roofline,
        "evals_per_sweep": evals,
        "persistent_vs_graph_ms_per_sweep": dict(
            persist, form="f32", what="device-timed sweeps of the plain FP32 form: the graph "
                                       "of three launches per sweep against one cooperative "
                                       "launch per segment (the chains are identical)"),
    }
    if st is not None:
        line["learned_timed"] = {"mh_genes": st["mh_genes"],
                                 "accept_rate": st["accepted"] / max(1, st["tried"])}
    if form in forms:
        h = forms[form]
        line["e2e"] = {"value": h["iters_per_s_e2e"] * world, "unit": "iters/s",
                       "h2d_bytes_per_step": h["h2d_bytes_per_step"],
                       "d2h_bytes_per_step": h["d2h_bytes_per_step"],
                       "what": "the whole configured job through fbs_init/fbs_run/fbs_moments "
                               "with pinned host counts: init upload, 20000 sweeps (for the "
                               "learned form also pair collection, training and calibration), "
                               "phi read back after every step, moments read back at the end"}
        line["min_ess_per_sec"] = h["min_ess_per_s"]
        line["forms"] = forms
        if "f64" in forms:
            b = forms["f64"]
            line["vs_plain_f64"] = {
                k: h[k] / b[k] for k in ("iters_per_s_e2e", "min_ess_per_s", "p05_ess_per_s",
                                         "median_ess_per_s")}
            if "f64_all_slice" in forms:
                a = forms["f64_all_slice"]
                line["all_slice_vs_exact_draws"] = {
                    k: a[k] / b[k] for k in ("iters_per_s_e2e", "min_ess_per_s",
                                             "median_ess_per_s", "min_phi_ess_per_s")}
            line["learned_vs_plain_f64"] = {
                f: {k: forms[f][k] / b[k] for k in ("min_ess_per_s", "p05_ess_per_s",
                                                    "median_ess_per_s", "min_phi_ess_per_s")}
                for f in LEARNED_FORMS if f in forms}
    if jobs_c:
        line["chains_job"] = jobs_c
        if "f64" in jobs_c and "learned" in jobs_c:
            a, b = jobs_c["learned"], jobs_c["f64"]
            line["chains_job_learned_vs_plain_f64"] = {
                k: a[k] / b[k] for k in ("iters_per_s_e2e", "min_ess_per_s", "p05_ess_per_s",
                                         "median_ess_per_s", "min_phi_ess_per_s")}
        if "learned" in jobs_c and "learned" in forms:
            line["chains_job_vs_one_chain"] = {
                k: jobs_c["learned"][k] / forms["learned"][k]
                for k in ("iters_per_s_e2e", "min_ess_per_s", "p05_ess_per_s", "median_ess_per_s")}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(data, args.cpu_seconds, G)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
