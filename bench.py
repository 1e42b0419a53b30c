"""Throughput benchmark of the GSGP hot path on GB300.

One step = one complete GSGP run on one batch of synthetic fitness cases
already resident in HBM: staging of the cases (feature-major transpose),
initialisation (program generation for P and R, interpretation over all
cases, initial fitness), G generations (tournament selection, geometric
semantic mutation fused with train/test RMSE, survival with elitism, trace),
reconstruction of the best individual and its prediction on the test cases.

metric = semantic updates/s = m * n_cases * G / step time (n_cases = train +
test cases), whole job (all ranks).  Under torchrun every rank runs an
independent replica (its own run index) of the same workload: weak scaling,
no collective on the data path.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload large]
  python bench.py --impl reference ...   # the CPU oracle timed on the host
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "semantic updates/s (pop·n·gens/s) and % of HBM peak, vs plain FP32 at stated err"
UNIT = "semantic updates/s"
PROFILE_DIR = os.path.join(ROOT, "profiles")
GEN_KERNEL_SRC = [os.path.join(ROOT, "paper_2106_04034_gb300", "csrc", f)
                  for f in ("k_persist.cu", "k_generation.cu", "stream.cuh", "common.cuh",
                            "reduce.cuh", "gridsync.cuh", "kernels.cuh")]


def measured_peak_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---- replicas: one independent run per rank, no collective on the data path
def replica_workload(w: W.Workload, rank: int) -> W.Workload:
    """The workload of rank `rank`: same shapes, its own run index (Philox
    counter word and data seed), so replicas draw independent data."""
    return w.replace(run=w.run + rank)


def max_over_ranks(x: float, world: int, device="cuda") -> float:
    """The slowest rank's value (the job's time); identity for one rank."""
    if world <= 1:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: units all ranks processed / the job's time."""
    return units_per_rank * world / seconds


def alu_peak_tops():
    """FP32 lane operations per second of the GPU (T/s): 152 SMs x 128 lanes
    x the maximum SM clock from MEASURED_PEAKS.json (2070 MHz if absent)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            mhz = float(json.load(fh)["sm_max_mhz"])
    except Exception:
        mhz = 2070.0
    return 152 * 128 * mhz * 1e6 / 1e12


def kernel_source_hash() -> str:
    """Hash of the generation kernels' sources, recorded in ncu summaries."""
    h = hashlib.sha256()
    for f in GEN_KERNEL_SRC:
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(workload_name: str, shape):
    """DRAM traffic of the generation kernel from the committed ncu summary
    of this workload (profiles/persist_kernel_<workload>.txt), if it was
    taken with the current kernel sources and holds the stream shape in use
    (else None): the measured ratio of DRAM bytes to the algorithmic bytes of the
    captured launch.  The caller multiplies it by its own launches'
    algorithmic bytes (a generation's traffic changes over a run as the
    population's distinct parents do, the ratio does not)."""
    try:
        src = kernel_source_hash()
        short = workload_name.split(":")[0].strip().replace("-", "_")
        kv = {}
        for line in open(os.path.join(PROFILE_DIR, f"persist_kernel_{short}.txt")):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("kernel_source_sha256_16") != src or kv.get("workload") != workload_name:
            return None
        return float(kv[f"traffic_to_algorithmic[{shape[0]},{shape[1]}]"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples taken during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def unique_bytes_per_generation(run, w: W.Workload, sigma_bytes: int):
    """Algorithmic DRAM bytes of each generation: every distinct parent row and
    every distinct random-tree row read once, every offspring row written
    once, the targets read once (n_cases elements each).  A crossover
    offspring (rt2 = -2 - second parent) reads two parent rows and one
    random-tree row."""
    par, r1, r2, _ = run.trace()
    n = w.n_cases
    out = []
    for g in range(par.shape[0]):
        mut = (r1[g] >= 0) & (r2[g] >= 0)
        cross = (r1[g] >= 0) & (r2[g] <= -2)
        u_p = len(np.unique(np.concatenate([par[g][mut | cross], -2 - r2[g][cross]])))
        u_r = len(np.unique(np.concatenate([r1[g][mut | cross], r2[g][mut]])))
        out.append((u_p + w.pop_size) * n * 4 + u_r * n * sigma_bytes + n * 4)
    return np.array(out, dtype=np.float64)


def resolve_workload(args) -> W.Workload:
    """The workload named on the command line with its overrides."""
    w = W.WORKLOADS[args.workload]
    if args.generations:
        w = w.replace(generations=args.generations)
    if args.pop_size:     # smaller pools of the same shape, e.g. for ncu captures
        w = w.replace(pop_size=args.pop_size, n_random_trees=args.pop_size,
                      name=f"{w.name.split(':')[0]} with m = r = {args.pop_size}")
    if args.p_crossover > 0:
        w = w.replace(p_crossover=args.p_crossover,
                      name=f"{w.name} with crossover p = {args.p_crossover}")
    return w


def run_ours(args, rank, world, local_rank):
    import torch

    import paper_2106_04034_gb300 as pkg
    from paper_2106_04034_gb300.build import build_library

    torch.cuda.set_device(local_rank)
    build_library()
    w = replica_workload(resolve_workload(args), rank)
    G = w.generations
    data = W.make_data(w)
    Xtr, ytr, Xte, yte = data
    dev = [torch.from_numpy(a).cuda() for a in data]
    stream = torch.cuda.current_stream()
    run = pkg.Run(make_config(pkg, w, stream))
    if args.shape:
        vec, opb = (int(v) for v in args.shape.split(","))
        run.set_evolve_shape(pkg.PATH_PERSISTENT, vec, opb)
    y_pred = torch.zeros(w.n_test, dtype=torch.float64, device="cuda")

    def step():
        run.load_device(*dev)
        run.init()
        run.evolve(G, log=False)
        if not w.p_crossover:   # a run with crossover predicts by replaying its trace
            run.best_trace()
        run.predict_device(dev[2], y_pred)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()
    run.set_kernel_timing(True)
    launches0 = run.info().kernel_launches
    clocks = ClockSampler(local_rank)
    clocks.start()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    barrier()
    clock = clocks.stop()
    kernel_ms = [run.kernel_times(1 << 22)]
    interp_ms = run.init_kernel_times()          # the last step's two interpreter launches
    launches = run.info().kernel_launches - launches0
    ms_total = e0.elapsed_time(e1)
    run.set_kernel_timing(False)
    ms_total = max_over_ranks(ms_total, world)
    ms_step = ms_total / args.steps
    updates = float(w.pop_size) * w.n_cases * G
    value = job_value(updates, world, ms_step / 1e3)

    # roofline of the generation kernel: algorithmic bytes / measured duration.
    # The persistent kernel runs up to `per` generations per launch; the
    # chained path's stream kernel one generation per launch.
    info = run.info()
    per = info.evolve_generations_per_launch
    kname = "persist_kernel" if info.evolve_path == 1 else "stream_kernel"
    sig_b = 2 if w.sigma_bf16 else 4
    ub = unique_bytes_per_generation(run, w, sig_b)
    bounds = list(range(0, G, per)) + [G]
    per_launch = np.array([ub[a:b].sum() for a, b in zip(bounds[:-1], bounds[1:])])
    kms = np.concatenate(kernel_ms)
    assert kms.size == per_launch.size * args.steps, (kms.size, per_launch.size)
    total_bytes = float(per_launch.sum()) * args.steps
    avg_bytes = total_bytes / kms.size
    avg_ms = float(kms.mean())
    achieved = total_bytes / (float(kms.sum()) / 1e3) / 1e9
    peak, peak_kind = measured_peak_gbs()
    ratio = profiled_traffic(w.name, (info.evolve_tile_cases // 1024,
                                      info.evolve_offspring_per_cta))
    traffic = None if ratio is None else ratio * avg_bytes
    stream_roofline = {
        "kernel": kname, "bound": "hbm", "achieved": achieved, "peak": peak,
        "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
        "algorithmic_bytes_per_launch": avg_bytes, "avg_launch_ms": avg_ms,
        "launches_timed": int(kms.size), "generations_per_launch": per,
        "shape": {"path": "persistent" if info.evolve_path == 1 else "chained",
                  "tile_cases": info.evolve_tile_cases,
                  "offspring_per_cta": info.evolve_offspring_per_cta,
                  "grid": info.evolve_grid}}

    # the interpreter (ComputeSemantics of P and R): one gene applied to one
    # case is the unit of work, one lane operation at the least, against the
    # FP32 lanes' issue rate (152 SMs x 128 lanes x clock)
    # (the evaluated genes: for linear genomes the live code, the expression
    # under register Out; generated trees are evaluated whole)
    info_i = run.info()
    gene_cases = float(info_i.pop_evaluated_genes + info_i.rt_evaluated_genes) * w.n_cases
    genome_cases = float(sum(run.programs(pool)[2].sum()
                             for pool in (pkg.POOL_POPULATION, pkg.POOL_RANDOM))) * w.n_cases
    interp_s = float(interp_ms.sum()) / 1e3
    alu_peak = alu_peak_tops()
    interp_tops = gene_cases / interp_s / 1e12
    interp_roofline = {
        "kernel": "interpret_kernel", "bound": "alu", "achieved": interp_tops,
        "peak": alu_peak, "peak_kind": "derived: 152 SMs x 128 FP32 lanes x max SM clock",
        "unit": "T lane-ops/s (1 per evaluated gene per case)", "frac": interp_tops / alu_peak,
        "traffic": None, "evaluated_gene_cases_per_init": gene_cases,
        "genome_gene_cases_per_init": genome_cases,
        "launch_ms": [float(v) for v in interp_ms]}
    # the dominant kernel of a step carries the headline roofline
    stream_ms_step = float(kms.sum()) / args.steps
    roofline = interp_roofline if float(interp_ms.sum()) > stream_ms_step else stream_roofline
    secondary = stream_roofline if roofline is interp_roofline else interp_roofline

    # end to end through host buffers: host->device copies of the cases from
    # pinned host memory, the whole run, prediction copied back to the host
    pinned = [torch.from_numpy(a).pin_memory() for a in (Xtr, ytr, Xte, yte)]
    hXtr, hytr, hXte, hyte = (t.numpy() for t in pinned)

    def step_host():
        run.load(hXtr, hytr, hXte, hyte)
        run.init()
        run.evolve(G, log=False)
        if not w.p_crossover:
            run.best_trace()
        return run.predict(hXte)

    step_host()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step_host()
    barrier()
    e2e_s = (time.perf_counter() - t0) / args.steps
    e2e_s = max_over_ranks(e2e_s, world)
    h2d = Xtr.nbytes + ytr.nbytes + Xte.nbytes + yte.nbytes + Xte.nbytes
    d2h = w.n_test * 8
    F_tr, F_te = run.fitness()
    best = int(np.argmin(F_tr))
    run.close()

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "pop_size": w.pop_size,
                   "n_random_trees": w.n_random_trees, "n_features": w.n_features,
                   "n_train": w.n_train, "n_test": w.n_test, "generations": G,
                   "tournament_size": w.tournament_size, "ms": w.ms,
                   "sigma": "bf16" if w.sigma_bf16 else "f32",
                   "programs": (f"linear genomes of {w.max_genes} genes" if w.init_mode == 1
                                else f"ramped half-and-half trees, depth {w.pop_min_depth}-"
                                     f"{w.pop_max_depth}"),
                   "parallelism": f"replicas x{world}",
                   "l2": "working set larger than L2 (semantic matrices %.0f MB)"
                         % ((2 * w.pop_size + w.n_random_trees) * w.n_cases * 4 / 1e6),
                   "step": ("load_device + init + evolve(G) + predict(test) by trace replay"
                            if w.p_crossover else
                            "load_device + init + evolve(G) + best_trace + predict(test)")},
        "roofline": roofline,
        "roofline_other": secondary,
        "e2e": {"value": job_value(updates, world, e2e_s), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "clocks": clock,
        "best_rmse": {"train": float(F_tr[best]), "test": float(F_te[best])},
    }
    return line, w


def make_config(pkg, w: W.Workload, stream):
    cfg = pkg.default_config(
        seed=w.seed, run=w.run, pop_size=w.pop_size, n_random_trees=w.n_random_trees,
        pop_min_depth=w.pop_min_depth, pop_max_depth=w.pop_max_depth,
        rt_min_depth=w.rt_min_depth, rt_max_depth=w.rt_max_depth, ms=w.ms,
        tournament_size=w.tournament_size, const_lo=w.const_lo, const_hi=w.const_hi,
        protect_eps=w.protect_eps,
        sigma_dtype=pkg.SIGMA_BF16 if w.sigma_bf16 else pkg.SIGMA_F32,
        init_mode=w.init_mode, max_genes=w.max_genes, p_crossover=w.p_crossover)
    cfg.stream = stream.cuda_stream
    return cfg


BATCH_RUNS = 48


def run_batched(args, rank, world, local_rank):
    """48 independent runs of uneven shapes: one step = every run staged,
    initialised, evolved G generations by the batched kernel (one
    cooperative launch per 64 generations of all runs), its best model
    rebuilt and applied to its test cases.  The same runs executed one after
    another through the single-run path are timed alongside."""
    import torch

    import paper_2106_04034_gb300 as pkg
    from paper_2106_04034_gb300.build import build_library

    torch.cuda.set_device(local_rank)
    build_library()
    G = args.generations or 500
    nruns = args.batch_runs
    ws = [replica_workload(w, 1000 * rank)
          for w in W.batched_runs(nruns, generations=G, max_train=args.max_train or None)]
    datas = [W.make_data(w) for w in ws]
    devs = [[torch.from_numpy(a).cuda() for a in d] for d in datas]
    stream = torch.cuda.current_stream()
    runs = [pkg.Run(make_config(pkg, w, stream)) for w in ws]
    for r, d in zip(runs, devs):
        r.load_device(*d)
        r.init()
    batch = pkg.Batch(runs)
    if args.shape:
        batch.set_shape(*(int(v) for v in args.shape.split(",")))
    y_pred = [torch.zeros(max(w.n_test, 1), dtype=torch.float64, device="cuda") for w in ws]

    def finish():
        for r, d, y in zip(runs, devs, y_pred):
            r.best_trace()
            r.predict_device(d[2], y)

    # CUDA events around the evolution alone (the per-run staging, init and
    # finishing are the same work in both forms)
    evolve_ev = {"batched": [], "sequential": []}

    def mark():
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e

    def step():
        for r, d in zip(runs, devs):
            r.load_device(*d)
            r.init()
        e = mark()
        batch.evolve(G, log=False)
        evolve_ev["batched"].append([(e, mark())])
        finish()

    def step_sequential():
        pairs = []
        for r, d in zip(runs, devs):
            r.load_device(*d)
            r.init()
            e = mark()
            r.evolve(G, log=False)
            pairs.append((e, mark()))
        evolve_ev["sequential"].append(pairs)
        finish()

    def evolve_ms(kind, steps):
        torch.cuda.synchronize()
        last = evolve_ev[kind][-steps:]
        return sum(a.elapsed_time(b) for pairs in last for a, b in pairs) / len(last)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def timed(fn, steps):
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1)
        ms = max_over_ranks(ms, world)
        return ms / steps

    for _ in range(args.warmup):
        step()
    batch.set_kernel_timing(True)
    launches0 = batch.info().kernel_launches + sum(r.info().kernel_launches for r in runs)
    clocks = ClockSampler(local_rank)
    clocks.start()
    ms_step = timed(step, args.steps)
    clock = clocks.stop()
    kms = batch.kernel_times(1 << 20)
    batch.set_kernel_timing(False)
    launches = batch.info().kernel_launches + sum(r.info().kernel_launches for r in runs) - launches0
    updates = float(sum(w.pop_size * w.n_cases for w in ws)) * G
    value = job_value(updates, world, ms_step / 1e3)

    # roofline of the batched kernel: algorithmic bytes of every run's
    # generations (distinct parents and random trees read once, offspring
    # written once, targets once) per launch of up to 64 generations
    info = batch.info()
    per = info.generations_per_launch
    ub = sum(unique_bytes_per_generation(r, w, 2 if w.sigma_bf16 else 4)
             for r, w in zip(runs, ws))
    bounds = list(range(0, G, per)) + [G]
    per_launch = np.array([ub[a:b].sum() for a, b in zip(bounds[:-1], bounds[1:])])
    assert kms.size == per_launch.size * args.steps, (kms.size, per_launch.size)
    total_bytes = float(per_launch.sum()) * args.steps
    achieved = total_bytes / (float(kms.sum()) / 1e3) / 1e9
    peak, peak_kind = measured_peak_gbs()

    # the same runs one after another through the single-run path
    step_sequential()                       # autotunes each run's layout once
    seq_steps = max(1, min(args.steps, 2))
    ms_seq = timed(step_sequential, seq_steps)
    value_seq = job_value(updates, world, ms_seq / 1e3)
    evolve_batched_ms = evolve_ms("batched", args.steps)
    evolve_sequential_ms = evolve_ms("sequential", seq_steps)

    # end to end through host buffers (pinned host memory)
    hdatas = [[torch.from_numpy(a).pin_memory().numpy() for a in d] for d in datas]

    def step_host():
        for r, d in zip(runs, hdatas):
            r.load(*d)
            r.init()
        batch.evolve(G, log=False)
        return [r.predict(d[2]) for r, d in zip(runs, hdatas)]

    e2e_s = float("nan")
    if not getattr(args, "skip_e2e", False):
        step_host()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step_host()
        barrier()
        e2e_s = (time.perf_counter() - t0) / args.steps
        e2e_s = max_over_ranks(e2e_s, world)
    h2d = sum(sum(a.nbytes for a in d) + d[2].nbytes for d in datas)
    d2h = sum(w.n_test * 8 for w in ws)
    batch.close()
    for r in runs:
        r.close()

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batched: {nruns} runs, n_train log-uniform 1e3-2e5"
                               + (f" capped at {args.max_train}" if args.max_train else "")
                               + f", n_test = n_train/4, l 5-100, m 256-2048, r 256-1024, "
                               f"depth 2-6, G={G}",
                   "runs": nruns, "generations": G,
                   "updates_per_generation": updates / G,
                   "parallelism": f"replicas x{world}",
                   "l2": "working set larger than L2 (%.1f GB of semantic rows)"
                         % (sum((2 * w.pop_size + w.n_random_trees) * w.n_cases * 4
                                for w in ws) / 1e9),
                   "step": "per run load_device + init; batched evolve(G); per run "
                           "best_trace + predict(test)"},
        "sequential": {"value": value_seq, "unit": UNIT, "ms_per_step": ms_seq,
                       "steps": seq_steps,
                       "what": "the same runs one after another through gsgp_evolve"},
        "evolve_only": {"batched_ms": evolve_batched_ms, "sequential_ms": evolve_sequential_ms,
                        "speedup": evolve_sequential_ms / evolve_batched_ms,
                        "what": "CUDA-event time of batch.evolve(G) against the sum of the "
                                "runs' gsgp_evolve(G), within the same timed steps"},
        "roofline": {"kernel": "batch_kernel", "bound": "hbm", "achieved": achieved,
                     "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None,
                     "algorithmic_bytes_per_launch": total_bytes / kms.size,
                     "avg_launch_ms": float(kms.mean()), "launches_timed": int(kms.size),
                     "generations_per_launch": per,
                     "shape": {"tile_cases": info.tile_cases,
                               "offspring_per_cta": info.offspring_per_cta,
                               "grid": info.grid, "graph": bool(info.graph)}},
        "e2e": {"value": job_value(updates, world, e2e_s), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "clocks": clock,
    }
    return line, ws


# The oracle keeps every semantic row of a run in float64 host memory; the
# large workloads (1.25M cases: about 25 GB) are sampled by their cases.
ORACLE_MAX_CASES = 100_000
ORACLE_CASE_FRACTION = 64


def oracle_sample(w: W.Workload, data=None):
    """(data, note) for the oracle on workload w: every case when the
    workload has at most ORACLE_MAX_CASES, else a seeded subset of
    1/ORACLE_CASE_FRACTION of its training and of its test cases (fitness
    cases are independent columns of every step but the RMSE sums, so the
    per-update work is that of the full workload)."""
    if data is None:
        data = W.make_data(w)
    n = int(data[1].shape[0] + data[3].shape[0])
    if n <= ORACLE_MAX_CASES:
        return data, (f"full n_cases={n}" if n == w.n_cases else f"{n} sampled cases")
    rng = np.random.default_rng([w.seed, w.wid, w.run, ORACLE_CASE_FRACTION])
    itr = np.sort(rng.choice(w.n_train, max(1, w.n_train // ORACLE_CASE_FRACTION), replace=False))
    ite = np.sort(rng.choice(w.n_test, w.n_test // ORACLE_CASE_FRACTION, replace=False)) \
        if w.n_test else np.zeros(0, np.int64)
    sub = (np.ascontiguousarray(data[0][itr]), np.ascontiguousarray(data[1][itr]),
           np.ascontiguousarray(data[2][ite]), np.ascontiguousarray(data[3][ite]))
    return sub, (f"seeded 1/{ORACLE_CASE_FRACTION} case subset: {len(itr)} + {len(ite)} of "
                 f"{w.n_train} + {w.n_test} cases")


def oracle_run(w: W.Workload, data=None):
    """The float64 oracle initialised on workload w, or on a sample of it:
    the cases of large workloads are sampled (oracle_sample); where the
    oracle's initialisation would take many minutes (long linear genomes)
    every case is kept but at most 128 programs per pool.  Returns (oracle,
    the workload it runs, the number of cases it holds, a note on the
    sample)."""
    from oracle import gsgp as og
    full_m = w.pop_size
    big = w.init_mode == 1 and w.pop_size * w.n_cases * w.max_genes > 2e10
    if big:
        w = w.replace(pop_size=min(w.pop_size, 128), n_random_trees=min(w.n_random_trees, 128))
    sub, note = oracle_sample(w, data)
    p = og.Params(seed=w.seed, run=w.run, pop_size=w.pop_size,
                  n_random_trees=w.n_random_trees, pop_min_depth=w.pop_min_depth,
                  pop_max_depth=w.pop_max_depth, rt_min_depth=w.rt_min_depth,
                  rt_max_depth=w.rt_max_depth, ms=w.ms, tournament_size=w.tournament_size,
                  const_lo=w.const_lo, const_hi=w.const_hi, protect_eps=w.protect_eps,
                  sigma_bf16=w.sigma_bf16, init_mode=w.init_mode, max_genes=w.max_genes,
                  p_crossover=w.p_crossover)
    o = og.GSGP(p, *sub)
    o.init()
    n = int(sub[1].shape[0] + sub[3].shape[0])
    if big:
        note += f", m and r cut from {full_m} to {w.pop_size}"
    return o, w, n, note


def _oracle_worker(w, sub, target_s, barrier, out):
    """One all-core leg process: an independent oracle run (its own run
    index) on the sampled cases, timed for about target_s seconds after
    every process has finished its initialisation."""
    o, w, n, _ = oracle_run(w, sub)
    barrier.wait()
    t0 = time.perf_counter()
    gens = 0
    while (time.perf_counter() - t0) < target_s:
        o.generation()
        gens += 1
    out.put((w.pop_size * n * gens, t0, time.perf_counter()))


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            k, _, v = line.partition(":")
            if k.strip() in ("model name", "CPU part", "Model"):
                return v.strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(w: W.Workload, target_s: float = 10.0, max_gens: int = 200):
    """The float64 oracle, as it stands, on the host cores: (1) one process,
    generations of the workload (cases sampled where it is large) until
    about target_s seconds were timed; (2) every host core: one independent
    oracle run per core (its own run index, one numpy thread each) on the
    same sampled cases, timed together for about target_s seconds.  value is
    the all-core rate; the single-thread rate is reported beside it."""
    import multiprocessing as mp
    data = W.make_data(w)
    o, wo, n, note = oracle_run(w, data)
    t0 = time.perf_counter()
    gens = 0
    while gens < max_gens and (time.perf_counter() - t0) < target_s:
        o.generation()
        gens += 1
    dt = time.perf_counter() - t0
    single = wo.pop_size * n * gens / dt
    del o
    sub, _ = oracle_sample(w, data)
    del data
    cores = cpu_cores()
    env_keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                               "MKL_NUM_THREADS")}
    for k in env_keep:
        os.environ[k] = "1"
    ctx = mp.get_context("spawn")   # never fork a process that has used the GPU
    barrier = ctx.Barrier(cores)
    out = ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker,
                         args=(w.replace(run=w.run + 1 + k), sub, target_s, barrier, out))
             for k in range(cores)]
    for pr in procs:
        pr.start()
    res = [out.get() for _ in procs]
    for pr in procs:
        pr.join()
    for k, v in env_keep.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v
    upd = sum(r[0] for r in res)
    span = max(r[2] for r in res) - min(r[1] for r in res)
    allcore = upd / span
    return {"value": allcore, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{w.name.split(':')[0]} workload, {note}, m={wo.pop_size}; float64 numpy; "
                      f"all-core leg: {cores} processes, one independent oracle run each (own "
                      f"run index, one numpy thread), timed together for ~{target_s:.0f} s "
                      f"after an untimed init; CPU: {cpu_model()}",
            "single_thread": {"value": single, "unit": UNIT, "cores": 1,
                              "sample": f"{gens} generations in one process after an untimed "
                                        f"init"}}


def run_reference(args, rank):
    """The CPU oracle as the reference arm: each step a bounded sample of the
    same workload (a few generations of the oracle after an untimed init)."""
    if args.workload == "batched":   # the smallest run of the batch
        w = min(W.batched_runs(args.batch_runs), key=lambda x: x.pop_size * x.n_cases)
    else:
        w = resolve_workload(args)
    o, w, n, note = oracle_run(w)
    gens_per_step = max(1, int(args.ref_gens_per_step))
    for _ in range(args.warmup):
        for _ in range(gens_per_step):
            o.generation()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for _ in range(gens_per_step):
            o.generation()
    dt = time.perf_counter() - t0
    gens = gens_per_step * args.steps
    value = w.pop_size * n * gens / dt
    sample = (f"{gens_per_step} oracle generations per step of the {w.name.split(':')[0]} "
              f"workload ({note}, m={w.pop_size}), float64 numpy, one process; the rate "
              f"counts offspring x cases x generations actually computed")
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": w.name, "pop_size": w.pop_size, "n_cases": w.n_cases,
                   "oracle_cases": n, "generations_per_step": gens_per_step},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def time_run(w: W.Workload, data, steps: int = 1, warmup_gens: int = 64):
    """One workload on this GPU through the same step as the headline
    (load_device + init + evolve(G) + best_trace + predict(test)): the
    autotuner's choice is made on an untimed warm-up of warmup_gens
    generations; then `steps` timed steps.  Returns updates/s, ms per step,
    the stream kernel's fraction of the measured HBM peak and its shape."""
    import torch

    import paper_2106_04034_gb300 as pkg
    dev = [torch.from_numpy(a).cuda() for a in data]
    stream = torch.cuda.current_stream()
    run = pkg.Run(make_config(pkg, w, stream))
    y = torch.zeros(max(w.n_test, 1), dtype=torch.float64, device="cuda")
    run.load_device(*dev)
    run.init()
    run.evolve(min(warmup_gens, w.generations), log=False)

    def step():
        run.load_device(*dev)
        run.init()
        run.evolve(w.generations, log=False)
        run.best_trace()
        run.predict_device(dev[2], y)

    torch.cuda.synchronize()
    run.set_kernel_timing(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    kms = run.kernel_times(1 << 22)
    interp_ms = run.init_kernel_times()          # the last step's two interpreter launches
    run.set_kernel_timing(False)
    ms = e0.elapsed_time(e1) / steps
    info = run.info()
    gene_cases = float(info.pop_evaluated_genes + info.rt_evaluated_genes) * w.n_cases
    interp_tops = gene_cases / (float(interp_ms.sum()) / 1e3) / 1e12
    ub = unique_bytes_per_generation(run, w, 2 if w.sigma_bf16 else 4)
    per = info.evolve_generations_per_launch
    bounds = list(range(0, w.generations, per)) + [w.generations]
    per_launch = np.array([ub[a:b].sum() for a, b in zip(bounds[:-1], bounds[1:])])
    achieved = float(per_launch.sum()) * steps / (float(kms.sum()) / 1e3) / 1e9
    peak, _ = measured_peak_gbs()
    run.close()
    return {"value": float(w.pop_size) * w.n_cases * w.generations / (ms / 1e3), "unit": UNIT,
            "ms_per_step": ms, "steps": steps, "generations": w.generations,
            "stream_frac_of_measured_hbm": achieved / peak,
            "shape": [info.evolve_tile_cases // 1024, info.evolve_offspring_per_cta],
            "interpreter": {"launch_ms": [float(v) for v in interp_ms],
                            "achieved": interp_tops, "peak": alu_peak_tops(),
                            "unit": "T lane-ops/s (1 per evaluated gene per case)",
                            "frac": interp_tops / alu_peak_tops()}}


def measure_variants(args):
    """The other workloads of the benchmark on the same GPU as the headline
    (one timed step each after an untimed autotuning warm-up), so that their
    comparisons are made on one machine: the tiny workload (C1, latency-
    bound, 20 steps); the mid workload (C2); the
    precision variant (large workload, G = 2000, sigma(R) stored bf16)
    against the same run with float32 sigma on the same data (C4); 48
    batched runs against the same runs evolved one after another (C5); the
    paper's speed-up shape with genomes of 2047 genes, where the interpreter
    (ComputeSemantics) takes half of the step."""
    out = {}
    tiny = W.TINY
    out["tiny"] = time_run(tiny, W.make_data(tiny), steps=20)
    out["tiny"]["workload"] = tiny.name
    mid = W.MID
    out["mid"] = time_run(mid, W.make_data(mid), steps=3)
    out["mid"]["workload"] = mid.name
    big = W.LARGE.replace(generations=2000)
    data = W.make_data(big)
    f32 = time_run(big, data)
    bf16 = time_run(W.LARGE_BF16, data)
    out["large_bf16"] = {"workload": W.LARGE_BF16.name, "bf16_sigma": bf16, "f32_sigma": f32,
                         "speedup_bf16_over_f32": bf16["value"] / f32["value"]}
    del data
    pk = W.PAPER_K2047
    out["paper_k2047"] = time_run(pk, W.make_data(pk))
    out["paper_k2047"]["workload"] = pk.name
    bargs = argparse.Namespace(**vars(args))
    bargs.steps, bargs.warmup, bargs.shape, bargs.generations = 1, 1, "", 0
    bargs.skip_e2e = True
    line, _ = run_batched(bargs, 0, 1, 0)
    out["batched"] = {"workload": line["config"]["workload"], "value": line["value"],
                      "unit": UNIT, "ms_per_step": line["ms_per_step"],
                      "sequential": line["sequential"],
                      "speedup_batched_over_sequential":
                          line["value"] / line["sequential"]["value"],
                      "evolve_only": line["evolve_only"],
                      "stream_frac_of_measured_hbm": line["roofline"]["frac"],
                      "shape": line["roofline"]["shape"]}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large", choices=sorted(W.WORKLOADS) + ["batched"])
    ap.add_argument("--generations", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-gens-per-step", type=int, default=3)
    ap.add_argument("--pop-size", type=int, default=0,
                    help="m = r override (smaller cases of a workload, e.g. for ncu captures)")
    ap.add_argument("--p-crossover", type=float, default=0.0,
                    help="probability of geometric semantic crossover (default 0)")
    ap.add_argument("--shape", default="",
                    help="vec,opb of the mutation stream instead of autotuning (e.g. 2,4)")
    ap.add_argument("--batch-runs", type=int, default=BATCH_RUNS,
                    help="runs of the batched workload")
    ap.add_argument("--max-train", type=int, default=0,
                    help="cap on n_train of the batched workload's runs (0: none)")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the mid / bf16 / batched comparison runs of the default workload")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return 0
        print(json.dumps(run_reference(args, rank)), flush=True)
        return 0

    if world > 1:
        import torch

        from paper_2106_04034_gb300.build import build_library
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
        # one process per node builds (or finds current) the library before
        # the others load it
        if local_rank == 0:
            build_library()
        torch.distributed.barrier()
    if args.workload == "batched":
        line, ws = run_batched(args, rank, world, local_rank)
        # the oracle on the smallest run of the batch
        w = min(ws, key=lambda x: x.pop_size * x.n_cases).replace(run=0)
    else:
        line, w = run_ours(args, rank, world, local_rank)
        if (world == 1 and args.workload == "large" and not args.no_variants
                and not args.generations and not args.pop_size and not args.shape
                and not args.p_crossover):
            line["variants"] = measure_variants(args)
    if rank == 0:
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(w.replace(run=0))
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
