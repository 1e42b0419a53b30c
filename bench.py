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

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload mid]
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
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "persist_kernel_mid.txt")
GEN_KERNEL_SRC = [os.path.join(ROOT, "paper_2106_04034_gb300", "csrc", f)
                  for f in ("k_persist.cu", "k_generation.cu", "stream.cuh", "common.cuh")]


def measured_peak_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def profiled_traffic(workload_name: str):
    """DRAM bytes per generation of the generation kernel from the committed
    ncu summary, if it was taken on this workload with the current kernel
    sources (else None)."""
    try:
        h = hashlib.sha256()
        for f in GEN_KERNEL_SRC:
            h.update(open(f, "rb").read())
        src = h.hexdigest()[:16]
        kv = {}
        for line in open(PROFILE_SUMMARY):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("kernel_source_sha256_16") != src or kv.get("workload") != workload_name:
            return None
        return float(kv["traffic_bytes_per_generation"])
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
    once, the targets read once (n_cases elements each)."""
    par, r1, r2, _ = run.trace()
    n = w.n_cases
    out = []
    for g in range(par.shape[0]):
        mut = r1[g] >= 0
        u_p = len(np.unique(par[g][mut]))
        u_r = len(np.unique(np.concatenate([r1[g][mut], r2[g][mut]])))
        out.append((u_p + w.pop_size) * n * 4 + u_r * n * sigma_bytes + n * 4)
    return np.array(out, dtype=np.float64)


def run_ours(args, rank, world, local_rank):
    import torch

    import paper_2106_04034_gb300 as pkg
    from paper_2106_04034_gb300.build import build_library

    torch.cuda.set_device(local_rank)
    build_library()
    w = W.WORKLOADS[args.workload]
    if args.generations:
        w = w.replace(generations=args.generations)
    w = w.replace(run=rank)
    G = w.generations
    data = W.make_data(w)
    Xtr, ytr, Xte, yte = data
    dev = [torch.from_numpy(a).cuda() for a in data]
    stream = torch.cuda.current_stream()
    cfg = pkg.default_config(
        seed=w.seed, run=w.run, pop_size=w.pop_size, n_random_trees=w.n_random_trees,
        pop_min_depth=w.pop_min_depth, pop_max_depth=w.pop_max_depth,
        rt_min_depth=w.rt_min_depth, rt_max_depth=w.rt_max_depth, ms=w.ms,
        tournament_size=w.tournament_size, const_lo=w.const_lo, const_hi=w.const_hi,
        protect_eps=w.protect_eps,
        sigma_dtype=pkg.SIGMA_BF16 if w.sigma_bf16 else pkg.SIGMA_F32)
    cfg.stream = stream.cuda_stream
    run = pkg.Run(cfg)
    y_pred = torch.zeros(w.n_test, dtype=torch.float64, device="cuda")

    def step():
        run.load_device(*dev)
        run.init()
        run.evolve(G, log=False)
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
    launches = run.info().kernel_launches - launches0
    ms_total = e0.elapsed_time(e1)
    run.set_kernel_timing(False)
    if world > 1:
        t = torch.tensor([ms_total], device="cuda", dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_total = float(t.item())
    ms_step = ms_total / args.steps
    updates = float(w.pop_size) * w.n_cases * G
    value = updates * world / (ms_step / 1e3)

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
    per_gen_traffic = profiled_traffic(w.name)
    traffic = None if per_gen_traffic is None else per_gen_traffic * G / per_launch.size

    # end to end through host buffers: host->device copies of the cases,
    # the whole run, prediction copied back to the host
    def step_host():
        run.load(Xtr, ytr, Xte, yte)
        run.init()
        run.evolve(G, log=False)
        run.best_trace()
        return run.predict(Xte)

    step_host()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step_host()
    barrier()
    e2e_s = (time.perf_counter() - t0) / args.steps
    if world > 1:
        t = torch.tensor([e2e_s], device="cuda", dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_s = float(t.item())
    h2d = Xtr.nbytes + ytr.nbytes + Xte.nbytes + yte.nbytes + Xte.nbytes
    d2h = w.n_test * 8
    bt = run.best_trace()
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
                   "parallelism": f"replicas x{world}",
                   "l2": "working set larger than L2 (semantic matrices %.0f MB)"
                         % ((2 * w.pop_size + w.n_random_trees) * w.n_cases * 4 / 1e6),
                   "step": "load_device + init + evolve(G) + best_trace + predict(test)"},
        "roofline": {"kernel": kname, "bound": "hbm", "achieved": achieved,
                     "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "algorithmic_bytes_per_launch": avg_bytes,
                     "avg_launch_ms": avg_ms, "launches_timed": int(kms.size),
                     "generations_per_launch": per,
                     "shape": {"path": "persistent" if info.evolve_path == 1 else "chained",
                               "tile_cases": info.evolve_tile_cases,
                               "offspring_per_cta": info.evolve_offspring_per_cta,
                               "grid": info.evolve_grid}},
        "e2e": {"value": updates * world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "clocks": clock,
        "best_rmse": {"train": bt["best_train_rmse"], "test": bt["best_test_rmse"]},
    }
    return line, w


def cpu_baseline(w: W.Workload, target_s: float = 12.0, max_gens: int = 200):
    """The float64 oracle, as it stands, on the host cores: generations of the
    same workload until about target_s seconds of evolution were timed."""
    from oracle import gsgp as og
    p = og.Params(seed=w.seed, run=w.run, pop_size=w.pop_size,
                  n_random_trees=w.n_random_trees, pop_min_depth=w.pop_min_depth,
                  pop_max_depth=w.pop_max_depth, rt_min_depth=w.rt_min_depth,
                  rt_max_depth=w.rt_max_depth, ms=w.ms, tournament_size=w.tournament_size,
                  const_lo=w.const_lo, const_hi=w.const_hi, protect_eps=w.protect_eps,
                  sigma_bf16=w.sigma_bf16)
    o = og.GSGP(p, *W.make_data(w))
    o.init()
    t0 = time.perf_counter()
    gens = 0
    while gens < max_gens and (time.perf_counter() - t0) < target_s:
        o.generation()
        gens += 1
    dt = time.perf_counter() - t0
    return {"value": w.pop_size * w.n_cases * gens / dt, "unit": UNIT, "cores": 1,
            "kind": "oracle",
            "sample": f"{gens} generations of the {w.name.split(':')[0]} workload "
                      f"(full n_cases={w.n_cases}, m={w.pop_size}) after an untimed init; "
                      f"float64 numpy, single thread, {os.cpu_count()} host cores present"}


def run_reference(args, rank):
    """The CPU oracle as the reference arm: each step a bounded sample of the
    same workload (a few generations of the oracle after an untimed init)."""
    from oracle import gsgp as og
    w = W.WORKLOADS[args.workload]
    if args.generations:
        w = w.replace(generations=args.generations)
    p = og.Params(seed=w.seed, run=w.run, pop_size=w.pop_size,
                  n_random_trees=w.n_random_trees, pop_min_depth=w.pop_min_depth,
                  pop_max_depth=w.pop_max_depth, rt_min_depth=w.rt_min_depth,
                  rt_max_depth=w.rt_max_depth, ms=w.ms, tournament_size=w.tournament_size,
                  const_lo=w.const_lo, const_hi=w.const_hi, protect_eps=w.protect_eps,
                  sigma_bf16=w.sigma_bf16)
    o = og.GSGP(p, *W.make_data(w))
    o.init()
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
    value = w.pop_size * w.n_cases * gens / dt
    sample = (f"{gens_per_step} oracle generations per step of the {w.name.split(':')[0]} "
              f"workload (full n_cases={w.n_cases}, m={w.pop_size}), float64 numpy, single thread")
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": w.name, "pop_size": w.pop_size, "n_cases": w.n_cases,
                   "generations_per_step": gens_per_step},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mid", choices=sorted(W.WORKLOADS))
    ap.add_argument("--generations", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-gens-per-step", type=int, default=3)
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
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    line, w = run_ours(args, rank, world, local_rank)
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
