"""Helpers for the GPU parity tests: build a library run and the matching
oracle run from one workload description."""
from __future__ import annotations

import numpy as np

import workloads as W
from oracle import gsgp as og
from oracle import interp as oi

SEM_RTOL = 1e-4      # semantics: |gpu - oracle| <= 1e-4 (1 + |v|)
RMSE_RTOL = 1e-5     # RMSE: relative


def oracle_params(w: W.Workload, **over) -> og.Params:
    p = og.Params(seed=w.seed, run=w.run, pop_size=w.pop_size,
                  n_random_trees=w.n_random_trees, pop_min_depth=w.pop_min_depth,
                  pop_max_depth=w.pop_max_depth, rt_min_depth=w.rt_min_depth,
                  rt_max_depth=w.rt_max_depth, const_lo=w.const_lo, const_hi=w.const_hi,
                  protect_eps=w.protect_eps, ms=w.ms, tournament_size=w.tournament_size,
                  sigma_bf16=w.sigma_bf16, init_mode=w.init_mode, max_genes=w.max_genes)
    for k, v in over.items():
        setattr(p, k, v)
    return p


def gpu_run(w: W.Workload, data=None, **over):
    import torch

    import paper_2106_04034_gb300 as pkg
    p = oracle_params(w, **over)
    cfg = pkg.default_config(
        seed=p.seed, run=p.run, pop_size=p.pop_size, n_random_trees=p.n_random_trees,
        pop_min_depth=p.pop_min_depth, pop_max_depth=p.pop_max_depth,
        rt_min_depth=p.rt_min_depth, rt_max_depth=p.rt_max_depth, const_lo=p.const_lo,
        const_hi=p.const_hi, protect_eps=p.protect_eps, ms=p.ms, ms_mode=p.ms_mode,
        tournament_size=p.tournament_size, elitism=int(p.elitism),
        p_grow_function=p.p_grow, p_feature_given_terminal=p.p_feature,
        sigma_dtype=pkg.SIGMA_BF16 if p.sigma_bf16 else pkg.SIGMA_F32,
        init_mode=p.init_mode, max_genes=p.max_genes, p_crossover=p.p_crossover)
    cfg.stream = torch.cuda.current_stream().cuda_stream
    run = pkg.Run(cfg)
    if data is None:
        data = W.make_data(w)
    run.load(*data)
    run.init()
    return run, data, p


# A GPU value outside 1e-4 (1 + |v|) of the exact float64 value passes only
# where the oracle's first-order float32 running error bound of that case is
# finite and the difference is within twice that bound (float32 evaluation of
# a deep program can legitimately lose more than 1e-4 relative, e.g. through
# cancellation or a protected division by a small operand), or where the
# bound is infinite (float32 overflow, or an operand so close to the
# protected-division threshold that float32 and float64 may take different
# branches).  Both shares are limited and reported: at most 1% of the cases
# may be decided by the bound, at most 0.1% may be ambiguous.
BY_BOUND_MAX = 1e-2
AMBIGUOUS_MAX = 1e-3

# (label, cases checked, share decided by the bound, share ambiguous) of every
# bounded comparison of the session, printed in the terminal summary
SHARES = []


def semantics_close(gpu, ref, bound=None, label=None):
    """Element-wise check: within 1e-4 (1 + |v|), or, where a float32 running
    error bound of the exact value is given, within twice that bound (finite
    bound) or excused (infinite bound).  With a bound, the shares of cases
    decided by the bound and of ambiguous cases are recorded under ``label``
    and must stay within BY_BOUND_MAX and AMBIGUOUS_MAX.  Returns (ok mask,
    fraction decided by the bound, fraction excluded as ambiguous)."""
    diff = np.abs(gpu.astype(np.float64) - ref)
    ok = diff <= SEM_RTOL * (1 + np.abs(ref))
    ok |= (gpu == ref)                       # equal infinities
    by_bound = np.zeros_like(ok)
    ambiguous = np.zeros_like(ok)
    if bound is not None:
        fin = np.isfinite(bound)
        by_bound = ~ok & fin & (diff <= 2 * bound)
        ambiguous = ~ok & ~fin
        ok = ok | by_bound | ambiguous
        b, a = float(by_bound.mean()), float(ambiguous.mean())
        SHARES.append((label or "unlabelled", int(ok.size), b, a))
        assert b <= BY_BOUND_MAX, f"{label}: {b:.3e} of the cases decided by the float32 bound"
        assert a <= AMBIGUOUS_MAX, f"{label}: {a:.3e} of the cases ambiguous"
    return ok, by_bound.mean(), ambiguous.mean()


def oracle_semantics_with_bounds(P, X, eps, logistic=False, linear=False):
    genes, consts, lengths = P
    vals, bounds = [], []
    for i in range(genes.shape[0]):
        L = int(lengths[i])
        v, e = oi.eval_postfix_fp32_bound(genes[i, :L], consts[i, :L], X, eps, linear=linear)
        if logistic:
            v = oi.sigma(v)
            e = oi.sigma_fp32_bound(e)
        vals.append(v)
        bounds.append(e)
    return np.stack(vals), np.stack(bounds)


def replay(ref: og.GSGP, trace, G0=0):
    par, r1, r2, ms = trace
    checks = {}
    for g in range(len(par)):
        ref.generation({"parent": par[g], "rt1": r1[g], "rt2": r2[g], "ms": ms[g]}, checks)
    return checks


def hard_failures(checks):
    return {k: v for k, v in checks.items() if not k.endswith("near_tie")}


def f32_program(genes, consts, X, eps):
    """Float32 value of one program on the cases X (features, n): a stack
    machine with the skip rule and the Out register."""
    n = X.shape[1]
    stack, out = [], None
    with np.errstate(all="ignore"):
        for g, c in zip(genes, consts):
            g = int(g)
            if g == -1:
                break
            op = g & 0xFF
            if op == 5:
                stack.append(X[g >> 8])
            elif op == 4:
                stack.append(np.full(n, c, np.float32))
            elif len(stack) >= 2:
                b = stack.pop()
                a = stack.pop()
                if op == 0:
                    r = a + b
                elif op == 1:
                    r = a - b
                elif op == 2:
                    r = a * b
                else:
                    r = np.where(np.abs(b) < eps, np.float32(1), a / b)
                r = r.astype(np.float32)
                stack.append(r)
                out = r
    if out is not None:
        return out
    return stack[-1] if stack else np.zeros(n, np.float32)
