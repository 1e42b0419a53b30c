"""Seeded synthetic inputs for the GSGP symbolic-regression workloads.

This module only draws data: feature matrices, targets and the run shapes of the
batched workload.  It contains none of the GSGP method (no program generation,
no interpreter, no mutation, no fitness): both the CPU oracle and the CUDA path
receive the same arrays from here and compute everything else on their own.

Fitness cases follow the paper's problem statement (Sec. 2): a case is a pair
(x_j, t_j) with x_j in R^l and t_j in R; the data files of the paper's tool hold
one case per row with the target in the last column (Sec. 3.3), so features are
returned row-major, shape (n, l), float32.

All draws use numpy's PCG64 generator keyed by (seed, workload id, run), so a
workload is reproducible on any machine.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np


@dataclasses.dataclass(frozen=True)
class Workload:
    """Shape and evolution parameters of one GSGP run."""

    name: str
    n_features: int
    n_train: int
    n_test: int
    pop_size: int          # m
    n_random_trees: int    # r
    pop_min_depth: int
    pop_max_depth: int
    rt_min_depth: int
    rt_max_depth: int
    generations: int
    ms: float = 0.1
    tournament_size: int = 4
    seed: int = 1
    run: int = 0
    const_lo: float = -1.0
    const_hi: float = 1.0
    protect_eps: float = 1e-3
    sigma_bf16: bool = False
    feature_dist: str = "uniform"   # "uniform" U[-1,1] or "normal" N(0,1)
    target: str = "poly"            # "poly" | "tree5" | "monomials" | "tree4"
    noise: float = 0.0              # standard deviation of the additive noise
    wid: int = 0                    # workload id, mixed into the data seed
    init_mode: int = 0              # 0 ramped half-and-half trees, 1 linear genomes
    max_genes: int = 127            # genome length (init_mode 1)
    p_crossover: float = 0.0        # probability of geometric semantic crossover

    @property
    def n_cases(self) -> int:
        return self.n_train + self.n_test

    def replace(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


# Five workloads of the symbolic-regression problem at increasing scale.
TINY = Workload(
    name="tiny: l=8 U[-1,1], n=256+64, m=128, r=256, depth 2-4, G=50",
    n_features=8, n_train=256, n_test=64, pop_size=128, n_random_trees=256,
    pop_min_depth=2, pop_max_depth=4, rt_min_depth=2, rt_max_depth=4,
    generations=50, target="poly", noise=0.01, wid=0)

MID = Workload(
    name="mid: l=64 U[-1,1], n=20000+5000, m=1024, r=1024, depth 2-6, G=1000",
    n_features=64, n_train=20000, n_test=5000, pop_size=1024, n_random_trees=1024,
    pop_min_depth=2, pop_max_depth=6, rt_min_depth=2, rt_max_depth=6,
    generations=1000, target="tree5", noise=0.05, wid=1)

LARGE = Workload(
    name="large: l=128 N(0,1), n=1000000+250000, m=1024, r=512, depth 2-6, G=200",
    n_features=128, n_train=1_000_000, n_test=250_000, pop_size=1024,
    n_random_trees=512, pop_min_depth=2, pop_max_depth=6, rt_min_depth=2,
    rt_max_depth=6, generations=200, feature_dist="normal", target="monomials",
    noise=0.1, wid=2)

# The precision variant: the same data, programs and draws as LARGE, only
# sigma(R) stored as bf16, over 2000 generations.
LARGE_BF16 = LARGE.replace(
    name="large-bf16: LARGE with sigma(R) stored bf16, G=2000",
    generations=2000, sigma_bf16=True)

# The shape of the paper's speed-up measurements (Sec. 3, "dummy datasets"):
# n = 102,400 cases, l = 1,024 features, m = 10,240, 50 generations, linear
# genomes of k in {127, 1023, 2047} genes.  The paper does not state the
# number of random trees; r = m here.  The train/test split and the target
# are this build's (the paper's dummy data is unspecified).
PAPER_K127 = Workload(
    name="paper k=127: l=1024 U[-1,1], n=81920+20480, m=10240, r=10240, linear genomes, G=50",
    n_features=1024, n_train=81920, n_test=20480, pop_size=10240, n_random_trees=10240,
    pop_min_depth=2, pop_max_depth=6, rt_min_depth=2, rt_max_depth=6, generations=50,
    target="tree5", noise=0.05, wid=5, init_mode=1, max_genes=127)
PAPER_K1023 = PAPER_K127.replace(
    name="paper k=1023: l=1024 U[-1,1], n=81920+20480, m=10240, r=10240, linear genomes, G=50",
    max_genes=1023)
PAPER_K2047 = PAPER_K127.replace(
    name="paper k=2047: l=1024 U[-1,1], n=81920+20480, m=10240, r=10240, linear genomes, G=50",
    max_genes=2047)

WORKLOADS = {"tiny": TINY, "mid": MID, "large": LARGE, "large_bf16": LARGE_BF16,
             "paper_k127": PAPER_K127, "paper_k1023": PAPER_K1023, "paper_k2047": PAPER_K2047}


def _rng(w: Workload, salt: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([w.seed, w.wid, w.run, salt]))


def _random_expression(rng: np.random.Generator, depth: int, leaves: np.ndarray,
                       cols: np.ndarray) -> np.ndarray:
    """Full binary expression of the given depth over {+, -, *}; leaves are
    columns picked from ``leaves``.  Evaluated in float64 on the fly."""
    if depth == 0:
        return cols[:, int(rng.choice(leaves))].astype(np.float64)
    a = _random_expression(rng, depth - 1, leaves, cols)
    b = _random_expression(rng, depth - 1, leaves, cols)
    op = int(rng.integers(0, 3))
    if op == 0:
        return a + b
    if op == 1:
        return a - b
    return a * b


def make_data(w: Workload):
    """Return (X_train, y_train, X_test, y_test) as float32 arrays.

    X_* are row-major (cases, features); y_* are (cases,).
    """
    rng = _rng(w, 0)
    n = w.n_cases
    if w.feature_dist == "uniform":
        X = rng.uniform(-1.0, 1.0, size=(n, w.n_features)).astype(np.float32)
    elif w.feature_dist == "normal":
        X = rng.standard_normal(size=(n, w.n_features), dtype=np.float32)
    else:
        raise ValueError(w.feature_dist)
    trng = _rng(w, 1)
    if w.target == "poly":
        Xd = X.astype(np.float64)
        y = Xd[:, 0] * Xd[:, 1] - 0.5 * Xd[:, 2] ** 2 + Xd[:, 3]
    elif w.target in ("tree5", "tree4"):
        depth = 5 if w.target == "tree5" else 4
        k = min(10, w.n_features)
        leaves = trng.choice(w.n_features, size=k, replace=False)
        y = _random_expression(trng, depth, leaves, X)
    elif w.target == "monomials":
        y = np.zeros(n, dtype=np.float64)
        for _ in range(20):
            a, b = (int(v) for v in trng.integers(0, w.n_features, size=2))
            c = float(trng.uniform(-1.0, 1.0))
            y += c * X[:, a].astype(np.float64) * X[:, b].astype(np.float64)
    else:
        raise ValueError(w.target)
    if w.noise > 0:
        y = y + trng.normal(0.0, w.noise, size=n)
    y = y.astype(np.float32)
    ntr = w.n_train
    return (np.ascontiguousarray(X[:ntr]), np.ascontiguousarray(y[:ntr]),
            np.ascontiguousarray(X[ntr:]), np.ascontiguousarray(y[ntr:]))


def make_new_cases(w: Workload, n: int, salt: int = 7) -> np.ndarray:
    """Fresh unseen cases with the workload's feature distribution (row-major)."""
    rng = _rng(w, salt)
    if w.feature_dist == "uniform":
        return rng.uniform(-1.0, 1.0, size=(n, w.n_features)).astype(np.float32)
    return rng.standard_normal(size=(n, w.n_features), dtype=np.float32)


def batched_runs(count: int = 48, seed: int = 1, generations: int = 500,
                 max_train: Optional[int] = None) -> List[Workload]:
    """Shapes of the batched workload: ``count`` independent runs with uneven
    sizes (n_train log-uniform in [1e3, 2e5], n_test = n_train // 4, features
    uniform in 5..100, m uniform in 256..2048, r uniform in 256..1024, depth
    2-6, target a random depth-4 expression + N(0, 0.05))."""
    rng = np.random.Generator(np.random.PCG64([seed, 4, 0, 0]))
    out = []
    for q in range(count):
        ntr = int(round(math.exp(rng.uniform(math.log(1e3), math.log(2e5)))))
        if max_train is not None:
            ntr = min(ntr, max_train)
        out.append(Workload(
            name=f"batched run {q}", n_features=int(rng.integers(5, 101)),
            n_train=ntr, n_test=ntr // 4, pop_size=int(rng.integers(256, 2049)),
            n_random_trees=int(rng.integers(256, 1025)), pop_min_depth=2,
            pop_max_depth=6, rt_min_depth=2, rt_max_depth=6,
            generations=generations, seed=seed, run=q, target="tree4",
            noise=0.05, wid=4))
    return out
