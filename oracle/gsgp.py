"""The GSGP evolutionary loop in float64 (Algorithm 1 and Sec. 2).

Steps, in the order of Algorithm 1:
  1. CreatePopulation(m, k) -> P, CreatePopulation(r, k) -> R      (trees.py)
  2. ComputeSemantics(P) -> S_T (m x n), ComputeSemantics(R) -> S_R (r x n),
     the random trees wrapped by the logistic function                (interp.py)
  3. ComputeFitness(S_T, t) -> F_T: RMSE of each row against the target
     (Sec. 2.2, "Fitness computation")
  4. for each generation:
       GSM(S_T, S_R) -> S_O: offspring = parent + ms * (R_u - R_v)   (Sec. 2)
       ComputeFitness(S_O, t) -> F_O
       survival: generational replacement with elitism of the best of parents
       and offspring (Sec. 2.2, "Survival")
  5. return the best individual.

Readings of points the paper leaves open or prints inconsistently:
  * GSM sign: the paper prints T + ms (R1 + R2); the standard operator (and
    the one implemented) is T + ms (R1 - R2).  ``gsm_sign_plus`` keeps the
    printed form for experiments only.
  * Selection: the paper mutates every individual (parent of slot i is i,
    tournament_size = 0 here); the default is a size-4 tournament on training
    RMSE, ties to the earliest drawn candidate.
  * Draws per offspring slot i at generation g come from the Philox stream
    (i, g): words 0..t-1 are the tournament candidates idx(w, m), word t the
    first random tree idx(w, r), word t+1 the second, word t+2 the mutation
    step (ms * u24(w) in uniform mode; reserved when ms is fixed).
  * Fitness: train RMSE over the first n_train cases, test RMSE over the rest;
    a non-finite value becomes +inf.  Selection uses training RMSE only.
  * Elitism: b_P = argmin F_T, b_O = argmin F_O (first index on ties); if
    F_T[b_P] < F_O[b_O] strictly, the first worst offspring argmax F_O is
    replaced by parent b_P, recorded in the trace as (b_P, -1, -1, 0).
  * Trace: per generation and slot (parent, rt1, rt2, ms); walking it back
    from the best slot gives the generation-0 ancestor and one coefficient per
    random tree, so the best model is ancestor + sum_k c_k R_k.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

from .interp import bf16_round, eval_linear_genome, eval_postfix, pool_semantics, sigma
from .philox import PURPOSE_POP, PURPOSE_RT, idx, streams_words, u24
from .trees import linear_pool, rhh_pool


@dataclasses.dataclass
class Params:
    seed: int = 1
    run: int = 0
    pop_size: int = 128
    n_random_trees: int = 256
    pop_min_depth: int = 2
    pop_max_depth: int = 4
    rt_min_depth: int = 2
    rt_max_depth: int = 4
    p_grow: float = 0.5
    p_feature: float = 0.14 / 0.18
    const_lo: float = -1.0
    const_hi: float = 1.0
    protect_eps: float = 1e-3
    ms: float = 0.1
    ms_mode: int = 0            # 0 fixed, 1 uniform [0, ms)
    tournament_size: int = 4    # 0 = every slot mutates its own parent
    elitism: bool = True
    sigma_bf16: bool = False
    gsm_sign_plus: bool = False  # the printed "+" form; experiments only
    init_mode: int = 0           # 0 ramped half-and-half trees, 1 the paper's linear genomes
    max_genes: int = 127         # genome length k (init_mode 1)
    p_crossover: float = 0.0     # probability an offspring comes from crossover (paper: 0)


def feature_major(X_rows: np.ndarray) -> np.ndarray:
    """(n, l) row-major cases -> (l, n) float64 feature-major."""
    return np.ascontiguousarray(np.asarray(X_rows, dtype=np.float64).T)


def rmse(S: np.ndarray, t: np.ndarray, n_train: int):
    """Training and test RMSE of every row of S against target t.

    RMSE = sqrt(mean_j (s_j - t_j)^2) (Sec. 2.2, "Fitness computation"),
    over cases [0, n_train) and [n_train, n) respectively; non-finite -> +inf.
    """
    S = np.atleast_2d(S)
    with np.errstate(all="ignore"):
        d = S - t[None, :]
        sq = d * d
        tr = np.sqrt(sq[:, :n_train].mean(axis=1)) if n_train > 0 else np.zeros(len(S))
        n_te = S.shape[1] - n_train
        te = np.sqrt(sq[:, n_train:].mean(axis=1)) if n_te > 0 else np.zeros(len(S))
    tr = np.where(np.isfinite(tr), tr, np.inf)
    te = np.where(np.isfinite(te), te, np.inf)
    return tr, te


def selection_draws(p: Params, g: int):
    """Philox draws of generation g for every offspring slot.

    Returns candidates (m, t) int64, rt1 (m,), rt2 (m,), ms (m,) float32.
    """
    m, r, t = p.pop_size, p.n_random_trees, p.tournament_size
    W = streams_words(p.seed, p.run, g, m, t + 3)
    cand = idx(W[:, :t], m) if t > 0 else np.zeros((m, 0), dtype=np.int64)
    a = idx(W[:, t], r)
    b = idx(W[:, t + 1], r)
    ms32 = np.float32(p.ms)
    if p.ms_mode == 1:
        ms = (np.float64(ms32) * u24(W[:, t + 2])).astype(np.float32)
    else:
        ms = np.full(m, ms32, dtype=np.float32)
    return cand, a, b, ms


def crossover_draws(p: Params, g: int):
    """Crossover draws of generation g (only when p_crossover > 0): words
    t+3 (crossover iff u24 < p_crossover) and t+4 .. 2t+3 (the second
    parent's tournament candidates) of each slot's stream.  The mask tree is
    rt1 (word t).  Returns is_crossover (m,) bool, candidates (m, t)."""
    m, t = p.pop_size, p.tournament_size
    W = streams_words(p.seed, p.run, g, m, 2 * t + 4)
    is_cross = u24(W[:, t + 3]) < float(np.float32(p.p_crossover))
    cand2 = idx(W[:, t + 4:2 * t + 4], m) if t > 0 else np.zeros((m, 0), dtype=np.int64)
    return is_cross, cand2


def gsc(S_T: np.ndarray, S_R: np.ndarray, p1, p2, c) -> np.ndarray:
    """Geometric semantic crossover on semantic vectors: with the random
    function R = sigma(random tree c) in [0, 1], the offspring is
    R * T1 + (1 - R) * T2 case by case (the original GSGP crossover the
    paper names beside mutation, Sec. 2)."""
    Rm = S_R[c]
    return Rm * S_T[p1] + (1.0 - Rm) * S_T[p2]


def tournament(F: np.ndarray, cand: np.ndarray) -> np.ndarray:
    """Winner of each tournament: the candidate with the smallest fitness,
    the earliest drawn one on ties.  With no candidates slot i keeps i."""
    m = cand.shape[0]
    if cand.shape[1] == 0:
        return np.arange(m, dtype=np.int64)
    win = np.empty(m, dtype=np.int64)
    for i in range(m):
        best = int(cand[i, 0])
        for k in cand[i, 1:]:
            k = int(k)
            if F[k] < F[best]:
                best = k
        win[i] = best
    return win


def gsm(S_T: np.ndarray, S_R: np.ndarray, parent, a, b, ms, sign_plus=False):
    """Geometric semantic mutation on semantic vectors (Sec. 2):
    s_O[i] = s_T[parent_i] + ms_i * (s_R[a_i] - s_R[b_i])."""
    ms64 = np.asarray(ms, dtype=np.float64)[:, None]
    if sign_plus:
        return S_T[parent] + ms64 * (S_R[a] + S_R[b])
    return S_T[parent] + ms64 * (S_R[a] - S_R[b])


def elitism_decision(F_T: np.ndarray, F_O: np.ndarray):
    """Survival with elitism (Sec. 2.2): returns (b_P, w) when the best parent
    must replace the worst offspring w, else None."""
    b_P = int(np.argmin(F_T))
    b_O = int(np.argmin(F_O))
    if F_T[b_P] < F_O[b_O]:
        return b_P, int(np.argmax(F_O))
    return None


class GSGP:
    """One GSGP run held entirely in float64 host memory."""

    def __init__(self, p: Params, X_train, y_train, X_test, y_test):
        self.p = p
        self.n_train = int(np.asarray(y_train).shape[0])
        Xr = np.concatenate([np.asarray(X_train, np.float32),
                             np.asarray(X_test, np.float32)], axis=0)
        self.X = feature_major(Xr)
        self.t = np.concatenate([np.asarray(y_train, np.float32),
                                 np.asarray(y_test, np.float32)]).astype(np.float64)
        self.n_features = self.X.shape[0]
        self.gen = 0
        self.trace_parent = []
        self.trace_rt1 = []
        self.trace_rt2 = []
        self.trace_ms = []
        self.best_train = []
        self.best_test = []

    # ---- Algorithm 1, initialisation -------------------------------------
    def create_programs(self):
        p = self.p
        if p.init_mode == 1:
            self.P = linear_pool(p.seed, p.run, PURPOSE_POP, p.pop_size, p.max_genes,
                                 self.n_features, p.const_lo, p.const_hi)
            self.R = linear_pool(p.seed, p.run, PURPOSE_RT, p.n_random_trees, p.max_genes,
                                 self.n_features, p.const_lo, p.const_hi)
            return
        self.P = rhh_pool(p.seed, p.run, PURPOSE_POP, p.pop_size, p.pop_min_depth,
                          p.pop_max_depth, self.n_features, p.p_grow, p.p_feature,
                          p.const_lo, p.const_hi)
        self.R = rhh_pool(p.seed, p.run, PURPOSE_RT, p.n_random_trees, p.rt_min_depth,
                          p.rt_max_depth, self.n_features, p.p_grow, p.p_feature,
                          p.const_lo, p.const_hi)

    def compute_semantics(self):
        p = self.p
        lin = p.init_mode == 1
        self.S_T = pool_semantics(*self.P, self.X, p.protect_eps, linear=lin)
        self.S_R = pool_semantics(*self.R, self.X, p.protect_eps, logistic=True,
                                  bf16=p.sigma_bf16, linear=lin)

    def compute_fitness(self):
        self.F_T, self.F_T_te = rmse(self.S_T, self.t, self.n_train)

    def init(self):
        self.create_programs()
        self.compute_semantics()
        self.compute_fitness()

    def set_state(self, S_T, S_R):
        """Start from given semantic matrices (e.g. another implementation's
        float32 initial semantics promoted to float64) to isolate later steps."""
        self.S_T = np.asarray(S_T, dtype=np.float64).copy()
        self.S_R = np.asarray(S_R, dtype=np.float64).copy()
        self.compute_fitness()

    # ---- Algorithm 1, one generation ---------------------------------------
    def generation(self, replay: Optional[dict] = None, checks: Optional[dict] = None):
        """Run one generation.  With ``replay`` = {'parent','rt1','rt2','ms'}
        (arrays of length m from another implementation's trace) the recorded
        parents and survival decision are followed after checking them."""
        p = self.p
        g = self.gen
        cand, a, b, ms = selection_draws(p, g)
        parent = tournament(self.F_T, cand)
        cross = np.zeros(p.pop_size, dtype=bool)
        parent2 = np.arange(p.pop_size, dtype=np.int64)
        if p.p_crossover > 0:
            cross, cand2 = crossover_draws(p, g)
            parent2 = tournament(self.F_T, cand2)
        elite_slot = None
        if replay is not None:
            rp = np.asarray(replay["parent"], dtype=np.int64)
            r1 = np.asarray(replay["rt1"], dtype=np.int64)
            elite_rows = np.nonzero(r1 < 0)[0]
            if len(elite_rows) > 1:
                raise AssertionError(f"gen {g}: more than one elite entry")
            if len(elite_rows) == 1:
                elite_slot = int(elite_rows[0])
            r2 = np.asarray(replay["rt2"], dtype=np.int64)
            for i in range(p.pop_size):
                if i == elite_slot:
                    continue
                if cross[i]:
                    # crossover entry: (parent 1, mask tree, -2 - parent 2, 0)
                    if int(r1[i]) != int(a[i]) or int(r2[i]) > -2:
                        _note(checks, "draw_mismatch", (g, i))
                    gp2 = -2 - int(r2[i])
                    _check_winner(g, i, gp2, cand2[i], self.F_T, checks)
                    parent2[i] = gp2
                else:
                    _check_draws(g, i, replay, a, b, ms, checks)
                _check_winner(g, i, int(rp[i]), cand[i], self.F_T, checks)
                parent[i] = rp[i]
        S_O = gsm(self.S_T, self.S_R, parent, a, b, ms, p.gsm_sign_plus)
        if cross.any():
            S_O[cross] = gsc(self.S_T, self.S_R, parent[cross], parent2[cross], a[cross])
        F_O, F_O_te = rmse(S_O, self.t, self.n_train)
        t_parent = parent.astype(np.int32).copy()
        t_rt1 = a.astype(np.int32).copy()
        t_rt2 = b.astype(np.int32).copy()
        t_ms = ms.copy()
        t_rt2[cross] = (-2 - parent2[cross]).astype(np.int32)
        t_ms[cross] = np.float32(0)
        dec = elitism_decision(self.F_T, F_O) if p.elitism else None
        if replay is not None:
            gpu_dec = None
            if elite_slot is not None:
                gpu_dec = (int(replay["parent"][elite_slot]), elite_slot)
            _check_elitism(g, dec, gpu_dec, self.F_T, F_O, checks)
            dec = gpu_dec
        if dec is not None:
            b_P, w = dec
            S_O[w] = self.S_T[b_P]
            F_O[w] = self.F_T[b_P]
            F_O_te[w] = self.F_T_te[b_P]
            t_parent[w], t_rt1[w], t_rt2[w], t_ms[w] = b_P, -1, -1, np.float32(0)
        self.S_T, self.F_T, self.F_T_te = S_O, F_O, F_O_te
        self.trace_parent.append(t_parent)
        self.trace_rt1.append(t_rt1)
        self.trace_rt2.append(t_rt2)
        self.trace_ms.append(t_ms)
        best = int(np.argmin(self.F_T))
        self.best_train.append(float(self.F_T[best]))
        self.best_test.append(float(self.F_T_te[best]))
        self.gen += 1

    def evolve(self, generations: int):
        for _ in range(generations):
            self.generation()

    # ---- returning the best individual ---------------------------------
    def best_slot(self) -> int:
        return int(np.argmin(self.F_T))

    def trace(self):
        return (np.array(self.trace_parent), np.array(self.trace_rt1),
                np.array(self.trace_rt2), np.array(self.trace_ms))

    def reconstruct(self, slot: Optional[int] = None):
        """Walk the trace back from ``slot`` (default: the best) and return
        (ancestor index in P, coefficient per random tree)."""
        if slot is None:
            slot = self.best_slot()
        return reconstruct(self.trace(), slot, self.p.n_random_trees)

    def predict(self, X_rows, slot: Optional[int] = None) -> np.ndarray:
        if slot is None:
            slot = self.best_slot()
        if self.p.p_crossover > 0:
            return predict_replay(self.trace(), slot, self.P, self.R, feature_major(X_rows),
                                  self.p.protect_eps, self.p.sigma_bf16, self.p.init_mode == 1)
        anc, c = self.reconstruct(slot)
        return predict(self.P, self.R, anc, c, feature_major(X_rows),
                       self.p.protect_eps, self.p.sigma_bf16, self.p.init_mode == 1)


def reconstruct(trace, slot: int, n_random_trees: int):
    """Ancestry walk over the trace (parent, rt1, rt2, ms per generation and
    slot) from generation G-1 down to 0: each mutation adds +ms to the
    coefficient of rt1 and -ms to that of rt2; elite copies carry none."""
    parent, rt1, rt2, ms = trace
    c = np.zeros(n_random_trees, dtype=np.float64)
    for g in range(len(parent) - 1, -1, -1):
        a = int(rt1[g][slot])
        if a >= 0:
            b = int(rt2[g][slot])
            step = float(ms[g][slot])
            c[a] += step
            c[b] -= step
        slot = int(parent[g][slot])
    return slot, c


def predict(P, R, ancestor: int, coef, X_fm, protect_eps=1e-3, sigma_bf16=False,
            linear=False):
    """Value of the rebuilt model on feature-major cases X_fm (l, n):
    ancestor(x) + sum_k coef_k * sigma(R_k(x)); linear: the programs are
    linear genomes (skip rule, Out register)."""
    evaluate = eval_linear_genome if linear else eval_postfix
    gP, cP, lP = P
    L = int(lP[ancestor])
    y = evaluate(gP[ancestor, :L], cP[ancestor, :L], X_fm, protect_eps)
    gR, cR, lR = R
    for k in np.nonzero(coef)[0]:
        L = int(lR[k])
        s = sigma(evaluate(gR[k, :L], cR[k, :L], X_fm, protect_eps))
        if sigma_bf16:
            s = bf16_round(s)
        y = y + coef[k] * s
    return y


def predict_replay(trace, slot: int, P, R, X_fm, protect_eps=1e-3, sigma_bf16=False,
                   linear=False):
    """Value of individual `slot` after the traced generations on new cases
    X_fm (l, n), by replaying the trace on them: the initial population and
    the random trees are evaluated on the new cases, then every generation
    applies its recorded mutation (parent + ms (sigma_a - sigma_b)),
    crossover (rt2 = -2 - parent 2: R parent1 + (1 - R) parent2, R =
    sigma(rt1)) or elite copy (rt1 = -1).  Holds for any run, with or
    without crossover."""
    S = pool_semantics(*P, X_fm, protect_eps, linear=linear)
    Sr = pool_semantics(*R, X_fm, protect_eps, logistic=True, bf16=sigma_bf16, linear=linear)
    parent, rt1, rt2, ms = trace
    for g in range(len(parent)):
        pa = np.asarray(parent[g], dtype=np.int64)
        a = np.asarray(rt1[g], dtype=np.int64)
        b = np.asarray(rt2[g], dtype=np.int64)
        step = np.asarray(ms[g], dtype=np.float64)[:, None]
        new = np.empty_like(S)
        copy = a < 0
        cross = ~copy & (b <= -2)
        mut = ~copy & ~cross
        new[copy] = S[pa[copy]]
        new[mut] = S[pa[mut]] + step[mut] * (Sr[a[mut]] - Sr[b[mut]])
        if cross.any():
            new[cross] = gsc(S, Sr, pa[cross], -2 - b[cross], a[cross])
        S = new
    return S[slot]


# ---- replay checks (a second implementation's trace against this one) ----

def _note(checks, key, item):
    if checks is None:
        raise AssertionError(f"{key}: {item}")
    checks.setdefault(key, []).append(item)


def _check_draws(g, i, replay, a, b, ms, checks):
    if (int(replay["rt1"][i]) != int(a[i]) or int(replay["rt2"][i]) != int(b[i])
            or np.float32(replay["ms"][i]) != ms[i]):
        _note(checks, "draw_mismatch", (g, i))


def _check_winner(g, i, gp, cand, F, checks, rel=1e-5):
    if len(cand) == 0:
        if gp != i:
            _note(checks, "winner_mismatch", (g, i, gp))
        return
    if gp not in [int(k) for k in cand]:
        _note(checks, "winner_not_candidate", (g, i, gp))
        return
    fmin = min(F[int(k)] for k in cand)
    if not (F[gp] <= fmin or F[gp] <= fmin * (1 + rel)):
        _note(checks, "winner_mismatch", (g, i, gp))
    elif F[gp] != fmin:
        _note(checks, "winner_near_tie", (g, i, gp))


def _check_elitism(g, mine, theirs, F_T, F_O, checks, rel=1e-5):
    if mine == theirs:
        return
    # Accept a different decision only when it hinges on a near tie.
    b_P = int(np.argmin(F_T))
    b_O = int(np.argmin(F_O))
    near = abs(F_T[b_P] - F_O[b_O]) <= rel * max(abs(F_T[b_P]), 1e-300)
    if theirs is not None and mine is not None:
        tp, tw = theirs
        near = near or (abs(F_T[tp] - F_T[b_P]) <= rel * F_T[b_P]
                         and (F_O[tw] == np.inf and F_O[mine[1]] == np.inf
                              or abs(F_O[tw] - F_O[mine[1]]) <= rel * F_O[mine[1]]))
    if near:
        _note(checks, "elitism_near_tie", (g, mine, theirs))
    else:
        _note(checks, "elitism_mismatch", (g, mine, theirs))
