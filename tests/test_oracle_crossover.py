"""Pins of the oracle's geometric semantic crossover (the GSGP crossover the
paper names beside mutation, Sec. 2) and of prediction by replaying the
trace: closed forms, draw frequencies, the per-offspring invariant, the
replay against a recursive evaluation of the lineage DAG and against the
ancestor-plus-coefficients model of mutation-only runs, and planted
mistakes."""
import functools
import math

import numpy as np
import pytest

import workloads as W
from oracle import gsgp as og
from oracle import interp as oi


def test_gsc_closed_forms():
    S_T = np.array([[1.0, 2.0, -3.0], [5.0, -7.0, 11.0]])
    S_R = np.array([[1.0, 0.0, 0.25]])
    got = og.gsc(S_T, S_R, np.array([0]), np.array([1]), np.array([0]))[0]
    assert got[0] == 1.0                       # R = 1: parent 1
    assert got[1] == -7.0                      # R = 0: parent 2
    assert got[2] == 0.25 * -3.0 + 0.75 * 11.0
    # planted mistake: the weights swapped
    Rm = S_R[[0]]
    swapped = (1 - Rm) * S_T[[0]] + Rm * S_T[[1]]
    assert not np.array_equal(swapped[0], got)


def test_crossover_draws_frequency_and_independence():
    p = og.Params(pop_size=512, p_crossover=0.3)
    hits = n = 0
    for g in range(40):
        cross, cand2 = og.crossover_draws(p, g)
        hits += int(cross.sum())
        n += cross.size
        assert cand2.shape == (512, 4) and cand2.min() >= 0 and cand2.max() < 512
        # the mutation words are untouched by crossover
        c0, a0, b0, m0 = og.selection_draws(og.Params(pop_size=512), g)
        c1, a1, b1, m1 = og.selection_draws(p, g)
        assert np.array_equal(a0, a1) and np.array_equal(b0, b1) and np.array_equal(c0, c1)
    z = (hits - 0.3 * n) / math.sqrt(n * 0.3 * 0.7)
    assert abs(z) < 5


@pytest.fixture(scope="module")
def crossover_run():
    w = W.TINY.replace(pop_size=64, n_random_trees=40)
    data = W.make_data(w)
    p = og.Params(pop_size=64, n_random_trees=40, p_crossover=0.4)
    o = og.GSGP(p, *data)
    o.init()
    snaps = [o.S_T.copy()]
    for _ in range(12):
        o.generation()
        snaps.append(o.S_T.copy())
    return o, data, snaps


def test_offspring_equal_the_recorded_combination(crossover_run):
    o, _, snaps = crossover_run
    par, r1, r2, ms = o.trace()
    assert (r2 <= -2).any() and (r1 >= 0).any()
    for g in range(len(par)):
        prev, cur = snaps[g], snaps[g + 1]
        for i in range(o.p.pop_size):
            a, b = int(r1[g][i]), int(r2[g][i])
            if a < 0:
                want = prev[par[g][i]]
            elif b <= -2:
                Rm = o.S_R[a]
                want = Rm * prev[par[g][i]] + (1 - Rm) * prev[-2 - b]
            else:
                want = prev[par[g][i]] + float(ms[g][i]) * (o.S_R[a] - o.S_R[b])
            assert np.allclose(cur[i], want, rtol=1e-12, atol=1e-12)
    assert np.all(np.diff(o.best_train) <= 0)


def test_replay_prediction(crossover_run):
    o, data, _ = crossover_run
    X_all = np.concatenate([data[0], data[2]])
    best = o.best_slot()
    # on the training and test cases the replay reproduces the semantics
    assert np.array_equal(o.predict(X_all), o.S_T[best])
    # a recursive evaluation of the lineage DAG on single new cases
    Xn = W.make_new_cases(W.TINY, 5)
    y = o.predict(Xn)
    par, r1, r2, ms = o.trace()
    P, R = o.P, o.R
    for j in range(5):
        x = og.feature_major(Xn[j:j + 1])

        @functools.lru_cache(maxsize=None)
        def val(g, slot):
            if g < 0:
                L = int(P[2][slot])
                return float(oi.eval_postfix(P[0][slot, :L], P[1][slot, :L], x)[0])
            a, b, pa = int(r1[g][slot]), int(r2[g][slot]), int(par[g][slot])
            if a < 0:
                return val(g - 1, pa)
            La = int(R[2][a])
            sa = float(oi.sigma(oi.eval_postfix(R[0][a, :La], R[1][a, :La], x))[0])
            if b <= -2:
                return sa * val(g - 1, pa) + (1 - sa) * val(g - 1, -2 - b)
            Lb = int(R[2][b])
            sb = float(oi.sigma(oi.eval_postfix(R[0][b, :Lb], R[1][b, :Lb], x))[0])
            return val(g - 1, pa) + float(ms[g][slot]) * (sa - sb)

        assert math.isclose(val(len(par) - 1, o.best_slot()), y[j], rel_tol=1e-12, abs_tol=1e-12)


def test_replay_equals_the_model_without_crossover():
    w = W.TINY
    data = W.make_data(w)
    o = og.GSGP(og.Params(), *data)
    o.init()
    o.evolve(15)
    X = W.make_new_cases(w, 50)
    anc, coef = o.reconstruct()
    model = og.predict(o.P, o.R, anc, coef, og.feature_major(X), o.p.protect_eps)
    replay = og.predict_replay(o.trace(), o.best_slot(), o.P, o.R, og.feature_major(X),
                               o.p.protect_eps)
    assert np.allclose(model, replay, rtol=1e-12, atol=1e-12)
    # planted mistake: a replay that drops the mutation step
    par, r1, r2, ms = o.trace()
    bad = og.predict_replay((par, r1, r2, np.zeros_like(ms)), o.best_slot(), o.P, o.R,
                            og.feature_major(X), o.p.protect_eps)
    assert not np.allclose(model, bad, rtol=1e-6)
