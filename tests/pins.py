"""Checks that pin the oracle to facts outside itself.

Each function raises AssertionError when the implementation it is given
violates a published value, a closed form, an invariant or a brute-force
result.  They take the functions under test as arguments so that
tests/test_oracle_mistakes.py can hand them a copy of the oracle with a
planted mistake and see them fail.
"""
from __future__ import annotations

import math

import numpy as np

from conftest import read_golden

TOK_OPS = {"+": 0, "-": 1, "*": 2, "/": 3}


def parse_program(text: str):
    genes, consts = [], []
    for tok in text.split():
        if tok in TOK_OPS:
            genes.append(TOK_OPS[tok])
            consts.append(np.float32(0))
        elif tok.startswith("x"):
            genes.append(5 | (int(tok[1:]) << 8))
            consts.append(np.float32(0))
        elif tok.startswith("c:"):
            genes.append(4)
            consts.append(np.float32(float(tok[2:])))
        else:
            raise ValueError(tok)
    return genes, consts


def pin_philox_kat(philox):
    """Published known-answer vectors of Philox4x32-10."""
    for row in read_golden("philox4x32_10_kat.txt"):
        w = [int(v, 16) for v in row[0].split()]
        ctr, key, want = w[0:4], w[4:6], w[6:10]
        got = [int(v) for v in philox(np.array(ctr, dtype=np.uint64),
                                      np.array(key, dtype=np.uint64))]
        assert got == want, (ctr, key, [hex(v) for v in got])


def pin_hand_programs(eval_postfix):
    """Hand-evaluated postfix programs (tests/golden/hand_programs.txt)."""
    for prog, xs, want in read_golden("hand_programs.txt"):
        x = [float(v) for v in xs.split()]
        genes, consts = parse_program(prog)
        X = np.array(x, dtype=np.float64)[:, None]
        got = eval_postfix(genes, consts, X, 1e-3)
        assert got.shape == (1,)
        assert math.isclose(float(got[0]), float(want), rel_tol=1e-12, abs_tol=1e-12), \
            (prog, x, float(got[0]), want)


def pin_hand_linear_genomes(eval_linear):
    for prog, xs, want in read_golden("hand_linear_genomes.txt"):
        x = [float(v) for v in xs.split()]
        genes, consts = parse_program(prog)
        X = np.array(x, dtype=np.float64)[:, None]
        got = eval_linear(genes, consts, X, 1e-3)
        assert math.isclose(float(got[0]), float(want), rel_tol=1e-12, abs_tol=1e-12), \
            (prog, x, float(got[0]), want)


def pin_sigma(sigma):
    """Closed forms of the logistic function 1/(1+exp(-v))."""
    assert sigma(np.array([0.0]))[0] == 0.5
    assert math.isclose(sigma(np.array([math.log(3.0)]))[0], 0.75, rel_tol=1e-15)
    v = np.linspace(-30, 30, 601)
    s = sigma(v)
    assert np.all((s >= 0) & (s <= 1))
    assert np.allclose(s + sigma(-v), 1.0, atol=1e-15)
    assert np.all(np.diff(s) >= 0)
    assert sigma(np.array([-1e6]))[0] == 0.0 and sigma(np.array([1e6]))[0] == 1.0


def pin_rmse(rmse):
    """Closed forms of the training/test RMSE split."""
    rng = np.random.default_rng(5)
    t = rng.normal(size=40)
    S = np.stack([t, t + 0.25, t - 3.0, t + np.where(np.arange(40) < 30, 1.0, 2.0)])
    tr, te = rmse(S, t, 30)
    assert tr[0] == 0.0 and te[0] == 0.0
    assert math.isclose(tr[1], 0.25, rel_tol=1e-12) and math.isclose(te[1], 0.25, rel_tol=1e-12)
    assert math.isclose(tr[2], 3.0, rel_tol=1e-12) and math.isclose(te[2], 3.0, rel_tol=1e-12)
    assert math.isclose(tr[3], 1.0, rel_tol=1e-12) and math.isclose(te[3], 2.0, rel_tol=1e-12)
    # RMSE of alternating +-d residuals is d; of residuals (1, 2, 3, 4)^T is sqrt(7.5)
    S2 = np.array([[1.0, -1.0, 1.0, -1.0], [1.0, 2.0, 3.0, 4.0]])
    tr2, _ = rmse(S2, np.zeros(4), 4)
    assert math.isclose(tr2[0], 1.0, rel_tol=1e-15)
    assert math.isclose(tr2[1], math.sqrt(7.5), rel_tol=1e-15)
    # a non-finite training value makes the fitness +inf; test cases do not
    S3 = np.array([[np.nan, 0, 0, 0], [0, 0, 0, np.inf]])
    tr3, te3 = rmse(S3, np.zeros(4), 3)
    assert tr3[0] == np.inf and tr3[1] == 0.0 and te3[1] == np.inf


def pin_tournament(tournament):
    """Tournament winner: smallest fitness, earliest drawn candidate on ties."""
    F = np.array([3.0, 1.0, 2.0, 1.0, np.inf, 0.5])
    cand = np.array([[0, 1, 2, 3], [3, 1, 0, 2], [4, 4, 4, 4], [2, 0, 4, 5],
                     [5, 5, 1, 1], [4, 0, 4, 2]])
    want = [1, 3, 4, 5, 5, 2]
    assert list(tournament(F, cand)) == want
    # t = 1: the only candidate wins; t = 0: every slot keeps itself
    assert list(tournament(F, cand[:, :1])) == [0, 3, 4, 2, 5, 4]
    assert list(tournament(F, np.zeros((6, 0), dtype=np.int64))) == list(range(6))
    # brute force over every 3-candidate tuple of 4 individuals with ties
    F4 = np.array([2.0, 1.0, 1.0, 0.0])
    import itertools
    tuples = np.array(list(itertools.product(range(4), repeat=3)))
    got = tournament(F4, tuples)
    for tup, g in zip(tuples, got):
        best = min(F4[k] for k in tup)
        first = next(k for k in tup if F4[k] == best)
        assert g == first


def pin_gsm(gsm):
    """Geometric semantic mutation: offspring = parent + ms (R_a - R_b)."""
    S_T = np.array([[1.0, 2.0, 3.0], [-1.0, 0.0, 5.0]])
    S_R = np.array([[1.0, 1.0, 1.0], [0.0, 0.0, 0.0], [0.25, 0.5, 0.75]])
    ms = np.array([0.5, 0.5, 0.25, 0.1], dtype=np.float32)
    par = np.array([0, 0, 1, 1])
    a = np.array([0, 1, 2, 2])
    b = np.array([1, 0, 1, 2])
    out = gsm(S_T, S_R, par, a, b, ms)
    assert np.allclose(out[0], [1.5, 2.5, 3.5])       # + ms when R_a = 1, R_b = 0
    assert np.allclose(out[1], [0.5, 1.5, 2.5])       # - ms when swapped
    assert np.allclose(out[2], [-1 + 0.0625, 0.125, 5 + 0.1875])
    assert np.array_equal(out[3], S_T[1])             # a == b gives the parent


def pin_elitism(elitism_decision):
    F_T = np.array([0.5, 0.2, 0.9])
    assert elitism_decision(F_T, np.array([0.3, 0.4, 0.6])) == (1, 2)
    assert elitism_decision(F_T, np.array([0.3, 0.1, 0.6])) is None
    assert elitism_decision(F_T, np.array([0.3, 0.2, 0.6])) is None     # tie: offspring win
    assert elitism_decision(F_T, np.array([np.inf, 0.4, np.inf])) == (1, 0)
    assert elitism_decision(np.array([0.2, 0.2]), np.array([0.7, 0.7])) == (0, 0)
