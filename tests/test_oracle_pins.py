"""The CPU oracle against published values, closed forms, invariants and
brute force (no GPU)."""
import itertools
import math

import numpy as np
import pytest

import workloads as W
from oracle import gsgp as og
from oracle import interp as oi
from oracle import philox as op
from oracle import trees as ot
from pins import (parse_program, pin_elitism, pin_gsm, pin_hand_linear_genomes,
                  pin_hand_programs, pin_philox_kat, pin_rmse, pin_sigma,
                  pin_tournament)


# ---------------------------------------------------------------- RNG ------
def test_philox_known_answers():
    pin_philox_kat(op.philox4x32_10)


def test_stream_layout_counter_fields():
    # word w of a stream is lane w % 4 of block w // 4, counter = (block, ind, gp, run)
    seed, run, gp, ind = 0x1234_5678_9ABC_DEF0, 7, 0x80000001, 42
    words = op.stream_words(seed, run, gp, ind, 12)
    for blk in range(3):
        out = op.philox4x32_10(np.array([blk, ind, gp, run], dtype=np.uint64),
                               np.array([0x9ABCDEF0, 0x12345678], dtype=np.uint64))
        assert list(words[4 * blk:4 * blk + 4]) == list(out)
    many = op.streams_words(seed, run, gp, 50, 9)
    assert np.array_equal(many[ind], op.stream_words(seed, run, gp, ind, 9))


def test_idx_and_u24_mappings():
    assert op.idx(0, 10) == 0
    assert op.idx(0xFFFFFFFF, 10) == 9
    assert op.idx(0x80000000, 10) == 5
    assert op.u24(0) == 0.0
    assert op.u24(0x100) == 2.0 ** -24
    assert op.u24(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    assert float(np.float32(op.u24(0xFFFFFFFF))) == op.u24(0xFFFFFFFF)   # exact in f32
    w = np.array([0, 0x100, 0xFFFFFFFF, 0x80000000], dtype=np.uint32)
    assert list(op.idx(w, 10)) == [0, 0, 9, 5]
    assert list(op.u24(w)) == [0.0, 2.0 ** -24, 1 - 2.0 ** -24, 0.5]


def test_uniformity_chi_square():
    w = op.streams_words(1, 0, 5, 64, 4096).reshape(-1)   # 262144 words
    k = 16
    counts = np.bincount(op.idx(w, k), minlength=k)
    e = len(w) / k
    chi2 = ((counts - e) ** 2 / e).sum()
    assert chi2 < 45.0          # df = 15, p ~ 1e-4
    u = op.u24(w)
    assert abs(u.mean() - 0.5) < 0.003
    assert abs(u.var() - 1.0 / 12) < 0.002
    # successive words are uncorrelated
    assert abs(np.corrcoef(u[:-1], u[1:])[0, 1]) < 0.01


def test_constants_in_range_and_rounded_once():
    w = op.streams_words(3, 1, 2, 8, 512).reshape(-1)
    c = np.array([op.erc(x, -1.0, 1.0) for x in w])
    assert c.dtype == np.float32
    assert np.all(c >= -1.0) and np.all(c < 1.0)
    c2 = np.array([op.erc(x, 1.0, 10.0) for x in w])
    assert np.all(c2 >= 1.0) and np.all(c2 <= 10.0)
    # endpoints: u24 = 0 gives lo exactly
    assert op.erc(0, -1.0, 1.0) == np.float32(-1.0)


# --------------------------------------------------------------- trees -----
def _depth_of_index(i, dmin, dmax):
    D = dmax - dmin + 1
    return dmin + i % D, (i // D) % 2 == 0


def _well_formed(genes):
    sp = 0
    for g in genes:
        if g == ot.PAD:
            break
        if (g & 0xFF) in (ot.OP_CONST, ot.OP_VAR):
            sp += 1
        else:
            assert sp >= 2
            sp -= 1
    return sp == 1


@pytest.mark.parametrize("dmin,dmax", [(2, 4), (2, 6), (1, 1), (3, 3)])
def test_rhh_structure(dmin, dmax):
    G, C, L = ot.rhh_pool(1, 0, op.PURPOSE_POP, 48, dmin, dmax, 8)
    K = ot.max_genes(dmax)
    assert G.shape == (48, K)
    for i in range(48):
        depth, full = _depth_of_index(i, dmin, dmax)
        genes = G[i, :L[i]]
        assert _well_formed(genes)
        assert np.all(G[i, L[i]:] == ot.PAD) and np.all(C[i, L[i]:] == 0)
        d = ot.postfix_depth(genes)
        if full:
            assert L[i] == 2 ** (depth + 1) - 1 and d == depth
        else:
            assert 1 <= d <= depth if depth > 0 else d == 0
        for g, c in zip(genes, C[i, :L[i]]):
            op_ = g & 0xFF
            if op_ == ot.OP_VAR:
                assert 0 <= (g >> 8) < 8 and c == 0
            elif op_ == ot.OP_CONST:
                assert -1.0 <= c < 1.0
            else:
                assert op_ in (0, 1, 2, 3) and c == 0


def test_rhh_grow_probability_extremes():
    # p_grow = 1: grow trees are full; p_grow = 0: a root function over two terminals
    G1, _, L1 = ot.rhh_pool(2, 0, 1, 20, 2, 5, 4, p_grow=1.0)
    G0, _, L0 = ot.rhh_pool(2, 0, 1, 20, 2, 5, 4, p_grow=0.0)
    for i in range(20):
        depth, full = _depth_of_index(i, 2, 5)
        assert L1[i] == 2 ** (depth + 1) - 1
        if not full:
            assert L0[i] == 3 and ot.postfix_depth(G0[i, :3]) == 1
    # p_feature = 1: no constants; p_feature = 0: no features
    Gf, _, Lf = ot.rhh_pool(2, 0, 1, 20, 2, 4, 4, p_feature=1.0)
    Gc, _, Lc = ot.rhh_pool(2, 0, 1, 20, 2, 4, 4, p_feature=0.0)
    assert not np.any((Gf & 0xFF) == ot.OP_CONST)
    assert not np.any(((Gc & 0xFF) == ot.OP_VAR) & (Gc >= 0))


def test_rhh_word_order_brute_force():
    """A depth-1 full tree consumes, in preorder: the root's operator, then
    per leaf a type word and a value word, and emits leaf, leaf, operator."""
    seed, run = 99, 3
    G, C, L = ot.rhh_pool(seed, run, op.PURPOSE_RT, 1, 1, 1, 6, const_lo=-2, const_hi=2)
    w = op.stream_words(seed, run, op.INIT_FLAG | op.PURPOSE_RT, 0, 5)
    p_feat = float(np.float32(0.14 / 0.18))

    def leaf(wt, wv):
        if op.u24(wt) < p_feat:
            return 5 | (op.idx(wv, 6) << 8), np.float32(0)
        return 4, op.erc(wv, -2.0, 2.0)

    l1, l2 = leaf(w[1], w[2]), leaf(w[3], w[4])
    assert L[0] == 3
    assert list(G[0, :3]) == [l1[0], l2[0], op.idx(w[0], 4)]
    assert list(C[0, :3]) == [l1[1], l2[1], 0]


def test_rhh_statistics():
    # under grow, an inner non-root node is a function with probability 0.5;
    # a terminal is a feature with probability 7/9; operators uniform.
    G, _, L = ot.rhh_pool(5, 0, 1, 400, 2, 6, 16)
    genes = np.concatenate([G[i, :L[i]] for i in range(400)])
    ops = genes[(genes & 0xFF) < 4]
    frac = np.bincount(ops & 0xFF, minlength=4) / len(ops)
    assert np.all(np.abs(frac - 0.25) < 0.02)
    term = genes[(genes & 0xFF) >= 4]
    feat = np.mean((term & 0xFF) == ot.OP_VAR)
    assert abs(feat - 7 / 9) < 0.02


# ----------------------------------------------------------- interpreter ---
def test_hand_programs():
    pin_hand_programs(oi.eval_postfix)


def test_hand_linear_genomes():
    pin_hand_linear_genomes(oi.eval_linear_genome)


def test_linear_genome_rule_equals_postfix_on_well_formed_programs():
    G, C, L = ot.rhh_pool(4, 0, 1, 30, 2, 5, 3)
    X = np.random.default_rng(0).uniform(-1, 1, size=(3, 50))
    for i in range(30):
        a = oi.eval_postfix(G[i, :L[i]], C[i, :L[i]], X)
        b = oi.eval_linear_genome(G[i, :L[i]], C[i, :L[i]], X)
        assert np.array_equal(a, b)


def _random_tree(rng, depth, l):
    if depth == 0 or rng.random() < 0.2:
        if rng.random() < 0.6:
            return ("var", int(rng.integers(0, l)))
        return ("const", float(np.float32(rng.uniform(-1, 1))))
    op_ = "+-*/"[int(rng.integers(0, 4))]
    return (op_, _random_tree(rng, depth - 1, l), _random_tree(rng, depth - 1, l))


def test_stack_interpreter_equals_recursive_evaluator():
    rng = np.random.default_rng(11)
    l = 5
    X = rng.uniform(-1, 1, size=(l, 64))
    X[:, 0] = 0.0                    # exercise the protected branch
    X[1, 1] = 0.0005
    for _ in range(300):
        tree = _random_tree(rng, int(rng.integers(0, 7)), l)
        genes, consts = oi.tree_to_postfix(tree)
        got = oi.eval_postfix(genes, consts, X)
        want = np.array([oi.eval_tree(tree, X[:, j]) for j in range(X.shape[1])])
        assert np.array_equal(got, want)
        assert oi.postfix_to_tree(genes, consts) == tree


def test_depth0_program_is_its_feature():
    X = np.random.default_rng(1).normal(size=(4, 33))
    for f in range(4):
        assert np.array_equal(oi.eval_postfix([5 | (f << 8)], [0], X), X[f])


def test_sigma_closed_forms():
    pin_sigma(oi.sigma)


def test_bf16_rounding():
    # bf16 keeps 8 significant bits: the spacing just above 1.0 is 2^-7
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -9, 1.0 + 3 * 2 ** -9,
                  1.0 + 2 ** -7 + 2 ** -8, 0.1, np.nan])
    r = oi.bf16_round(v)
    assert r[0] == 1.0
    assert r[1] == 1.0                           # exact tie -> even significand
    assert r[2] == 1.0                           # below half a spacing
    assert r[3] == 1.0 + 2 ** -7                 # above half a spacing
    assert r[4] == 1.0 + 2 ** -6                 # tie from an odd significand -> up
    assert abs(r[5] - 0.1) <= 0.1 * 2 ** -8
    assert np.isnan(r[6])


# -------------------------------------------------------------- fitness ----
def test_rmse_closed_forms():
    pin_rmse(og.rmse)


def test_tournament_brute_force():
    pin_tournament(og.tournament)


def test_gsm_closed_form():
    pin_gsm(og.gsm)


def test_elitism_cases():
    pin_elitism(og.elitism_decision)


def test_selection_draw_layout():
    p = og.Params(seed=9, run=2, pop_size=50, n_random_trees=30, tournament_size=4,
                  ms=0.25, ms_mode=1)
    cand, a, b, ms = og.selection_draws(p, 17)
    for i in (0, 13, 49):
        w = op.stream_words(9, 2, 17, i, 7)
        assert list(cand[i]) == [op.idx(x, 50) for x in w[:4]]
        assert a[i] == op.idx(w[4], 30) and b[i] == op.idx(w[5], 30)
        assert ms[i] == np.float32(np.float64(np.float32(0.25)) * op.u24(w[6]))
    p0 = og.Params(seed=9, run=2, pop_size=50, n_random_trees=30, tournament_size=0)
    c0, a0, b0, ms0 = og.selection_draws(p0, 17)
    assert c0.shape == (50, 0) and np.all(ms0 == np.float32(0.1))
    w = op.stream_words(9, 2, 17, 3, 3)
    assert a0[3] == op.idx(w[0], 30) and b0[3] == op.idx(w[1], 30)


# ---------------------------------------------------- whole-run invariants -
def _tiny_run(generations=12, **kw):
    w = W.TINY.replace(n_train=64, n_test=16, pop_size=32, n_random_trees=24)
    d = W.make_data(w)
    p = og.Params(seed=w.seed, run=w.run, pop_size=w.pop_size,
                  n_random_trees=w.n_random_trees, **kw)
    o = og.GSGP(p, *d)
    o.init()
    o.evolve(generations)
    return o, d


def test_best_train_rmse_is_non_increasing():
    o, _ = _tiny_run(25)
    bt = np.array(o.best_train)
    assert np.all(np.diff(bt) <= 0)
    assert bt[-1] < bt[0]


def test_offspring_equal_recorded_linear_combination():
    """Trace invariant: every slot of every generation equals its recorded
    parent plus ms (R_rt1 - R_rt2), or a copy of the parent for elites."""
    w = W.TINY.replace(n_train=64, n_test=16, pop_size=32, n_random_trees=24)
    d = W.make_data(w)
    p = og.Params(seed=1, run=0, pop_size=32, n_random_trees=24)
    o = og.GSGP(p, *d)
    o.init()
    for _ in range(8):
        prev = o.S_T.copy()
        o.generation()
        par, r1, r2, ms = (x[-1] for x in o.trace())
        for i in range(32):
            if r1[i] < 0:
                assert np.array_equal(o.S_T[i], prev[par[i]])
            else:
                want = prev[par[i]] + float(ms[i]) * (o.S_R[r1[i]] - o.S_R[r2[i]])
                assert np.allclose(o.S_T[i], want, rtol=0, atol=1e-15)


def test_predict_reproduces_best_semantics():
    o, d = _tiny_run(15)
    X_all = np.concatenate([d[0], d[2]])
    for slot in (o.best_slot(), 0, 7):
        y = o.predict(X_all, slot)
        assert np.allclose(y, o.S_T[slot], rtol=1e-12, atol=1e-12)
    tr, te = og.rmse(o.predict(X_all)[None, :], o.t, o.n_train)
    assert math.isclose(tr[0], o.best_train[-1], rel_tol=1e-12)
    assert math.isclose(te[0], o.best_test[-1], rel_tol=1e-12)


def _eval_expanded(node, x):
    kind = node[0]
    if kind == "sig":
        v = _eval_expanded(node[1], x)
        return 1.0 / (1.0 + math.exp(-v)) if v > -700 else 0.0
    if kind == "lin":            # parent + ms * (a - b), plain arithmetic
        return _eval_expanded(node[1], x) + node[2] * (
            _eval_expanded(node[3], x) - _eval_expanded(node[4], x))
    if kind == "prog":
        return oi.eval_tree(node[1], x)
    raise ValueError(kind)


def test_best_individual_brute_force_expansion():
    """Expand the best individual into one explicit expression (ancestor
    tree wrapped by one mutation node per generation of its lineage) and
    evaluate it from scratch on every case."""
    o, d = _tiny_run(5)
    par, r1, r2, ms = o.trace()
    slot = o.best_slot()
    lineage = []
    for g in range(len(par) - 1, -1, -1):
        lineage.append((int(r1[g][slot]), int(r2[g][slot]), float(ms[g][slot])))
        slot = int(par[g][slot])
    gP, cP, lP = o.P
    expr = ("prog", oi.postfix_to_tree(gP[slot, :lP[slot]], cP[slot, :lP[slot]]))
    gR, cR, lR = o.R
    for a, b, step in reversed(lineage):
        if a < 0:
            continue
        ta = ("sig", ("prog", oi.postfix_to_tree(gR[a, :lR[a]], cR[a, :lR[a]])))
        tb = ("sig", ("prog", oi.postfix_to_tree(gR[b, :lR[b]], cR[b, :lR[b]])))
        expr = ("lin", expr, step, ta, tb)
    X_all = np.concatenate([d[0], d[2]]).astype(np.float64)
    vals = np.array([_eval_expanded(expr, X_all[j]) for j in range(len(X_all))])
    assert np.allclose(vals, o.S_T[o.best_slot()], rtol=1e-12, atol=1e-12)


def test_paper_mode_mutates_every_slot():
    o, _ = _tiny_run(4, tournament_size=0, elitism=False)
    par, r1, _, _ = o.trace()
    assert np.all(par == np.arange(32)[None, :]) and np.all(r1 >= 0)


def test_replay_of_own_trace_is_consistent():
    o, d = _tiny_run(10)
    par, r1, r2, ms = o.trace()
    w = W.TINY.replace(n_train=64, n_test=16, pop_size=32, n_random_trees=24)
    p = og.Params(seed=w.seed, run=w.run, pop_size=32, n_random_trees=24)
    rp = og.GSGP(p, *d)
    rp.init()
    checks = {}
    for g in range(10):
        rp.generation({"parent": par[g], "rt1": r1[g], "rt2": r2[g], "ms": ms[g]}, checks)
    assert not checks
    assert np.array_equal(rp.S_T, o.S_T)


def test_replay_detects_a_wrong_parent():
    o, d = _tiny_run(3)
    par, r1, r2, ms = o.trace()
    bad = par[0].copy()
    i = int(np.nonzero(r1[0] >= 0)[0][0])
    bad[i] = (bad[i] + 1) % 32
    p = og.Params(pop_size=32, n_random_trees=24)
    rp = og.GSGP(p, *d)
    rp.init()
    checks = {}
    rp.generation({"parent": bad, "rt1": r1[0], "rt2": r2[0], "ms": ms[0]}, checks)
    assert checks.get("winner_not_candidate") or checks.get("winner_mismatch")
