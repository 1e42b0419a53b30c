"""Pins of the oracle's paper-style linear genomes (Sec. 2.2,
"Initialization" and "Interpreter"): gene-class, operator, feature and
constant distributions against the printed probabilities (read as weights
0.8 : 0.14 : 0.04), independence of genes, exact length, the skip rule and
the Out register, and planted mistakes that the pins must catch."""
import math

import numpy as np
import pytest

from oracle import interp as oi
from oracle import trees as ot
from pins import pin_hand_linear_genomes

SEED, RUN = 7, 3


@pytest.fixture(scope="module")
def pool():
    return ot.linear_pool(SEED, RUN, 1, 3000, 127, 10, -1.0, 1.0)


def classes(genes):
    op = genes & 0xFF
    return np.where(genes < 4, 0, np.where(op == ot.OP_VAR, 1, 2))


def _z(count, n, p):
    return (count - n * p) / math.sqrt(n * p * (1 - p))


def test_gene_class_frequencies(pool):
    g, c, L = pool
    assert np.all(L == 127) and g.shape == (3000, 127)     # fixed length, no padding
    cl = classes(g).ravel()
    n = cl.size
    for k, p in enumerate((0.8 / 0.98, 0.14 / 0.98, 0.04 / 0.98)):
        assert abs(_z((cl == k).sum(), n, p)) < 5, k


def test_operators_features_and_constants(pool):
    g, c, _ = pool
    ops = g[g < 4]
    counts = np.bincount(ops, minlength=4)
    chi2 = ((counts - ops.size / 4) ** 2 / (ops.size / 4)).sum()
    assert chi2 < 25            # 3 degrees of freedom
    feats = g[(g & 0xFF) == ot.OP_VAR] >> 8
    fc = np.bincount(feats, minlength=10)
    assert fc.size == 10 and fc.min() > 0
    chi2 = ((fc - feats.size / 10) ** 2 / (feats.size / 10)).sum()
    assert chi2 < 40            # 9 degrees of freedom
    cv = c[g == ot.OP_CONST]
    assert cv.size > 1000 and np.all((cv >= -1.0) & (cv < 1.0))
    assert abs(cv.mean()) < 5 * math.sqrt(1 / 3 / cv.size)
    assert np.all(c[g != ot.OP_CONST] == 0)


def test_genes_are_independent(pool):
    g, _, _ = pool
    cl = classes(g)
    a, b = cl[:, :-1].ravel(), cl[:, 1:].ravel()
    table = np.zeros((3, 3))
    np.add.at(table, (a, b), 1)
    expect = np.outer(table.sum(1), table.sum(0)) / table.sum()
    chi2 = ((table - expect) ** 2 / expect).sum()
    assert chi2 < 40            # 4 degrees of freedom


def test_streams_are_per_individual_and_purpose():
    a = ot.linear_genome(SEED, RUN, 1, 5, 64, 10, -1, 1)
    b = ot.linear_genome(SEED, RUN, 1, 5, 64, 10, -1, 1)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    for other in (ot.linear_genome(SEED, RUN, 1, 6, 64, 10, -1, 1),
                  ot.linear_genome(SEED, RUN, 2, 5, 64, 10, -1, 1),
                  ot.linear_genome(SEED, RUN + 1, 1, 5, 64, 10, -1, 1)):
        assert not np.array_equal(a[0], other[0])
    # a prefix of a longer genome is the shorter genome (words 2j, 2j+1)
    longer = ot.linear_genome(SEED, RUN, 1, 5, 100, 10, -1, 1)
    assert np.array_equal(longer[0][:64], a[0]) and np.array_equal(longer[1][:64], a[1])


def test_max_stack_depth_by_hand():
    P = {"+": 0, "-": 1, "*": 2, "/": 3}
    x = lambda f: ot.OP_VAR | (f << 8)  # noqa: E731
    assert ot.genome_max_stack([P["+"], x(0), x(1), P["*"]]) == 2
    assert ot.genome_max_stack([x(0), x(1), x(2), P["+"], P["+"]]) == 3
    assert ot.genome_max_stack([P["/"], P["/"]]) == 0
    assert ot.genome_max_stack([x(0), P["-"], x(1), x(2), x(3)]) == 4


def test_linear_bound_evaluator_agrees_with_the_rule(pool):
    g, c, _ = pool
    X = np.random.default_rng(0).uniform(-1, 1, (10, 50))
    for i in range(40):
        v = oi.eval_linear_genome(g[i], c[i], X)
        w, e = oi.eval_postfix_fp32_bound(g[i], c[i], X, linear=True)
        assert np.array_equal(np.isnan(v), np.isnan(w))
        fin = np.isfinite(v)
        assert np.array_equal(v[fin], w[fin])
        assert np.all(e[fin] >= 0)


def test_interpreter_rule_mistakes_are_caught():
    def out_is_top(genes, consts, X, eps=1e-3):       # the final stack top instead of Out
        n = X.shape[1]
        st = []
        for gg, cc in zip(genes, consts):
            o = gg & 0xFF
            if o == ot.OP_VAR:
                st.append(X[gg >> 8].astype(np.float64))
            elif o == ot.OP_CONST:
                st.append(np.full(n, float(cc)))
            elif len(st) >= 2:
                b = st.pop()
                a = st.pop()
                st.append(oi._apply(o, a, b, float(np.float32(eps))))
        return st[-1] if st else np.zeros(n)

    def no_skip(genes, consts, X, eps=1e-3):          # a short function consumes what it finds
        n = X.shape[1]
        st, out = [], None
        for gg, cc in zip(genes, consts):
            o = gg & 0xFF
            if o == ot.OP_VAR:
                st.append(X[gg >> 8].astype(np.float64))
            elif o == ot.OP_CONST:
                st.append(np.full(n, float(cc)))
            else:
                b = st.pop() if st else np.zeros(n)
                a = st.pop() if st else np.zeros(n)
                out = oi._apply(o, a, b, float(np.float32(eps)))
                st.append(out)
        return out if out is not None else (st[-1] if st else np.zeros(n))

    for bad in (out_is_top, no_skip):
        with pytest.raises(AssertionError):
            pin_hand_linear_genomes(bad)


def test_class_threshold_mistake_is_caught():
    """Unnormalised thresholds (0.8 and 0.94 without dividing by 0.98) shift
    the class frequencies far beyond the pins' tolerance."""
    rng = np.random.default_rng(1)
    u = rng.random(200000)
    cl = np.where(u < 0.8, 0, np.where(u < 0.94, 1, 2))
    assert abs(_z((cl == 0).sum(), cl.size, 0.8 / 0.98)) > 5
