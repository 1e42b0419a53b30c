"""Plant plausible mistakes in copies of oracle functions (on the CPU) and
check that the pins catch each of them."""
import numpy as np
import pytest

from oracle import gsgp as og
from oracle import interp as oi
from oracle import philox as op
from pins import (pin_elitism, pin_gsm, pin_hand_programs, pin_philox_kat,
                  pin_rmse, pin_sigma, pin_tournament)


def _fails(pin, fn):
    with pytest.raises((AssertionError, IndexError, ValueError)):
        pin(fn)


def test_philox_mistakes_are_caught():
    def swapped_multipliers(ctr, key):
        saved = op.M0, op.M1
        try:
            op.M0, op.M1 = saved[1], saved[0]
            return op.philox4x32_10(ctr, key)
        finally:
            op.M0, op.M1 = saved

    def nine_rounds(ctr, key):
        c = np.asarray(ctr, dtype=np.uint64)
        k = np.asarray(key, dtype=np.uint64)
        out = c.copy()
        k0, k1 = int(k[0]), int(k[1])
        for rnd in range(9):
            if rnd:
                k0 = (k0 + op.W0) & 0xFFFFFFFF
                k1 = (k1 + op.W1) & 0xFFFFFFFF
            p0 = int(out[0]) * op.M0
            p1 = int(out[2]) * op.M1
            out = np.array([(p1 >> 32) ^ int(out[1]) ^ k0, p1 & 0xFFFFFFFF,
                            (p0 >> 32) ^ int(out[3]) ^ k1, p0 & 0xFFFFFFFF], dtype=np.uint64)
        return out

    _fails(pin_philox_kat, swapped_multipliers)
    _fails(pin_philox_kat, nine_rounds)


def _patched_eval(mistake):
    def ev(genes, consts, X, eps=1e-3):
        n = X.shape[1]
        st = []
        for g, c in zip(genes, consts):
            o = g & 0xFF
            if o == 5:
                st.append(X[g >> 8].astype(np.float64))
            elif o == 4:
                st.append(np.full(n, float(c)))
            else:
                b = st.pop()
                a = st.pop()
                if mistake == "operands_transposed":
                    a, b = b, a
                if o == 0:
                    v = a + b
                elif o == 1:
                    v = a - b
                elif o == 2:
                    v = a * b
                else:
                    if mistake == "protect_returns_zero":
                        v = np.where(np.abs(b) < eps, 0.0, a / np.where(np.abs(b) < eps, 1, b))
                    elif mistake == "protect_non_strict_1e-2":
                        v = np.where(np.abs(b) < 1e-2, 1.0, a / np.where(np.abs(b) < 1e-2, 1, b))
                    else:
                        v = np.where(np.abs(b) < eps, 1.0, a / np.where(np.abs(b) < eps, 1, b))
                st.append(v)
        return st[-1]
    return ev


@pytest.mark.parametrize("mistake", ["operands_transposed", "protect_returns_zero",
                                     "protect_non_strict_1e-2"])
def test_interpreter_mistakes_are_caught(mistake):
    pin_hand_programs(_patched_eval(None))      # the unpatched copy passes
    _fails(pin_hand_programs, _patched_eval(mistake))


def test_sigma_mistakes_are_caught():
    _fails(pin_sigma, lambda v: 1.0 / (1.0 + np.exp(np.asarray(v, float))))   # sign
    _fails(pin_sigma, lambda v: np.tanh(np.asarray(v, float)))


def test_rmse_mistakes_are_caught():
    def mse_not_rmse(S, t, ntr):
        tr, te = og.rmse(S, t, ntr)
        return tr ** 2, te ** 2

    def split_off_by_one(S, t, ntr):
        return og.rmse(S, t, ntr + 1)

    def mean_abs(S, t, ntr):
        d = np.abs(np.atleast_2d(S) - t[None, :])
        return d[:, :ntr].mean(1), d[:, ntr:].mean(1)

    for bad in (mse_not_rmse, split_off_by_one, mean_abs):
        _fails(pin_rmse, bad)


def test_tournament_mistakes_are_caught():
    _fails(pin_tournament, lambda F, c: og.tournament(-np.nan_to_num(F, posinf=1e9), c))

    def last_on_ties(F, cand):
        if cand.shape[1] == 0:
            return np.arange(cand.shape[0])
        out = []
        for row in cand:
            best = row[0]
            for k in row[1:]:
                if F[k] <= F[best]:
                    best = k
            out.append(best)
        return np.array(out)

    _fails(pin_tournament, last_on_ties)


def test_gsm_mistakes_are_caught():
    _fails(pin_gsm, lambda S_T, S_R, p, a, b, ms: og.gsm(S_T, S_R, p, a, b, ms, sign_plus=True))
    _fails(pin_gsm, lambda S_T, S_R, p, a, b, ms: og.gsm(S_T, S_R, p, b, a, ms))
    _fails(pin_gsm, lambda S_T, S_R, p, a, b, ms: S_T[p] + (S_R[a] - S_R[b]))   # dropped ms


def test_elitism_mistakes_are_caught():
    def non_strict(F_T, F_O):
        b_P, b_O = int(np.argmin(F_T)), int(np.argmin(F_O))
        return (b_P, int(np.argmax(F_O))) if F_T[b_P] <= F_O[b_O] else None

    def replaces_best(F_T, F_O):
        d = og.elitism_decision(F_T, F_O)
        return None if d is None else (d[0], int(np.argmin(F_O)))

    _fails(pin_elitism, non_strict)
    _fails(pin_elitism, replaces_best)


def test_reconstruction_mistake_is_caught():
    """A wrong sign on the second random tree breaks predict == semantics."""
    import workloads as W
    w = W.TINY.replace(n_train=48, n_test=16, pop_size=24, n_random_trees=16)
    d = W.make_data(w)
    o = og.GSGP(og.Params(pop_size=24, n_random_trees=16), *d)
    o.init()
    o.evolve(6)

    def bad_reconstruct(trace, slot, r):
        parent, rt1, rt2, ms = trace
        c = np.zeros(r)
        for g in range(len(parent) - 1, -1, -1):
            if rt1[g][slot] >= 0:
                c[rt1[g][slot]] += ms[g][slot]
                c[rt2[g][slot]] += ms[g][slot]
            slot = parent[g][slot]
        return slot, c

    X_all = np.concatenate([d[0], d[2]])
    anc, c = bad_reconstruct(o.trace(), o.best_slot(), 16)
    y = og.predict(o.P, o.R, anc, c, og.feature_major(X_all))
    assert not np.allclose(y, o.S_T[o.best_slot()], rtol=1e-9, atol=1e-9)
