"""The paper's linear-genome representation on the GPU (init_mode 1,
Sec. 2.2 "Initialization" and "Interpreter"): genomes bit-exact against the
oracle's, semantics of the population and the sigma-wrapped random trees
against the oracle's skip-rule / Out evaluation within the float32 error
bound, initial fitness, a replayed run, the rebuilt model, and bit-identical
results across paths, shapes and batching."""
import numpy as np
import pytest

import workloads as W
from gpu_util import (RMSE_RTOL, gpu_run, hard_failures, oracle_semantics_with_bounds, replay,
                      semantics_close)
from oracle import gsgp as og
from oracle import trees as ot

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2106_04034_gb300 as pkg  # noqa: E402

LIN = W.TINY.replace(name="tiny linear genomes", init_mode=1, max_genes=127)
LIN_LONG = W.TINY.replace(name="long linear genomes", init_mode=1, max_genes=2047,
                          pop_size=48, n_random_trees=40, n_train=2000, n_test=500)


@pytest.mark.parametrize("w", [LIN, LIN_LONG], ids=["k127", "k2047"])
def test_genomes_bit_exact(w):
    run, data, p = gpu_run(w)
    ref = og.GSGP(p, *data)
    ref.create_programs()
    for pool, mine in ((pkg.POOL_POPULATION, ref.P), (pkg.POOL_RANDOM, ref.R)):
        g, c, L = run.programs(pool)
        assert g.shape == (mine[0].shape[0], w.max_genes)
        assert np.array_equal(L, mine[2]) and np.all(L == w.max_genes)
        assert np.array_equal(g, mine[0])
        assert np.array_equal(c.view(np.uint32), mine[1].view(np.uint32))
    run.close()


@pytest.mark.parametrize("w", [LIN, LIN_LONG], ids=["k127", "k2047"])
def test_semantics_and_fitness(w):
    run, data, p = gpu_run(w)
    ref = og.GSGP(p, *data)
    ref.create_programs()
    S_T = run.semantics(pkg.POOL_POPULATION)
    S_R = run.semantics(pkg.POOL_RANDOM)
    vT, eT = oracle_semantics_with_bounds(ref.P, ref.X, p.protect_eps, linear=True)
    vR, eR = oracle_semantics_with_bounds(ref.R, ref.X, p.protect_eps, logistic=True, linear=True)
    for name, got, v, e in (("population", S_T, vT, eT), ("random trees", S_R, vR, eR)):
        ok, _, _ = semantics_close(got, v, e, label=f"linear genomes k={w.max_genes}, {name}")
        assert ok.all(), np.argwhere(~ok)[:5]
    # the deepest stack of each pool fits the interpreter (checked by init)
    assert max(ot.genome_max_stack(gg) for gg in ref.P[0]) <= 32
    F_tr, _ = run.fitness()
    o_tr, _ = og.rmse(S_T.astype(np.float64), ref.t, ref.n_train)
    # below 1e15 no float32 square can overflow; long genomes also reach far
    # larger values, whose float32 squared errors overflow to +inf fitness
    fin = np.isfinite(o_tr) & (o_tr < 1e15)
    assert fin.sum() >= len(o_tr) // 4
    assert np.allclose(F_tr[fin], o_tr[fin], rtol=RMSE_RTOL, atol=0)
    assert np.all(np.isinf(F_tr[~fin]) | (F_tr[~fin] >= 1e14))
    run.close()


def test_replay_and_model():
    w = LIN
    run, data, p = gpu_run(w)
    S_T0 = run.semantics(pkg.POOL_POPULATION)
    S_R = run.semantics(pkg.POOL_RANDOM)
    best_tr, _ = run.evolve(30)
    ref = og.GSGP(p, *data)
    ref.create_programs()
    ref.set_state(S_T0, S_R)
    checks = replay(ref, run.trace())
    assert not hard_failures(checks), hard_failures(checks)
    ok, _, _ = semantics_close(run.semantics(pkg.POOL_POPULATION), ref.S_T)
    assert ok.all()
    F_tr, _ = run.fitness()
    assert np.allclose(F_tr, ref.F_T, rtol=RMSE_RTOL)
    assert np.allclose(best_tr, ref.best_train, rtol=RMSE_RTOL)
    # the rebuilt model: predict(train + test) is the best's semantics, and
    # on new cases it equals the oracle's float64 model of linear genomes
    bt = run.best_trace()
    S = run.semantics(pkg.POOL_POPULATION)
    y = run.predict(np.concatenate([data[0], data[2]]))
    ok, _, _ = semantics_close(S[bt["best_slot"]], y)
    assert ok.all()
    Xn = W.make_new_cases(w, 500)
    want = og.predict(ref.P, ref.R, bt["ancestor"], bt["coef"], og.feature_major(Xn),
                      p.protect_eps, linear=True)
    assert np.allclose(run.predict(Xn), want, rtol=1e-9, atol=1e-9)
    run.close()


def test_paths_and_batching_are_bit_identical():
    base, _, _ = gpu_run(LIN)
    base.evolve(20, log=False)
    chained, _, _ = gpu_run(LIN)
    chained.set_evolve_shape(pkg.PATH_CHAINED, 1, 2)
    chained.evolve(20, log=False)
    batched, _, _ = gpu_run(LIN)
    other, _, _ = gpu_run(LIN.replace(run=5))
    b = pkg.Batch([batched, other])
    b.evolve(20, log=False)
    for r in (chained, batched):
        assert np.array_equal(base.semantics(pkg.POOL_POPULATION), r.semantics(pkg.POOL_POPULATION))
        for x, y in zip(base.trace(), r.trace()):
            assert np.array_equal(x, y)
    b.close()
    for r in (base, chained, batched, other):
        r.close()
