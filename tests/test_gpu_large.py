"""Full-size parity on the large workload (1.25M cases, m=1024, r=512) in
the launch configuration bench.py times (default path and autotuned shape):
programs bit-exact, sampled semantics against the oracle, fitness against the
float64 RMSE of the GPU's own rows, every draw and tournament of three
generations, the per-element mutation identity on sampled offspring, and the
prediction of the rebuilt model on new cases."""
import numpy as np
import pytest

import workloads as W
from gpu_util import RMSE_RTOL, gpu_run, oracle_semantics_with_bounds, semantics_close
from oracle import gsgp as og

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2106_04034_gb300 as pkg  # noqa: E402


@pytest.fixture(scope="module")
def large():
    torch.cuda.set_device(0)
    w = W.LARGE
    run, data, p = gpu_run(w)
    ref = og.GSGP(p, *data)
    ref.create_programs()
    yield w, run, data, p, ref
    run.close()


def test_large_programs_bit_exact(large):
    w, run, data, p, ref = large
    for pool, mine in ((pkg.POOL_POPULATION, ref.P), (pkg.POOL_RANDOM, ref.R)):
        g, c, L = run.programs(pool)
        assert np.array_equal(g, mine[0]) and np.array_equal(L, mine[2])
        assert np.array_equal(c.view(np.uint32), mine[1].view(np.uint32))


def test_large_sampled_semantics_and_fitness(large):
    w, run, data, p, ref = large
    rng = np.random.default_rng(3)
    rows = np.sort(rng.choice(w.pop_size, 48, replace=False))
    rrows = np.sort(rng.choice(w.n_random_trees, 48, replace=False))
    cols = np.sort(rng.choice(w.n_cases, 4096, replace=False))
    Xs = ref.X[:, cols]
    sub = lambda P, r: tuple(a[r] for a in P)  # noqa: E731
    vT, eT = oracle_semantics_with_bounds(sub(ref.P, rows), Xs, p.protect_eps)
    vR, eR = oracle_semantics_with_bounds(sub(ref.R, rrows), Xs, p.protect_eps, logistic=True)
    F_tr, F_te = run.fitness()
    got = np.empty(vT.shape, np.float32)
    for k, i in enumerate(rows):
        full = run.semantics(pkg.POOL_POPULATION, int(i), 1)[0]
        got[k] = full[cols]
        tr, te = og.rmse(full.astype(np.float64)[None, :], ref.t, ref.n_train)
        if np.isfinite(tr[0]) and tr[0] < 1e30:
            assert abs(F_tr[i] - tr[0]) <= RMSE_RTOL * tr[0]
            assert abs(F_te[i] - te[0]) <= RMSE_RTOL * te[0]
    ok, _, _ = semantics_close(got, vT, eT, label="large, sampled population")
    assert ok.all()
    got = np.empty(vR.shape, np.float32)
    for k, i in enumerate(rrows):
        got[k] = run.semantics(pkg.POOL_RANDOM, int(i), 1)[0][cols]
    ok, _, _ = semantics_close(got, vR, eR, label="large, sampled random trees")
    assert ok.all()


def test_large_generations(large):
    """Three generations: every slot's draws bit-exact against Philox and
    every tournament won by the candidate the GPU's own fitness ranks first;
    then one more generation with the mutation identity checked on sampled
    offspring over all 1.25M cases."""
    w, run, data, p, ref = large
    m = w.pop_size
    for _ in range(3):
        g = run.info().generation
        F_prev, _ = run.fitness()
        run.evolve(1)
        par, r1, r2, ms = (x[0] for x in run.trace(g, 1))
        cand, a, b, ms_want = og.selection_draws(p, g)
        mut = r1 >= 0
        assert mut.sum() >= m - 1                    # at most one elite copy
        assert np.array_equal(r1[mut], a[mut]) and np.array_equal(r2[mut], b[mut])
        assert np.array_equal(ms[mut], ms_want[mut])
        win = og.tournament(F_prev, cand)
        assert np.array_equal(par[mut], win[mut])
    g = run.info().generation
    rng = np.random.default_rng(5)
    sample = np.sort(rng.choice(m, 8, replace=False))
    cand, _, _, _ = og.selection_draws(p, g)
    F_prev, _ = run.fitness()
    win = og.tournament(F_prev, cand)
    prev = {int(win[i]): run.semantics(pkg.POOL_POPULATION, int(win[i]), 1)[0] for i in sample}
    run.evolve(1)
    par, r1, r2, ms = (x[0] for x in run.trace(g, 1))
    for i in sample:
        if r1[i] < 0:
            continue
        assert par[i] == win[i]
        sa = run.semantics(pkg.POOL_RANDOM, int(r1[i]), 1)[0]
        sb = run.semantics(pkg.POOL_RANDOM, int(r2[i]), 1)[0]
        want = (np.float64(ms[i]) * (sa - sb).astype(np.float64)
                + prev[int(par[i])].astype(np.float64)).astype(np.float32)
        got = run.semantics(pkg.POOL_POPULATION, int(i), 1)[0]
        assert np.all(np.abs(got - want) <= np.spacing(np.abs(want)))


def test_large_predict_new_cases(large):
    w, run, data, p, ref = large
    bt = run.best_trace()
    Xn = W.make_new_cases(w, 3000)
    y = run.predict(Xn)
    want = og.predict(ref.P, ref.R, bt["ancestor"], bt["coef"], og.feature_major(Xn),
                      p.protect_eps)
    assert np.allclose(y, want, rtol=1e-9, atol=1e-9)
    info = run.info()
    assert info.evolve_path == pkg.PATH_PERSISTENT and info.evolve_tile_cases > 0
