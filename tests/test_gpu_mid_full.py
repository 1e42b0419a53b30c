"""Full-size parity on the mid workload, the benchmark's default (64
features, 20,000 + 5,000 cases, m = r = 1024, depths 2-6), in the launch
configuration bench.py times (persistent path, autotuned shape): programs
bit-exact; every initial semantic value within the float32 error bound of the
oracle's; 20 generations of the GPU's trace replayed by the oracle (every
draw, tournament and survival decision checked), with every semantic value
and fitness after them; and the rebuilt model on new cases."""
import numpy as np
import pytest

import workloads as W
from gpu_util import (RMSE_RTOL, gpu_run, hard_failures, oracle_semantics_with_bounds, replay,
                      semantics_close)
from oracle import gsgp as og

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2106_04034_gb300 as pkg  # noqa: E402

G = 20


def test_mid_full_size():
    w = W.MID
    run, data, p = gpu_run(w)
    ref = og.GSGP(p, *data)
    ref.create_programs()
    for pool, mine in ((pkg.POOL_POPULATION, ref.P), (pkg.POOL_RANDOM, ref.R)):
        g, c, L = run.programs(pool)
        assert np.array_equal(g, mine[0]) and np.array_equal(L, mine[2])
        assert np.array_equal(c.view(np.uint32), mine[1].view(np.uint32))
    S_T0 = run.semantics(pkg.POOL_POPULATION)
    S_R = run.semantics(pkg.POOL_RANDOM)
    vT, eT = oracle_semantics_with_bounds(ref.P, ref.X, p.protect_eps)
    ok, _, _ = semantics_close(S_T0, vT, eT, label="mid full size, population")
    assert ok.all()
    del vT, eT
    vR, eR = oracle_semantics_with_bounds(ref.R, ref.X, p.protect_eps, logistic=True)
    ok, _, _ = semantics_close(S_R, vR, eR, label="mid full size, random trees")
    assert ok.all()
    del vR, eR
    ref.set_state(S_T0, S_R)
    best_tr, best_te = run.evolve(G)
    info = run.info()
    assert info.evolve_path == pkg.PATH_PERSISTENT
    checks = replay(ref, run.trace())
    assert not hard_failures(checks), hard_failures(checks)
    ok, _, _ = semantics_close(run.semantics(pkg.POOL_POPULATION), ref.S_T)
    assert ok.all()
    F_tr, F_te = run.fitness()
    assert np.allclose(F_tr, ref.F_T, rtol=RMSE_RTOL)
    assert np.allclose(F_te, ref.F_T_te, rtol=RMSE_RTOL)
    assert np.allclose(best_tr, ref.best_train, rtol=RMSE_RTOL)
    assert np.allclose(best_te, ref.best_test, rtol=RMSE_RTOL)
    bt = run.best_trace()
    Xn = W.make_new_cases(w, 2000)
    want = og.predict(ref.P, ref.R, bt["ancestor"], bt["coef"], og.feature_major(Xn),
                      p.protect_eps)
    assert np.allclose(run.predict(Xn), want, rtol=1e-9, atol=1e-9)
    run.close()
