"""Geometric semantic crossover on the GPU (p_crossover > 0: the crossover of
the original GSGP, offspring R T1 + (1 - R) T2 case by case with R a
sigma-wrapped random tree).  A run is replayed by the oracle (crossover
decisions, both tournaments, elitism, semantics and fitness); the kernel
paths and batching give bit-identical results; a checkpoint resumes a run
with crossover; and prediction, which replays the trace on the new cases in
float64, matches the best individual's semantics and the oracle's replay."""
import numpy as np
import pytest

import workloads as W
from gpu_util import RMSE_RTOL, gpu_run, hard_failures, replay, semantics_close
from oracle import gsgp as og

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2106_04034_gb300 as pkg  # noqa: E402

XO = W.TINY.replace(name="tiny with crossover")
CASES = {
    "f32": (XO, 0.5),
    "bf16": (XO.replace(sigma_bf16=True), 0.5),
    "linear": (XO.replace(init_mode=1, max_genes=127), 0.3),
    "always": (XO, 1.0),
}


def _best(run):
    F_tr, _ = run.fitness()
    return int(np.argmin(F_tr))


@pytest.mark.parametrize("case", list(CASES))
def test_replay_semantics_and_prediction(case):
    w, pc = CASES[case]
    run, data, p = gpu_run(w, p_crossover=pc)
    S_T0 = run.semantics(pkg.POOL_POPULATION)
    S_R = run.semantics(pkg.POOL_RANDOM)
    best_tr, _ = run.evolve(25)
    tr = run.trace()
    cross = (tr[1] >= 0) & (tr[2] <= -2)
    mut = (tr[1] >= 0) & (tr[2] >= 0)
    assert cross.any()
    if pc < 1.0:
        assert mut.any() and 0.2 < cross.mean() / (cross.mean() + mut.mean()) / pc < 1.8
    else:
        assert not mut.any()
    assert np.all(tr[3][cross] == 0)
    ref = og.GSGP(p, *data)
    ref.create_programs()
    ref.set_state(S_T0, S_R)
    checks = replay(ref, tr)
    assert not hard_failures(checks), hard_failures(checks)
    S = run.semantics(pkg.POOL_POPULATION)
    ok, _, _ = semantics_close(S, ref.S_T)
    assert ok.all(), np.argwhere(~ok)[:5]
    F_tr, _ = run.fitness()
    assert np.allclose(F_tr, ref.F_T, rtol=RMSE_RTOL)
    assert np.allclose(best_tr, ref.best_train, rtol=RMSE_RTOL)
    # no ancestor-plus-coefficients model for a run with crossover
    with pytest.raises(RuntimeError):
        run.best_trace()
    # prediction replays the trace: on the training and test cases it is the
    # best individual's semantics; on new cases the oracle's replay
    b = _best(run)
    y = run.predict(np.concatenate([data[0], data[2]]))
    ok, _, _ = semantics_close(S[b], y)
    assert ok.all()
    Xn = W.make_new_cases(w, 700)
    got = run.predict(Xn)
    want = og.predict_replay(tr, b, ref.P, ref.R, og.feature_major(Xn), p.protect_eps,
                             p.sigma_bf16, p.init_mode == 1)
    if p.sigma_bf16:
        # sigma of a random tree rounds to bf16 after a float32 logistic; the
        # two sides' float32 exp may differ by an ulp, which flips the rounding
        # of a rare value, so most cases agree to 1e-9 and all to 1e-2
        close = np.isclose(got, want, rtol=1e-9, atol=1e-9)
        assert close.mean() > 0.95
        assert np.allclose(got, want, rtol=1e-2, atol=1e-2)
    else:
        assert np.allclose(got, want, rtol=1e-9, atol=1e-9)
    # the device-pointer entry point gives the same values
    Xd = torch.from_numpy(np.ascontiguousarray(Xn, dtype=np.float32)).cuda()
    yd = torch.empty(len(Xn), dtype=torch.float64, device="cuda")
    run.predict_device(Xd, yd)
    torch.cuda.synchronize()
    assert np.array_equal(yd.cpu().numpy(), got)
    run.close()


def test_paths_and_batching_are_bit_identical():
    base, _, _ = gpu_run(XO, p_crossover=0.5)
    base.evolve(20, log=False)
    chained, _, _ = gpu_run(XO, p_crossover=0.5)
    chained.set_evolve_shape(pkg.PATH_CHAINED, 1, 2)
    chained.evolve(20, log=False)
    persist, _, _ = gpu_run(XO, p_crossover=0.5)
    persist.set_evolve_shape(pkg.PATH_PERSISTENT, 2, 4)
    persist.evolve(20, log=False)
    batched, _, _ = gpu_run(XO, p_crossover=0.5)
    other, _, _ = gpu_run(XO.replace(run=5), p_crossover=0.5)
    b = pkg.Batch([batched, other])
    b.evolve(20, log=False)
    for r in (chained, persist, batched):
        assert np.array_equal(base.semantics(pkg.POOL_POPULATION), r.semantics(pkg.POOL_POPULATION))
        for x, y in zip(base.trace(), r.trace()):
            assert np.array_equal(x, y)
    b.close()
    for r in (base, chained, persist, batched, other):
        r.close()


def test_tma_stream_refuses_crossover():
    run, _, _ = gpu_run(XO, p_crossover=0.5)
    with pytest.raises(RuntimeError):
        run.set_evolve_shape(pkg.PATH_PERSISTENT, 1, 0)
    run.close()


def test_checkpoint_resumes_a_run_with_crossover():
    straight, data, _ = gpu_run(XO, p_crossover=0.5)
    straight.evolve(16, log=False)
    a, _, _ = gpu_run(XO, p_crossover=0.5, data=data)
    a.evolve(7, log=False)
    ck = a.checkpoint()
    b, _, _ = gpu_run(XO, p_crossover=0.5, data=data)
    b.restore(ck)
    b.evolve(9, log=False)
    assert np.array_equal(straight.semantics(pkg.POOL_POPULATION), b.semantics(pkg.POOL_POPULATION))
    for x, y in zip(straight.trace(), b.trace()):
        assert np.array_equal(x, y)
    Xn = W.make_new_cases(XO, 200)
    assert np.array_equal(straight.predict(Xn), b.predict(Xn))
    # the probability is part of the run's identity
    c, _, _ = gpu_run(XO, p_crossover=0.25, data=data)
    with pytest.raises(RuntimeError):
        c.restore(ck)
    for r in (straight, a, b, c):
        r.close()


def test_prediction_of_pools_too_large_for_shared_memory():
    # 2m + r float64 values per case no longer fit one CTA's shared memory:
    # prediction takes one replay launch per generation instead of the tiles
    w = XO.replace(pop_size=10240, n_random_trees=10240)
    run, data, p = gpu_run(w, p_crossover=0.5)
    run.evolve(6, log=False)
    ref = og.GSGP(p, *data)
    ref.create_programs()
    Xn = W.make_new_cases(w, 300)
    got = run.predict(Xn)
    want = og.predict_replay(run.trace(), _best(run), ref.P, ref.R, og.feature_major(Xn),
                             p.protect_eps)
    assert np.allclose(got, want, rtol=1e-9, atol=1e-9)
    run.close()
