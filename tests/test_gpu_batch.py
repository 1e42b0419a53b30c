"""Batched runs: uneven independent runs advanced by the batched persistent
kernel give, run by run, bit-identical semantics, fitness, traces and
best-of-generation logs to the same runs evolved alone (whose parity with
the oracle the other GPU tests establish); one batched run is also replayed
by the oracle directly.  Covers every batch shape, launch-boundary
crossings, interleaving with single-run evolve, runs on separate streams,
and the rebuilt models of batched runs."""
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

T = W.TINY
# uneven runs: sizes, feature counts, pools, depths and evolution settings differ
RUNS = [
    (T.replace(name="b0", n_train=300, n_test=77, pop_size=50, n_random_trees=30, run=0), {}),
    (T.replace(name="b1", n_features=13, n_train=2500, n_test=600, pop_size=333,
               n_random_trees=100, pop_max_depth=5, run=1, wid=7), dict(ms_mode=1, ms=0.3)),
    (T.replace(name="b2", n_features=5, n_train=1000, n_test=0, pop_size=128,
               n_random_trees=64, run=2, tournament_size=0), dict(elitism=False)),
    (T.replace(name="b3", n_features=20, n_train=5000, n_test=1250, pop_size=200,
               n_random_trees=257, run=3, tournament_size=7, ms=0.05), {}),
    (T.replace(name="b4", n_train=61, n_test=3, pop_size=2, n_random_trees=1, run=4), {}),
]


_STREAMS = []   # side streams of the runs, kept alive for the module


def make_runs(stream_per_run=False):
    out = []
    for w, over in RUNS:
        if stream_per_run:
            _STREAMS.append(torch.cuda.Stream())
            with torch.cuda.stream(_STREAMS[-1]):
                run, data, p = gpu_run(w, **over)
        else:
            run, data, p = gpu_run(w, **over)
        out.append((run, data, p))
    return out


def state(run):
    return (run.semantics(pkg.POOL_POPULATION), run.fitness(), run.trace(), run.info().generation)


def assert_same(a, b):
    sa, fa, ta, ga = a
    sb, fb, tb, gb = b
    assert ga == gb
    assert np.array_equal(sa, sb)
    for x, y in zip(fa, fb):
        assert np.array_equal(x, y)
    for x, y in zip(ta, tb):
        assert np.array_equal(x, y)


@pytest.fixture(scope="module")
def singles():
    """Each run evolved alone: states after 12 and after 70 generations."""
    torch.cuda.set_device(0)
    res = []
    for run, _, _ in make_runs():
        l1 = run.evolve(12)
        s12 = state(run)
        l2 = run.evolve(58)
        res.append(dict(s12=s12, s70=state(run), log=(np.concatenate([l1[0], l2[0]]),
                                                      np.concatenate([l1[1], l2[1]]))))
        run.close()
    return res


def test_batch_equals_single_runs(singles):
    runs = make_runs()
    batch = pkg.Batch([r for r, _, _ in runs])
    tr, te = batch.evolve(70)          # one graph-replayed launch of 64 + a launch of 6
    info = batch.info()
    assert info.runs == len(RUNS) and info.generations_per_launch == 64
    assert info.offspring == sum(w.pop_size for w, _ in RUNS)
    assert info.updates_per_generation == sum(w.pop_size * w.n_cases for w, _ in RUNS)
    assert info.kernel_launches >= 2 and info.grid >= 1
    for k, (run, _, _) in enumerate(runs):
        assert_same(state(run), singles[k]["s70"])
        assert np.array_equal(tr[k], singles[k]["log"][0])
        assert np.array_equal(te[k], singles[k]["log"][1])
    batch.close()
    for r, _, _ in runs:
        r.close()


@pytest.mark.parametrize("vec,opb", [(1, 1), (1, 2), (1, 4), (1, 8), (2, 1), (2, 2), (2, 4)])
def test_every_batch_shape_gives_identical_results(singles, vec, opb):
    runs = make_runs()
    batch = pkg.Batch([r for r, _, _ in runs])
    batch.set_shape(vec, opb)
    batch.evolve(5, log=False)
    batch.evolve(7, log=False)
    info = batch.info()
    assert info.tile_cases == 1024 * vec and info.offspring_per_cta == opb
    for k, (run, _, _) in enumerate(runs):
        assert_same(state(run), singles[k]["s12"])
    batch.close()
    for r, _, _ in runs:
        r.close()


def test_batch_interleaved_with_single_evolve(singles):
    """Runs keep working alone between batch calls: run 1 is advanced by
    itself, the batch continues every run from its own generation."""
    runs = make_runs()
    batch = pkg.Batch([r for r, _, _ in runs])
    batch.evolve(5, log=False)
    runs[1][0].evolve(7, log=False)
    batch.evolve(7, log=False)       # run 1 reaches 19, the others 12
    for k, (run, _, _) in enumerate(runs):
        if k != 1:
            assert_same(state(run), singles[k]["s12"])
    ref, _, _ = gpu_run(*RUNS[1][:1], **RUNS[1][1])
    ref.evolve(19, log=False)
    assert_same(state(runs[1][0]), state(ref))
    ref.close()
    batch.close()
    for r, _, _ in runs:
        r.close()


def test_batch_runs_on_separate_streams(singles):
    runs = make_runs(stream_per_run=True)
    batch = pkg.Batch([r for r, _, _ in runs])
    batch.evolve(12, log=False)
    for k, (run, _, _) in enumerate(runs):
        assert_same(state(run), singles[k]["s12"])
    batch.close()
    for r, _, _ in runs:
        r.close()


def test_batched_run_replays_in_the_oracle():
    runs = make_runs()
    S0 = [(r.semantics(pkg.POOL_POPULATION), r.semantics(pkg.POOL_RANDOM)) for r, _, _ in runs]
    batch = pkg.Batch([r for r, _, _ in runs])
    tr, te = batch.evolve(15)
    for k in (1, 2, 4):             # random step, paper mode, smallest pools
        run, data, p = runs[k]
        ref = og.GSGP(p, *data)
        ref.create_programs()
        ref.set_state(*S0[k])
        checks = replay(ref, run.trace())
        assert not hard_failures(checks), (k, hard_failures(checks))
        ok, _, _ = semantics_close(run.semantics(pkg.POOL_POPULATION), ref.S_T)
        assert ok.all()
        F_tr, _ = run.fitness()
        assert np.allclose(F_tr, ref.F_T, rtol=RMSE_RTOL)
        assert np.allclose(tr[k], ref.best_train, rtol=RMSE_RTOL)
    batch.close()
    for r, _, _ in runs:
        r.close()


def test_best_model_of_batched_runs():
    runs = make_runs()
    batch = pkg.Batch([r for r, _, _ in runs])
    batch.evolve(20, log=False)
    for run, data, p in runs:
        bt = run.best_trace()
        S = run.semantics(pkg.POOL_POPULATION)
        X_all = np.concatenate([data[0], data[2]]) if len(data[2]) else data[0]
        ok, _, _ = semantics_close(S[bt["best_slot"]], run.predict(X_all))
        assert ok.all()
    batch.close()
    for r, _, _ in runs:
        r.close()


def test_batch_kernel_timing():
    runs = make_runs()
    batch = pkg.Batch([r for r, _, _ in runs])
    batch.set_kernel_timing(True)
    batch.evolve(70, log=False)
    t = batch.kernel_times()
    assert len(t) == 2 and np.all(t > 0)
    batch.close()
    for r, _, _ in runs:
        r.close()


def test_batch_of_more_runs_than_one_launch_holds():
    """170 small runs: the batch splits them into launches of at most 160
    runs; runs on both sides of the split match their single-run evolution."""
    base = T.replace(n_train=40, n_test=9, pop_size=6, n_random_trees=5, pop_max_depth=3,
                     rt_max_depth=3)
    ws = [base.replace(run=k, n_train=40 + (k % 7)) for k in range(170)]
    runs = [gpu_run(w)[0] for w in ws]
    batch = pkg.Batch(runs)
    batch.evolve(66, log=False)
    assert batch.info().kernel_launches >= 4     # two blocks of runs, two chunks
    for k in (0, 159, 160, 169):
        ref, _, _ = gpu_run(ws[k])
        ref.evolve(66, log=False)
        assert_same(state(runs[k]), state(ref))
        ref.close()
    batch.close()
    for r in runs:
        r.close()
