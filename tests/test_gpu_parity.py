"""CUDA path against the CPU oracle, element by element, through the C ABI."""
import numpy as np
import pytest

import workloads as W
from gpu_util import (RMSE_RTOL, SEM_RTOL, gpu_run, hard_failures, oracle_params,
                      oracle_semantics_with_bounds, replay, semantics_close)
from oracle import gsgp as og
from oracle import interp as oi
from oracle import philox as op

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2106_04034_gb300 as pkg  # noqa: E402

TINY = W.TINY
# mid-size shape scaled down so the oracle finishes in seconds: several
# 2048-case tiles plus a ragged tail (6250 cases), m not a multiple of the
# offspring group, depth 2-6 programs over 64 features
MID_S = W.MID.replace(name="mid-scaled", n_train=5000, n_test=1250, pop_size=250,
                      n_random_trees=200)


@pytest.fixture(autouse=True)
def _device():
    torch.cuda.set_device(0)
    yield
    torch.cuda.synchronize()


# ------------------------------------------------------------------ RNG ---
def test_rng_words_bit_exact():
    total = 0
    for seed, run, gp, ind, n in [(1, 0, 0, 0, 4096), (1, 0, 0x80000001, 17, 1000),
                                  (0xDEADBEEFCAFEF00D, 7, 123456, 99999, 65536),
                                  (2, 3, 0x80000002, 0xFFFFFFFF, 33)]:
        got = pkg.rng_words(seed, run, gp, ind, n)
        want = op.stream_words(seed, run, gp, ind, n)
        assert np.array_equal(got, want)
        total += n
    # a million words over many streams
    for ind in range(16):
        got = pkg.rng_words(5, 1, ind * 3, ind, 65536)
        assert np.array_equal(got, op.stream_words(5, 1, ind * 3, ind, 65536))
        total += 65536
    assert total >= 1_000_000


# ---------------------------------------------------------- programs -------
@pytest.mark.parametrize("w", [TINY, MID_S], ids=["tiny", "mid-scaled"])
def test_programs_bit_exact(w):
    run, data, p = gpu_run(w)
    ref = og.GSGP(p, *data)
    ref.create_programs()
    for pool, mine in ((pkg.POOL_POPULATION, ref.P), (pkg.POOL_RANDOM, ref.R)):
        g, c, L = run.programs(pool)
        assert np.array_equal(L, mine[2])
        assert np.array_equal(g, mine[0])
        assert np.array_equal(c.view(np.uint32), mine[1].view(np.uint32))
    run.close()


def test_programs_bit_exact_deep_and_paper_constants():
    w = TINY.replace(pop_size=24, n_random_trees=12, pop_min_depth=0, pop_max_depth=10,
                     rt_min_depth=9, rt_max_depth=10, const_lo=1.0, const_hi=10.0,
                     n_train=70, n_test=0)
    run, data, p = gpu_run(w, p_grow=0.8, p_feature=0.3)
    ref = og.GSGP(p, *data)
    ref.create_programs()
    for pool, mine in ((pkg.POOL_POPULATION, ref.P), (pkg.POOL_RANDOM, ref.R)):
        g, c, L = run.programs(pool)
        assert np.array_equal(g, mine[0]) and np.array_equal(L, mine[2])
        assert np.array_equal(c.view(np.uint32), mine[1].view(np.uint32))
    run.close()


# -------------------------------------------------------- semantics --------
@pytest.mark.parametrize("w", [TINY, MID_S], ids=["tiny", "mid-scaled"])
def test_initial_semantics_and_fitness(w):
    run, data, p = gpu_run(w)
    ref = og.GSGP(p, *data)
    ref.create_programs()
    S_T = run.semantics(pkg.POOL_POPULATION)
    S_R = run.semantics(pkg.POOL_RANDOM)
    vT, eT = oracle_semantics_with_bounds(ref.P, ref.X, p.protect_eps)
    vR, eR = oracle_semantics_with_bounds(ref.R, ref.X, p.protect_eps, logistic=True)
    name = w.name.split(":")[0]
    okT, _, _ = semantics_close(S_T, vT, eT, label=f"{name} (scaled), population")
    okR, _, _ = semantics_close(S_R, vR, eR, label=f"{name} (scaled), random trees")
    assert okT.all() and okR.all()
    # fitness: the float64 RMSE of the GPU's own float32 semantics (reduction
    # check) and the oracle's RMSE where no case was ambiguous
    F_tr, F_te = run.fitness()
    own_tr, own_te = og.rmse(S_T.astype(np.float64), ref.t, ref.n_train)
    fin = np.isfinite(own_tr) & (own_tr < 1e30)
    assert np.allclose(F_tr[fin], own_tr[fin], rtol=RMSE_RTOL, atol=0)
    fin = np.isfinite(own_te) & (own_te < 1e30)
    assert np.allclose(F_te[fin], own_te[fin], rtol=RMSE_RTOL, atol=0)
    # against the oracle's exact RMSE: |RMSE(s') - RMSE(s)| <= RMS(s' - s), so
    # the float32 semantic error bound carries over to the RMSE
    o_tr, _ = og.rmse(vT, ref.t, ref.n_train)
    with np.errstate(all="ignore"):
        eb = np.sqrt(np.mean(eT[:, :ref.n_train] ** 2, axis=1))
    fin = np.isfinite(eb) & np.isfinite(o_tr)
    assert fin.mean() > 0.9
    assert np.all(np.abs(F_tr[fin] - o_tr[fin]) <= RMSE_RTOL * o_tr[fin] + eb[fin])
    run.close()


# ------------------------------------------------ evolution (replay) -------
@pytest.mark.parametrize("w,G", [(TINY, 50), (MID_S, 24)], ids=["tiny", "mid-scaled"])
def test_trace_replay(w, G):
    run, data, p = gpu_run(w)
    S_T0 = run.semantics(pkg.POOL_POPULATION)
    S_R = run.semantics(pkg.POOL_RANDOM)
    best_tr, best_te = run.evolve(G)
    trace = run.trace()
    ref = og.GSGP(p, *data)
    ref.create_programs()
    ref.set_state(S_T0, S_R)
    checks = replay(ref, trace)
    assert not hard_failures(checks), hard_failures(checks)
    S_G = run.semantics(pkg.POOL_POPULATION)
    ok, _, _ = semantics_close(S_G, ref.S_T)
    assert ok.all()
    F_tr, F_te = run.fitness()
    fin = np.isfinite(ref.F_T)
    assert np.allclose(F_tr[fin], ref.F_T[fin], rtol=RMSE_RTOL, atol=0)
    assert np.all(np.isinf(F_tr[~fin]))
    fin = np.isfinite(ref.F_T_te)
    assert np.allclose(F_te[fin], ref.F_T_te[fin], rtol=RMSE_RTOL, atol=0)
    assert np.allclose(best_tr, ref.best_train, rtol=RMSE_RTOL)
    assert np.allclose(best_te, ref.best_test, rtol=RMSE_RTOL)
    assert np.all(np.diff(best_tr) <= 0)          # elitism: best never worsens
    run.close()


def test_offspring_equal_recorded_combination_every_generation():
    """Trace invariant on every slot of every generation: offspring =
    parent + ms (sR[rt1] - sR[rt2]) in float32 (one fused multiply-add),
    or an exact copy of the parent for the elite."""
    w = MID_S.replace(pop_size=66, n_random_trees=40)
    run, data, p = gpu_run(w)
    S_R = run.semantics(pkg.POOL_RANDOM)
    prev = run.semantics(pkg.POOL_POPULATION)
    for g in range(6):
        run.evolve(1)
        cur = run.semantics(pkg.POOL_POPULATION)
        par, r1, r2, ms = (x[0] for x in run.trace(g, 1))
        for i in range(w.pop_size):
            if r1[i] < 0:
                assert np.array_equal(cur[i], prev[par[i]])
            else:
                d = (S_R[r1[i]] - S_R[r2[i]]).astype(np.float32)
                want = (np.float64(ms[i]) * d.astype(np.float64)
                        + prev[par[i]].astype(np.float64)).astype(np.float32)
                ulp = np.spacing(np.abs(want))
                assert np.all(np.abs(cur[i] - want) <= ulp)
        prev = cur
    run.close()


def test_independent_oracle_run_tiny():
    """The oracle run on its own (its own programs, semantics and decisions)
    reaches the same lineage and RMSE series as the GPU on the tiny case."""
    w = TINY
    run, data, p = gpu_run(w)
    gtr, gte = run.evolve(w.generations)
    par, r1, r2, ms = run.trace()
    ref = og.GSGP(p, *data)
    ref.init()
    ref.evolve(w.generations)
    opar, o1, o2, oms = ref.trace()
    same = (par == opar).all(axis=1) & (r1 == o1).all(axis=1) & (ms == oms).all(axis=1)
    # decisions agree generation by generation (a near tie between float32 and
    # float64 fitness would show up here as the first differing generation)
    assert same.all(), np.nonzero(~same)[0][:5]
    assert np.allclose(gtr, ref.best_train, rtol=1e-4)
    assert np.allclose(gte, ref.best_test, rtol=1e-4)
    run.close()


# ---------------------------------------------------- best individual ------
@pytest.mark.parametrize("w,G", [(TINY, 30), (MID_S, 12)], ids=["tiny", "mid-scaled"])
def test_best_trace_and_predict(w, G):
    run, data, p = gpu_run(w)
    S_T0 = run.semantics(pkg.POOL_POPULATION)
    S_R = run.semantics(pkg.POOL_RANDOM)
    run.evolve(G)
    bt = run.best_trace()
    S_G = run.semantics(pkg.POOL_POPULATION)
    F_tr, F_te = run.fitness()
    b = bt["best_slot"]
    assert b == int(np.argmin(F_tr))
    assert bt["best_train_rmse"] == F_tr[b] and bt["best_test_rmse"] == F_te[b]
    # the lineage agrees with the full trace and rebuilds the oracle's model
    trace = run.trace()
    anc, coef = og.reconstruct(trace, b, w.n_random_trees)
    assert anc == bt["ancestor"]
    assert np.array_equal(coef, bt["coef"])
    ref = og.GSGP(p, *data)
    ref.create_programs()
    L = bt["ancestor_length"]
    assert np.array_equal(bt["anc_genes"][:L], ref.P[0][anc, :L])
    # predict == the best's semantics (closed-form invariant of GSM)
    X_all = np.concatenate([data[0], data[2]])
    y = run.predict(X_all)
    ok, _, _ = semantics_close(S_G[b], y)
    assert ok.all()
    # predict == the oracle's float64 model on new cases
    Xn = W.make_new_cases(w, 777)
    yn = run.predict(Xn)
    want = og.predict(ref.P, ref.R, anc, coef, og.feature_major(Xn), p.protect_eps)
    assert np.allclose(yn, want, rtol=1e-9, atol=1e-9)
    run.close()


def test_bit_reproducible_runs():
    outs = []
    for _ in range(2):
        run, data, p = gpu_run(MID_S)
        run.evolve(10)
        outs.append((run.semantics(pkg.POOL_POPULATION), run.fitness(), run.trace()))
        run.close()
    (s1, f1, t1), (s2, f2, t2) = outs
    assert np.array_equal(s1, s2)
    assert np.array_equal(f1[0], f2[0]) and np.array_equal(f1[1], f2[1])
    for a, b in zip(t1, t2):
        assert np.array_equal(a, b)


# ------------------------------------------------------------ edge cases ---
@pytest.mark.parametrize("over", [
    dict(n_test=0),                                  # no test cases
    dict(n_train=3, n_test=2),                       # fewer cases than one float4 row
    dict(pop_size=2, n_random_trees=1),              # smallest pools; rt1 == rt2
    dict(pop_size=131),                              # ragged offspring group
], ids=["no-test", "five-cases", "m2-r1", "m131"])
def test_edge_shapes_replay(over):
    w = TINY.replace(**over)
    run, data, p = gpu_run(w)
    S_T0 = run.semantics(pkg.POOL_POPULATION)
    S_R = run.semantics(pkg.POOL_RANDOM)
    run.evolve(9)
    ref = og.GSGP(p, *data)
    ref.create_programs()
    ref.set_state(S_T0, S_R)
    checks = replay(ref, run.trace())
    assert not hard_failures(checks)
    ok, _, _ = semantics_close(run.semantics(pkg.POOL_POPULATION), ref.S_T)
    assert ok.all()
    F_tr, F_te = run.fitness()
    assert np.allclose(F_tr, ref.F_T, rtol=RMSE_RTOL)
    if w.n_test == 0:
        assert np.all(F_te == 0)
    run.close()


@pytest.mark.parametrize("over", [
    dict(tournament_size=0, elitism=False),          # the paper's setting
    dict(ms_mode=1, ms=0.5),                         # random mutation step
    dict(tournament_size=7),
], ids=["paper-mode", "uniform-ms", "tournament7"])
def test_variants_replay(over):
    w = TINY
    run, data, p = gpu_run(w, **over)
    S_T0 = run.semantics(pkg.POOL_POPULATION)
    S_R = run.semantics(pkg.POOL_RANDOM)
    run.evolve(12)
    ref = og.GSGP(p, *data)
    ref.create_programs()
    ref.set_state(S_T0, S_R)
    checks = replay(ref, run.trace())
    assert not hard_failures(checks)
    ok, _, _ = semantics_close(run.semantics(pkg.POOL_POPULATION), ref.S_T)
    assert ok.all()
    par, r1, _, _ = run.trace()
    if over.get("tournament_size") == 0:
        assert np.all(par == np.arange(w.pop_size)) and np.all(r1 >= 0)
    run.close()


def test_evolve_in_pieces_equals_one_call():
    a, _, _ = gpu_run(TINY)
    a.evolve(21)
    b, _, _ = gpu_run(TINY)
    for n in (1, 8, 3, 9):     # crosses the graph replay size and direct launches
        b.evolve(n)
    assert np.array_equal(a.semantics(pkg.POOL_POPULATION), b.semantics(pkg.POOL_POPULATION))
    for x, y in zip(a.trace(), b.trace()):
        assert np.array_equal(x, y)
    a.close()
    b.close()


def test_device_load_and_torch_allocator():
    w = TINY
    data = W.make_data(w)
    run_h, _, p = gpu_run(w, data=data)
    run_h.evolve(5)
    cfg = pkg.default_config(pop_size=w.pop_size, n_random_trees=w.n_random_trees,
                             pop_min_depth=2, pop_max_depth=4, rt_min_depth=2, rt_max_depth=4)
    cfg.stream = torch.cuda.current_stream().cuda_stream
    run_d = pkg.Run(cfg, torch_allocator=True)
    t = [torch.from_numpy(a).cuda() for a in data]
    run_d.load_device(*t)
    run_d.init()
    run_d.evolve(5)
    assert np.array_equal(run_h.semantics(pkg.POOL_POPULATION),
                          run_d.semantics(pkg.POOL_POPULATION))
    Xn = torch.from_numpy(W.make_new_cases(w, 100)).cuda()
    y = torch.zeros(100, dtype=torch.float64, device="cuda")
    run_d.predict_device(Xn, y)
    torch.cuda.synchronize()
    assert np.allclose(y.cpu().numpy(), run_h.predict(Xn.cpu().numpy()), rtol=0, atol=0)
    bad = t[0].clone()
    bad[3, 1] = float("nan")
    with pytest.raises(pkg.GsgpError):
        run_d.load_device(bad, t[1], t[2], t[3])
    run_h.close()
    run_d.close()


@pytest.mark.parametrize("path,vec,opb", [
    (pkg.PATH_CHAINED, 1, 2), (pkg.PATH_CHAINED, 2, 4), (pkg.PATH_CHAINED, 4, 8),
    (pkg.PATH_PERSISTENT, 1, 1), (pkg.PATH_PERSISTENT, 1, 4), (pkg.PATH_PERSISTENT, 1, 8),
    (pkg.PATH_PERSISTENT, 1, 16),
    (pkg.PATH_PERSISTENT, 2, 2), (pkg.PATH_PERSISTENT, 2, 8), (pkg.PATH_PERSISTENT, 2, 16),
    (pkg.PATH_PERSISTENT, 1, 0), (pkg.PATH_PERSISTENT, 2, 0), (pkg.PATH_PERSISTENT, 4, 0),
])
def test_every_path_and_shape_gives_identical_results(path, vec, opb):
    """The generation path (persistent cooperative kernel or chained
    launches) and the stream shape change only the work split: the
    per-chunk summation order is fixed, so semantics, fitness and trace are
    bit-identical to the default run's."""
    base, _, _ = gpu_run(MID_S)
    base.evolve(70)          # crosses a persistent-kernel launch boundary (64)
    other, _, _ = gpu_run(MID_S)
    other.set_evolve_shape(path, vec, opb)
    for n in (1, 8, 61):     # direct launches, graph replays, several chunks
        other.evolve(n)
    info = other.info()
    assert info.evolve_path == path
    assert info.evolve_tile_cases == 1024 * vec and info.evolve_offspring_per_cta == opb
    if opb == 0:          # TMA-staged stream: 9 warps, one CTA per SM
        assert 1 <= info.evolve_grid <= 2 * 152
    assert np.array_equal(base.semantics(pkg.POOL_POPULATION), other.semantics(pkg.POOL_POPULATION))
    for a, b in zip(base.fitness(), other.fitness()):
        assert np.array_equal(a, b)
    for a, b in zip(base.trace(), other.trace()):
        assert np.array_equal(a, b)
    bt1, bt2 = base.best_trace(), other.best_trace()
    assert bt1["best_slot"] == bt2["best_slot"] and np.array_equal(bt1["coef"], bt2["coef"])
    base.close()
    other.close()


@pytest.mark.parametrize("path", [pkg.PATH_PERSISTENT, pkg.PATH_CHAINED])
def test_kernel_timing_is_reported(path):
    run, _, _ = gpu_run(MID_S)
    run.set_evolve_shape(path)
    run.set_kernel_timing(True)
    run.evolve(19)
    t = run.kernel_times()
    info = run.info()
    per = info.evolve_generations_per_launch
    assert t.shape == (-(-19 // per),) and np.all(t > 0) and np.all(t < 1000)
    assert run.kernel_times().size == 0  # cleared
    run.set_kernel_timing(False)
    run.close()


def test_default_path_is_persistent():
    run, _, _ = gpu_run(TINY)
    run.evolve(3)
    info = run.info()
    assert info.evolve_path == pkg.PATH_PERSISTENT and info.evolve_grid >= 1
    assert info.evolve_offspring_per_cta > 0     # the autotuner picks a register-stream shape
    run.close()


def test_non_finite_host_inputs_are_rejected_on_the_device():
    """gsgp_load and gsgp_predict check host inputs after copying them to the
    device; a rejected load leaves the loaded data and the run untouched."""
    w = TINY
    data = W.make_data(w)
    run, _, _ = gpu_run(w, data=data)
    ref, _, _ = gpu_run(w, data=data)
    for k, v in ((0, np.nan), (1, np.inf), (2, -np.inf), (3, np.nan)):
        bad = [a.copy() for a in data]
        bad[k].reshape(-1)[len(bad[k].reshape(-1)) // 2] = v
        with pytest.raises(pkg.GsgpError):
            run.load(*bad)
    run.evolve(4, log=False)
    ref.evolve(4, log=False)
    assert np.array_equal(run.semantics(pkg.POOL_POPULATION), ref.semantics(pkg.POOL_POPULATION))
    Xn = W.make_new_cases(w, 50)
    y = run.predict(Xn)
    Xn[7, 0] = np.nan
    with pytest.raises(pkg.GsgpError):
        run.predict(Xn)
    Xn[7, 0] = 0.5
    assert np.all(np.isfinite(run.predict(Xn))) and np.all(np.isfinite(y))
    run.close()
    ref.close()
