"""Case-sharded runs on the GPU: shard contexts that each hold a
1024-case-aligned slice of the cases and exchange their per-chunk partial
sums (gsgp_shard_*) give, bit for bit, the programs' initial fitness, every
selection and survival decision, the trace, the fitness and the semantics of
one unsharded run over all the cases, and the same model.  The shards run on
one GPU here, driven from one process; the exchange is the element-wise sum
of their arrays (on several GPUs it is an all-reduce).  Cases: two and three
shards, a train/test boundary inside a shard and inside a chunk, a shard
with test cases only, a ragged last chunk, bf16 sigma, crossover and the
paper's linear genomes."""
import numpy as np
import pytest

import workloads as W
from gpu_util import gpu_run, oracle_params

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2106_04034_gb300 as pkg  # noqa: E402
from paper_2106_04034_gb300 import binding as B  # noqa: E402
from paper_2106_04034_gb300 import shard  # noqa: E402

MID_S = W.MID.replace(name="mid-scaled", n_train=5000, n_test=1250, pop_size=250,
                      n_random_trees=200)
G = 23

CASES = {
    "2 shards": (MID_S, 2, {}),
    "3 shards": (MID_S, 3, {}),
    "test-only shard": (MID_S.replace(n_train=2000, n_test=3000), 3, {}),
    "bf16 sigma": (MID_S.replace(sigma_bf16=True), 2, {}),
    "crossover": (MID_S, 3, {"p_crossover": 0.5}),
    "linear genomes": (MID_S.replace(init_mode=1, max_genes=127), 2, {}),
}


def _shards(w, k, over):
    data = W.make_data(w)
    runs = []
    for c0, a, b in shard.plan(w.n_train, w.n_test, k):
        run = _config_run(w, over)
        run.shard_configure(c0, w.n_train, w.n_test)
        Xtr, ytr, Xte, yte = shard.slice_cases(data, c0, a, b)
        run.load(Xtr, ytr, Xte if b else None, yte if b else None)
        runs.append(run)
    return runs, data


def _config_run(w, over):
    p = oracle_params(w, **over)
    cfg = pkg.default_config(
        seed=p.seed, run=p.run, pop_size=p.pop_size, n_random_trees=p.n_random_trees,
        pop_min_depth=p.pop_min_depth, pop_max_depth=p.pop_max_depth,
        rt_min_depth=p.rt_min_depth, rt_max_depth=p.rt_max_depth, const_lo=p.const_lo,
        const_hi=p.const_hi, protect_eps=p.protect_eps, ms=p.ms,
        tournament_size=p.tournament_size,
        sigma_dtype=pkg.SIGMA_BF16 if p.sigma_bf16 else pkg.SIGMA_F32,
        init_mode=p.init_mode, max_genes=p.max_genes, p_crossover=p.p_crossover)
    cfg.stream = torch.cuda.current_stream().cuda_stream
    return pkg.Run(cfg)


@pytest.mark.parametrize("case", sorted(CASES))
def test_shards_equal_one_run(case):
    torch.cuda.set_device(0)
    w, k, over = CASES[case]
    ref, data, _ = gpu_run(w, **over)
    F0 = ref.fitness()
    ref.evolve(G)
    runs, _ = _shards(w, k, over)
    shard.init(runs)
    for r in runs:   # initial fitness from the exchanged interpreter sums
        for a, b in zip(r.fitness(), F0):
            assert np.array_equal(a, b)
    shard.evolve(runs, G)
    want_S = ref.semantics(pkg.POOL_POPULATION)
    got_S = np.concatenate([r.semantics(pkg.POOL_POPULATION) for r in runs], axis=1)
    assert np.array_equal(got_S, want_S)
    want_R = ref.semantics(pkg.POOL_RANDOM)
    got_R = np.concatenate([r.semantics(pkg.POOL_RANDOM) for r in runs], axis=1)
    assert np.array_equal(got_R, want_R)
    for r in runs:
        for a, b in zip(r.fitness(), ref.fitness()):
            assert np.array_equal(a, b)
        for a, b in zip(r.trace(), ref.trace()):
            assert np.array_equal(a, b)
        assert r.info().generation == G
    X_new = W.make_new_cases(w, 777)
    y_ref = ref.predict(X_new)
    for r in runs:
        assert np.array_equal(r.predict(X_new), y_ref)
    if not over.get("p_crossover"):
        bt, bt_ref = runs[-1].best_trace(), ref.best_trace()
        assert bt["best_slot"] == bt_ref["best_slot"]
        assert np.array_equal(bt["coef"], bt_ref["coef"])
    for r in runs:
        r.close()
    ref.close()


def test_shard_call_order_is_enforced():
    torch.cuda.set_device(0)
    runs, _ = _shards(MID_S, 2, {})
    r = runs[0]
    with pytest.raises(pkg.GsgpError) as e:
        r.shard_generation()                      # before init
    assert e.value.status == B.E_STATE
    for x in runs:
        x.init()
    with pytest.raises(pkg.GsgpError) as e:
        r.shard_generation()                      # exchange of init pending
    assert e.value.status == B.E_STATE
    shard.local_sum(runs)
    for x in runs:
        x.shard_finish()
    with pytest.raises(pkg.GsgpError) as e:
        r.evolve(2)                               # shards step one generation at a time
    assert e.value.status == B.E_STATE
    with pytest.raises(pkg.GsgpError) as e:
        r.checkpoint()
    assert e.value.status == B.E_STATE
    with pytest.raises(pkg.GsgpError) as e:
        r.shard_finish()                          # nothing pending
    assert e.value.status == B.E_STATE
    shard.evolve(runs, 2)
    assert r.info().generation == 2
    for x in runs:
        x.close()
