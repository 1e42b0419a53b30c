"""Case sharding, host side (no GPU).

* plan / slice_cases: contiguous 1024-case-aligned slices that cover the
  problem once, training cases first, including shards that hold test cases
  only and a ragged last shard.
* the boundary's checks of shard contexts (no device work: they fail before
  any CUDA call).
* the exchange and the decisions on two gloo ranks: each rank runs the
  float64 oracle's generation steps (Algorithm 1: tournament, GSM, RMSE,
  survival with elitism) on its own slice of the cases, with fitness taken
  from per-chunk squared-error sums that the ranks all-reduce (each rank's
  array zero outside its chunks).  Every rank must make the same selections
  and survival decisions, and the run must equal, bit for bit, the same
  steps on all the cases in one process with the chunk sums added in the
  same order."""
import ctypes as C
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import paper_2106_04034_gb300 as pkg  # noqa: E402
import workloads as W  # noqa: E402
from oracle import gsgp as og  # noqa: E402
from paper_2106_04034_gb300 import binding as B  # noqa: E402
from paper_2106_04034_gb300 import shard  # noqa: E402


@pytest.mark.parametrize("n_train,n_test,k", [(5000, 1250, 2), (5000, 1250, 3), (2000, 3000, 3),
                                              (1024, 0, 1), (3072, 1, 4), (100, 5000, 2)])
def test_plan_covers_the_cases_on_chunk_boundaries(n_train, n_test, k):
    p = shard.plan(n_train, n_test, k)
    assert len(p) == k
    n = n_train + n_test
    pos, tr = 0, 0
    for i, (c0, a, b) in enumerate(p):
        assert c0 == pos and c0 % 1024 == 0 and a + b >= 1
        if i < k - 1:
            assert (a + b) % 1024 == 0
        assert a == max(0, min(c0 + a + b, n_train) - c0)    # training cases first
        pos += a + b
        tr += a
    assert pos == n and tr == n_train
    sizes = [a + b for _, a, b in p[:-1]]
    assert max(sizes, default=0) - min(sizes, default=0) <= 1024


def test_plan_refuses_more_shards_than_chunks():
    with pytest.raises(ValueError):
        shard.plan(1000, 100, 3)


def test_slice_cases_takes_each_shard_its_rows():
    w = W.TINY.replace(n_train=2500, n_test=700)
    data = W.make_data(w)
    X_all = np.concatenate([data[0], data[2]])
    y_all = np.concatenate([data[1], data[3]])
    for c0, a, b in shard.plan(w.n_train, w.n_test, 3):
        Xtr, ytr, Xte, yte = shard.slice_cases(data, c0, a, b)
        assert len(Xtr) == a and len(Xte) == b
        assert np.array_equal(np.concatenate([Xtr, Xte]), X_all[c0:c0 + a + b])
        assert np.array_equal(np.concatenate([ytr, yte]), y_all[c0:c0 + a + b])


def test_shard_contexts_check_their_slice_before_any_device_work():
    lib = pkg.load_library()
    r = pkg.Run(pop_size=8, n_random_trees=4)
    X = np.zeros((2048, 3), np.float32)
    y = np.zeros(2048, np.float32)
    for bad in ((-1024, 5000, 10), (100, 5000, 10), (6000, 5000, 10), (0, 0, 10), (0, 10, -1)):
        assert lib.gsgp_shard_configure(r.ctx, *bad) == B.E_INVALID, bad
    # shard 1 of 5000 + 1000 cases holds [1024, ...): 3976 training cases at most
    assert lib.gsgp_shard_configure(r.ctx, 1024, 5000, 1000) == B.OK
    p = lambda a: a.ctypes.data_as(C.c_void_p)  # noqa: E731
    # not a multiple of 1024 although not the last shard
    assert lib.gsgp_load(r.ctx, p(X), p(y), 1000, 3, None, None, 0) == B.E_INVALID
    # 2048 cases from 1024 are all training cases: a test part is refused
    assert lib.gsgp_load(r.ctx, p(X), p(y), 1024, 3, p(X), p(y), 1024) == B.E_INVALID
    assert b"training cases" in lib.gsgp_last_error(r.ctx)
    # beyond the last case
    big = np.zeros((6144, 3), np.float32)
    assert lib.gsgp_load(r.ctx, p(big), p(big[:, 0].copy()), 6144, 3, None, None, 0) == \
        B.E_INVALID
    # stepping calls need a loaded, initialised shard
    assert lib.gsgp_shard_generation(r.ctx) == B.E_STATE
    assert lib.gsgp_shard_finish(r.ctx) == B.E_STATE
    assert lib.gsgp_shard_partials(r.ctx, None, None, None) == B.E_STATE
    r.close()
    u = pkg.Run(pop_size=8, n_random_trees=4)
    assert lib.gsgp_shard_generation(u.ctx) == B.E_STATE     # not a shard
    u.close()


# ------------------------------------------------------ gloo exchange -----
WL = W.TINY.replace(n_train=2500, n_test=600, pop_size=40, n_random_trees=30)
G = 6


def _chunk_sums(S, t, n_train_all, case0):
    """(rows, chunks, 2) float64 squared-error sums of the cases of S (which
    start at global case case0) per 1024-case chunk, split train / test."""
    rows, n = S.shape
    chunks = -(-n // 1024)
    out = np.zeros((rows, chunks, 2))
    d = (S - t[None, :]) ** 2
    glob = case0 + np.arange(n)
    for c in range(chunks):
        sl = slice(c * 1024, min(n, (c + 1) * 1024))
        tr = glob[sl] < n_train_all
        out[:, c, 0] = d[:, sl][:, tr].sum(axis=1)
        out[:, c, 1] = d[:, sl][:, ~tr].sum(axis=1)
    return out


def _rmse(partials, n_train_all, n_test_all):
    """RMSE from the complete chunk sums, chunks added in a fixed order."""
    tr = np.zeros(partials.shape[0])
    te = np.zeros(partials.shape[0])
    for c in range(partials.shape[1]):
        tr = tr + partials[:, c, 0]
        te = te + partials[:, c, 1]
    f_tr = np.sqrt(tr / n_train_all)
    f_te = np.sqrt(te / n_test_all) if n_test_all else np.zeros_like(te)
    return np.where(np.isfinite(f_tr), f_tr, np.inf), np.where(np.isfinite(f_te), f_te, np.inf)


def _sharded_run(rank, world, exchange):
    """The oracle's steps on this rank's slice with exchanged chunk sums."""
    data = W.make_data(WL)
    p = og.Params(seed=WL.seed, run=WL.run, pop_size=WL.pop_size,
                  n_random_trees=WL.n_random_trees, pop_min_depth=WL.pop_min_depth,
                  pop_max_depth=WL.pop_max_depth, rt_min_depth=WL.rt_min_depth,
                  rt_max_depth=WL.rt_max_depth)
    full = og.GSGP(p, *data)
    full.create_programs()
    full.compute_semantics()
    c0, a, b = shard.plan(WL.n_train, WL.n_test, world)[rank]
    cols = slice(c0, c0 + a + b)
    S_T, S_R, t = full.S_T[:, cols].copy(), full.S_R[:, cols].copy(), full.t[cols]
    chunks_all = -(-WL.n_cases // 1024)

    def fitness(S):
        mine = _chunk_sums(S, t, WL.n_train, c0)
        arr = np.zeros((S.shape[0], chunks_all, 2))
        arr[:, c0 // 1024:c0 // 1024 + mine.shape[1]] = mine
        return _rmse(exchange(arr), WL.n_train, WL.n_test)

    F_T, Fte_T = fitness(S_T)
    trace = []
    for g in range(G):
        cand, ra, rb, ms = og.selection_draws(p, g)
        par = og.tournament(F_T, cand)
        S_O = og.gsm(S_T, S_R, par, ra, rb, ms)
        F_O, Fte_O = fitness(S_O)
        ent = [par.copy(), ra.copy(), rb.copy()]
        e = og.elitism_decision(F_T, F_O)
        if e is not None:
            bP, w = e
            S_O[w], F_O[w], Fte_O[w] = S_T[bP], F_T[bP], Fte_T[bP]
            ent[0][w], ent[1][w], ent[2][w] = bP, -1, -1
        trace.append(np.stack(ent))
        S_T, F_T, Fte_T = S_O, F_O, Fte_O
    return S_T, F_T, Fte_T, np.stack(trace)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)

    def exchange(arr):
        t = torch.from_numpy(arr)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return t.numpy()

    S, F, Fte, tr = _sharded_run(rank, world, exchange)
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), S=S, F=F, Fte=Fte, trace=tr)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_equal_one_process(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [np.load(tmp_path / f"rank{k}.npz") for k in range(world)]
    S1, F1, Fte1, tr1 = _sharded_run(0, 1, lambda arr: arr)
    for k in range(world):
        assert np.array_equal(r[k]["F"], F1) and np.array_equal(r[k]["Fte"], Fte1)
        assert np.array_equal(r[k]["trace"], tr1)
    assert np.array_equal(np.concatenate([r[0]["S"], r[1]["S"]], axis=1), S1)
    assert tr1.shape == (G, 3, WL.pop_size)
