"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): every rank
runs an independent replica (its own run index, hence its own data and
Philox streams, with the same shapes), the job's time is the slowest
rank's, and the job's throughput counts the units of all ranks.  There is
no collective on the data path: each rank's oracle run evolves on its own,
and only the timing is reduced."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402
import workloads as W  # noqa: E402
from oracle import gsgp as og  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = bench.replica_workload(W.TINY.replace(generations=3), rank)
    data = W.make_data(w)
    p = og.Params(seed=w.seed, run=w.run, pop_size=w.pop_size,
                  n_random_trees=w.n_random_trees, pop_min_depth=w.pop_min_depth,
                  pop_max_depth=w.pop_max_depth, rt_min_depth=w.rt_min_depth,
                  rt_max_depth=w.rt_max_depth)
    o = og.GSGP(p, *data)
    o.init()
    o.evolve(w.generations)
    # the job's time is the slowest rank's; throughput counts every rank
    fake_seconds = 1.0 + rank
    t = bench.max_over_ranks(fake_seconds, world, device="cpu")
    v = bench.job_value(w.pop_size * w.n_cases * w.generations, world, t)
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), run=w.run, t=t, v=v,
             X=data[0], best=np.array(o.best_train), programs=o.P[0])
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_on_gloo(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [np.load(tmp_path / f"rank{k}.npz") for k in range(world)]
    assert int(r[0]["run"]) != int(r[1]["run"])                  # independent replicas
    assert r[0]["X"].shape == r[1]["X"].shape                     # of the same workload
    assert not np.array_equal(r[0]["X"], r[1]["X"])               # with their own data
    assert not np.array_equal(r[0]["programs"], r[1]["programs"])  # and their own programs
    for k in range(world):
        assert float(r[k]["t"]) == 2.0                            # max over ranks
        w = W.TINY.replace(generations=3)
        assert float(r[k]["v"]) == w.pop_size * w.n_cases * 3 * world / 2.0
        assert np.all(np.diff(r[k]["best"]) <= 0)                 # each replica evolved


def test_single_rank_helpers_need_no_process_group():
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_value(10.0, 1, 2.0) == 5.0
    w = bench.replica_workload(W.MID, 0)
    assert w == W.MID
