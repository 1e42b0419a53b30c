"""The boundary's failure statuses, provoked only in the allowed ways.

GSGP_E_OOM: the caller's device allocator (config.alloc) returns NULL on its
k-th request.  The failing call reports GSGP_E_OOM, the context can be
destroyed with every block the allocator handed out given back, and a
context that retries with a working allocator gives the same run as a fresh
one.

GSGP_E_TIMEOUT: gsgp_arm_barrier_fault bounds the persistent kernel's grid
barrier waits at a few thousand naps and starts its first barrier one
arrival short (as if one CTA never arrived), so every wait of that barrier
runs out (no fault, no trap, no unbounded wait).  The next synchronising call returns GSGP_E_TIMEOUT;
after gsgp_init the same context evolves exactly as a fresh run does."""
import ctypes as C

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

WL = W.TINY.replace(n_train=3000, n_test=700, pop_size=96, n_random_trees=80)


class FailingAllocator:
    """Device allocator hooks over torch's caching allocator that return NULL
    on request number `fail_at` (1-based; 0: never) and count what is
    outstanding."""

    def __init__(self, fail_at: int):
        self.fail_at = fail_at
        self.requests = 0
        self.live = {}

        def _alloc(user, nbytes, stream):
            self.requests += 1
            if self.requests == self.fail_at:
                return None
            ptr = int(torch.cuda.caching_allocator_alloc(int(nbytes), 0,
                                                         stream if stream else 0))
            self.live[ptr] = int(nbytes)
            return ptr

        def _free(user, ptr, stream):
            if ptr:
                assert ptr in self.live, "freed a block the allocator did not hand out"
                del self.live[ptr]
                torch.cuda.caching_allocator_delete(ptr)

        self.alloc_fn = B.ALLOC_FN(_alloc)
        self.free_fn = B.FREE_FN(_free)


def _config(w):
    p = oracle_params(w)
    cfg = pkg.default_config(
        seed=p.seed, run=p.run, pop_size=p.pop_size, n_random_trees=p.n_random_trees,
        pop_min_depth=p.pop_min_depth, pop_max_depth=p.pop_max_depth,
        rt_min_depth=p.rt_min_depth, rt_max_depth=p.rt_max_depth)
    cfg.stream = torch.cuda.current_stream().cuda_stream
    return cfg


def _fresh_result(w, data, G):
    run = pkg.Run(_config(w))
    run.load(*data)
    run.init()
    run.evolve(G)
    out = run.fitness(), run.trace()
    run.close()
    return out


def _requests_of_a_whole_run(w, data, G):
    a = FailingAllocator(0)
    cfg = _config(w)
    cfg.alloc, cfg.free = a.alloc_fn, a.free_fn
    run = pkg.Run(cfg)
    run.load(*data)
    run.init()
    run.evolve(G)
    run.close()
    assert not a.live
    return a.requests


@pytest.mark.parametrize("which", ["first", "middle", "last"])
def test_allocator_failure_reports_oom_and_the_context_recovers(which):
    torch.cuda.set_device(0)
    data = W.make_data(WL)
    G = 4
    total = _requests_of_a_whole_run(WL, data, G)
    assert total >= 3
    fail_at = {"first": 1, "middle": (total + 1) // 2, "last": total}[which]
    a = FailingAllocator(fail_at)
    cfg = _config(WL)
    cfg.alloc, cfg.free = a.alloc_fn, a.free_fn
    run = pkg.Run(cfg)
    with pytest.raises(pkg.GsgpError) as e:
        run.load(*data)
        run.init()
        run.evolve(G)
    assert e.value.status == B.E_OOM, str(e.value)
    assert "allocator returned NULL" in str(e.value)
    # the same context retries once the allocator works again
    a.fail_at = 0
    run.load(*data)
    run.init()
    run.evolve(G)
    (f_tr, f_te), trace = run.fitness(), run.trace()
    run.close()
    assert not a.live, f"{len(a.live)} device blocks not given back"
    (g_tr, g_te), gtrace = _fresh_result(WL, data, G)
    assert np.array_equal(f_tr, g_tr) and np.array_equal(f_te, g_te)
    for x, y in zip(trace, gtrace):
        assert np.array_equal(x, y)


def test_destroy_after_oom_gives_every_block_back():
    torch.cuda.set_device(0)
    data = W.make_data(WL)
    total = _requests_of_a_whole_run(WL, data, 2)
    for fail_at in range(1, total + 1):
        a = FailingAllocator(fail_at)
        cfg = _config(WL)
        cfg.alloc, cfg.free = a.alloc_fn, a.free_fn
        run = pkg.Run(cfg)
        with pytest.raises(pkg.GsgpError) as e:
            run.load(*data)
            run.init()
            run.evolve(2)
        assert e.value.status == B.E_OOM
        run.close()
        assert not a.live, (fail_at, len(a.live))


def test_barrier_timeout_is_reported_and_cleared_by_init():
    torch.cuda.set_device(0)
    run, data, _ = gpu_run(WL)
    run.set_evolve_shape(pkg.PATH_PERSISTENT)
    run.evolve(2)                                   # the shape is chosen
    assert run.info().evolve_path == pkg.PATH_PERSISTENT
    run.arm_barrier_fault(4096)                     # first barrier one arrival short
    with pytest.raises(pkg.GsgpError) as e:
        run.evolve(3)                               # with the log: synchronises
    assert e.value.status == B.E_TIMEOUT, str(e.value)
    # sticky until init
    with pytest.raises(pkg.GsgpError) as e:
        run.evolve(1)
    assert e.value.status == B.E_TIMEOUT
    run.init()
    G = 6
    run.evolve(G)
    got = run.fitness(), run.trace()
    run.close()
    want = _fresh_result(WL, data, G)
    assert np.array_equal(got[0][0], want[0][0]) and np.array_equal(got[0][1], want[0][1])
    for x, y in zip(got[1], want[1]):
        assert np.array_equal(x, y)
