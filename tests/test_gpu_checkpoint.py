"""Checkpoint and restore: a run resumed from a checkpoint in a fresh
context continues bit for bit as the uninterrupted run (semantics, fitness,
trace, best-of-generation log, rebuilt model), for trees and linear genomes,
float32 and bf16 sigma, across the persistent kernel's launch boundary and
through a batch; and a checkpoint is refused by another configuration or
other data."""
import numpy as np
import pytest

import workloads as W
from gpu_util import gpu_run

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2106_04034_gb300 as pkg  # noqa: E402

BASE = W.MID.replace(n_train=3000, n_test=700, pop_size=200, n_random_trees=150)


def state(run):
    return (run.semantics(pkg.POOL_POPULATION), run.fitness(), run.trace(), run.info().generation,
            run.best_trace())


def assert_same(a, b):
    assert a[3] == b[3]
    assert np.array_equal(a[0], b[0])
    for x, y in zip(a[1], b[1]):
        assert np.array_equal(x, y)
    for x, y in zip(a[2], b[2]):
        assert np.array_equal(x, y)
    assert a[4]["best_slot"] == b[4]["best_slot"] and np.array_equal(a[4]["coef"], b[4]["coef"])


@pytest.mark.parametrize("w", [
    BASE,
    BASE.replace(sigma_bf16=True),
    BASE.replace(init_mode=1, max_genes=255),
], ids=["trees", "bf16", "genomes"])
def test_resume_is_bit_identical(w):
    a, data, p = gpu_run(w)
    log1 = a.evolve(41)                 # ends inside a persistent launch
    ck = a.checkpoint()
    log2 = a.evolve(30)                 # crosses the next 64-generation boundary
    b, _, _ = gpu_run(w, data=data)
    b.evolve(3, log=False)              # state that the restore must replace
    b.restore(ck)
    assert b.info().generation == 41
    assert np.array_equal(b.trace()[0], a.trace(0, 41)[0])
    log2b = b.evolve(30)
    assert np.array_equal(log2[0], log2b[0]) and np.array_equal(log2[1], log2b[1])
    assert_same(state(a), state(b))
    assert np.array_equal(a.predict(data[2]), b.predict(data[2]))
    a.close()
    b.close()


def test_restored_runs_evolve_in_a_batch():
    a, data, _ = gpu_run(BASE)
    a.evolve(10, log=False)
    ck = a.checkpoint()
    a.evolve(20, log=False)
    b, _, _ = gpu_run(BASE, data=data)
    c, _, _ = gpu_run(BASE.replace(run=9))
    b.restore(ck)
    batch = pkg.Batch([b, c])
    batch.evolve(20, log=False)
    assert_same(state(a), state(b))
    batch.close()
    for r in (a, b, c):
        r.close()


def test_checkpoint_is_refused_elsewhere():
    a, data, _ = gpu_run(BASE)
    a.evolve(5, log=False)
    ck = a.checkpoint()
    other, _, _ = gpu_run(BASE.replace(run=1), data=data)      # another run index
    with pytest.raises(pkg.GsgpError) as e:
        other.restore(ck)
    assert e.value.status == pkg.binding.E_INVALID
    y2 = data[1].copy()
    y2[0] += 1.0                                               # other targets
    moved, _, _ = gpu_run(BASE, data=(data[0], y2, data[2], data[3]))
    with pytest.raises(pkg.GsgpError):
        moved.restore(ck)
    with pytest.raises(pkg.GsgpError):
        a.restore(ck[:100])                                    # truncated
    bad = bytearray(ck)
    bad[:8] = b"XXXXXXXX"
    with pytest.raises(pkg.GsgpError):
        a.restore(bytes(bad))
    for r in (a, other, moved):
        r.close()
