"""Host inputs reach the device by two routes: page-locked, 16-byte aligned
buffers are read by a kernel through their device-mapped address, any other
host memory is copied by cudaMemcpyAsync.  Both must stage the same bytes, so
a run loaded (and a model applied) from pinned, pinned-but-misaligned and
ordinary pageable arrays is bit for bit the same run."""
import numpy as np
import pytest

import workloads as W
from gpu_util import gpu_run

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2106_04034_gb300 as pkg  # noqa: E402

WL = W.TINY.replace(n_train=5000, n_test=1300, n_features=12, pop_size=96, n_random_trees=80)


def _pinned(a: np.ndarray, offset_floats: int = 0) -> np.ndarray:
    """A copy of a in page-locked memory, starting offset_floats floats into
    the pinned block (offset 1: 4-byte aligned only)."""
    flat = torch.empty(a.size + offset_floats, dtype=torch.float32).pin_memory()
    v = flat.numpy()[offset_floats:offset_floats + a.size].reshape(a.shape)
    v[...] = a
    v.flags.writeable = False
    _pinned.keep.append(flat)   # the pinned block outlives the view
    return v


_pinned.keep = []


def _run(data, X_new, G=6):
    torch.cuda.set_device(0)
    run, _, _ = gpu_run(WL, data=data)
    run.evolve(G)
    launches = run.info().kernel_launches
    y = run.predict(X_new)
    out = (run.fitness(), run.trace(), run.semantics(pkg.POOL_POPULATION), y,
           run.info().kernel_launches - launches)
    run.close()
    return out


@pytest.mark.parametrize("offset", [0, 1], ids=["pinned aligned", "pinned misaligned"])
def test_pinned_inputs_stage_the_same_bytes_as_pageable(offset):
    data = W.make_data(WL)
    X_new = np.ascontiguousarray(data[2][::-1])
    ref = _run(data, X_new)
    pinned = [_pinned(np.ascontiguousarray(a), offset) for a in data]
    got = _run(pinned, _pinned(X_new, offset))
    (f_tr, f_te), trace, sem, y, _ = got
    (g_tr, g_te), gtrace, gsem, gy, _ = ref
    assert np.array_equal(f_tr, g_tr) and np.array_equal(f_te, g_te)
    for a, b in zip(trace, gtrace):
        assert np.array_equal(a, b)
    assert np.array_equal(sem, gsem)
    assert np.array_equal(y, gy)
    if offset == 0:
        # the aligned pinned prediction input went through the staging kernel
        assert got[4] > ref[4], (got[4], ref[4])
    else:
        assert got[4] == ref[4]
