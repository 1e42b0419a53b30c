"""gsgp_mutate_noalloc, the entry point for callers that cannot allocate
device memory (for example code running inside a framework's CUDA-graph
capture, where cudaMalloc is forbidden), checked against the library's own
generation step (gsgp_evolve) on two calls in a row.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

import workloads as W
from gpu_util import RMSE_RTOL, SEM_RTOL, gpu_run

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2106_04034_gb300 as pkg  # noqa: E402
from paper_2106_04034_gb300.binding import E_INVALID, mutate_noalloc  # noqa: E402

# several 1024-case chunks plus a ragged tail; m not a multiple of anything
WL = W.MID.replace(name="mid-scaled", n_train=5000, n_test=1250, pop_size=250,
                   n_random_trees=200)


def _rows(a, ld):
    t = torch.zeros((a.shape[0], ld), dtype=torch.float32, device="cuda")
    t[:, :a.shape[1]] = torch.from_numpy(np.ascontiguousarray(a))
    return t


def test_noalloc_matches_evolve_on_two_calls_in_a_row():
    torch.cuda.set_device(0)
    run, data, _ = gpu_run(WL)
    m, n = WL.pop_size, WL.n_cases
    ld = (n + 63) // 64 * 64
    sig = _rows(run.semantics(pkg.POOL_RANDOM), ld)
    target = torch.zeros(ld, dtype=torch.float32, device="cuda")
    target[:n] = torch.from_numpy(np.concatenate([data[1], data[3]]))
    off = torch.empty((m, ld), dtype=torch.float32, device="cuda")
    rtr = torch.empty(m, dtype=torch.float64, device="cuda")
    rte = torch.empty(m, dtype=torch.float64, device="cuda")
    for call in range(2):
        prev = run.semantics(pkg.POOL_POPULATION)
        run.evolve(1)
        cur = run.semantics(pkg.POOL_POPULATION)
        f_tr, f_te = run.fitness()
        par, r1, r2, ms = (x[0] for x in run.trace(call, 1))
        # the elite slot's entry (parent, -1, -1, 0) is a plain copy of its parent
        idx = [torch.from_numpy(np.ascontiguousarray(v, dtype=np.int32)).cuda()
               for v in (par, np.maximum(r1, 0), np.maximum(r2, 0))]
        step = torch.from_numpy(np.ascontiguousarray(ms, dtype=np.float32)).cuda()
        parents = _rows(prev, ld)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        mutate_noalloc(parents, sig, target, WL.n_train, WL.n_test, idx[0], idx[1], idx[2], step,
                       off, rtr, rte)
        torch.cuda.synchronize()
        if call == 1:   # the first call may load the kernels' module
            assert torch.cuda.mem_get_info()[0] == free_before
        got = off[:, :n].cpu().numpy()
        # the same per-case arithmetic and summation order as gsgp_evolve:
        # equal values (the elite's copy of its parent included), and within
        # the tests' tolerances in any case
        assert np.all(np.abs(got - cur) <= SEM_RTOL * (1 + np.abs(cur)))
        assert np.allclose(rtr.cpu().numpy(), f_tr, rtol=RMSE_RTOL, atol=0)
        assert np.allclose(rte.cpu().numpy(), f_te, rtol=RMSE_RTOL, atol=0)
        assert np.array_equal(got, cur, equal_nan=True)
        assert np.array_equal(rtr.cpu().numpy(), f_tr)
        assert np.array_equal(rte.cpu().numpy(), f_te)
    run.close()


def test_noalloc_refuses_an_in_place_call():
    """offspring == parents would race (rows are read while others are
    written); the library refuses it before any launch."""
    torch.cuda.set_device(0)
    m, n = 4, 2048
    rows = torch.zeros((m, n), dtype=torch.float32, device="cuda")
    sig = torch.zeros((2, n), dtype=torch.float32, device="cuda")
    target = torch.zeros(n, dtype=torch.float32, device="cuda")
    i32 = torch.zeros(m, dtype=torch.int32, device="cuda")
    f32 = torch.zeros(m, dtype=torch.float32, device="cuda")
    r = torch.zeros(m, dtype=torch.float64, device="cuda")
    # straight through the C ABI: the binding would refuse it first
    lib = pkg.load_library()
    msg = ctypes.create_string_buffer(256)
    ptr = [t.data_ptr() for t in (rows, sig, target, i32, f32, r)]
    st = lib.gsgp_mutate_noalloc(ptr[0], ptr[1], n, ptr[2], n - 48, 48, ptr[3], ptr[3], ptr[3],
                                 ptr[4], m, ptr[0], ptr[5], ptr[5],
                                 torch.cuda.current_stream().cuda_stream, msg, 256)
    torch.cuda.synchronize()
    assert st == E_INVALID and b"overlap" in msg.value


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch.cuda.set_device(0)
    m, n = 200, 700 * 1024          # 200 * 700 chunks > 131072 partial sums
    ld = n
    rows = torch.zeros((2, ld), dtype=torch.float32, device="cuda")
    target = torch.zeros(ld, dtype=torch.float32, device="cuda")
    i32 = torch.zeros(m, dtype=torch.int32, device="cuda")
    f32 = torch.zeros(m, dtype=torch.float32, device="cuda")
    out = torch.zeros((m, ld), dtype=torch.float32, device="cuda")
    r = torch.zeros(m, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.GsgpError) as e:
        mutate_noalloc(rows, rows, target, n - 100, 100, i32, i32, i32, f32, out, r, r)
    assert e.value.status == E_INVALID and "scratch" in str(e.value)
