"""The precision variant at full size: the large workload (1.25M cases,
m=1024, r=512) run 2000 generations on the GPU with sigma(R) stored as
float32 and as bf16.  Cases are independent columns of every semantic
matrix, so the GPU's trace can be replayed exactly in the float64 oracle on
a subset of the cases (every 4096th): with the GPU's own initial semantics
(same rounded sigma) the offspring semantics must agree within
1e-4 (1 + |v|); with the oracle's exact float64 sigma the difference is what
the storage precision costs, reported and loosely bounded.  (The oracle's
subset fitness cannot judge the GPU's selections, which use all cases: only
the draws are checked here; the selections are checked at full size by the
other tests.)"""
import numpy as np
import pytest

import workloads as W
from gpu_util import gpu_run, semantics_close
from oracle import gsgp as og
from oracle import interp as oi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2106_04034_gb300 as pkg  # noqa: E402

G = 2000
STRIDE = 4096


def subset_rows(run, pool, rows, cols, block=64):
    out = []
    for r0 in range(0, rows, block):
        n = min(block, rows - r0)
        out.append(run.semantics(pool, r0, n)[:, cols])
    return np.concatenate(out)


def replay_subset(p, S_T0, S_R, trace):
    """Follow the GPU's trace with the oracle's draws and GSM (Sec. 2) in
    float64 on the sampled cases; the draws must be the oracle's, bit for
    bit, and an elite entry copies the recorded parent's row."""
    S = np.asarray(S_T0, dtype=np.float64)
    R = np.asarray(S_R, dtype=np.float64)
    par, r1, r2, ms = trace
    for g in range(len(par)):
        _, a, b, ms_g = og.selection_draws(p, g)
        mut = r1[g] >= 0
        assert mut.sum() >= len(mut) - 1
        assert np.array_equal(r1[g][mut], a[mut]) and np.array_equal(r2[g][mut], b[mut])
        assert np.array_equal(ms[g][mut], ms_g[mut])
        S_new = og.gsm(S, R, par[g], a, b, ms_g)
        for w in np.nonzero(~mut)[0]:
            S_new[w] = S[par[g][w]]
        S = S_new
    return S


def exact_sigma(p, data, cols):
    Xtr, ytr, Xte, yte = data
    X = np.concatenate([Xtr, Xte])[cols]
    ref = og.GSGP(og.Params(**{**p.__dict__, "sigma_bf16": False}), X, np.zeros(len(cols)),
                  X[:0], np.zeros(0))
    ref.create_programs()
    return oi.pool_semantics(*ref.R, ref.X, p.protect_eps, logistic=True)


@pytest.mark.parametrize("bf16", [False, True], ids=["f32-sigma", "bf16-sigma"])
def test_full_size_precision_variant(bf16, capsys):
    w = W.LARGE_BF16.replace(generations=G, sigma_bf16=bf16)
    run, data, p = gpu_run(w)
    cols = np.arange(0, w.n_cases, STRIDE)
    S_T0 = subset_rows(run, pkg.POOL_POPULATION, w.pop_size, cols)
    S_R = subset_rows(run, pkg.POOL_RANDOM, w.n_random_trees, cols)
    best_tr, _ = run.evolve(G)
    trace = run.trace()
    S_G = subset_rows(run, pkg.POOL_POPULATION, w.pop_size, cols)
    run.close()
    # same rounded sigma: the GPU's semantics within 1e-4 (1 + |v|)
    S_ref = replay_subset(p, S_T0, S_R, trace)
    ok, _, _ = semantics_close(S_G, S_ref)
    assert ok.all(), np.argwhere(~ok)[:5]
    assert np.all(np.diff(best_tr) <= 0)
    # exact float64 sigma: what the storage precision costs
    S_ex = replay_subset(p, S_T0, exact_sigma(p, data, cols), trace)
    fin = np.isfinite(S_ex)
    err = np.max(np.abs(S_G[fin] - S_ex[fin]) / (1 + np.abs(S_ex[fin])))
    with capsys.disabled():
        print(f"\n[large, {'bf16' if bf16 else 'f32'} sigma, {G} generations, "
              f"{len(cols)} sampled cases] max |s - s64| / (1 + |s64|) = {err:.3e}")
    assert err < (2e-2 if bf16 else 1e-4)
