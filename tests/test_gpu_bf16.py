"""Random-tree semantics stored as bfloat16 (the precision variant): storage
rounding, replay parity with the same rounded values, prediction, and the
error against exact float64 sigma (reported, loosely bounded)."""
import numpy as np
import pytest

import workloads as W
from gpu_util import RMSE_RTOL, gpu_run, hard_failures, replay, semantics_close
from oracle import gsgp as og
from oracle import interp as oi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2106_04034_gb300 as pkg  # noqa: E402
from gpu_util import oracle_semantics_with_bounds  # noqa: E402

MID_S = W.MID.replace(name="mid-scaled", n_train=5000, n_test=1250, pop_size=250,
                      n_random_trees=200, sigma_bf16=True)


def _bf16_ulp(v):
    e = np.floor(np.log2(np.maximum(np.abs(v), 1e-30)))
    return 2.0 ** (e - 7)


def test_bf16_sigma_is_the_rounded_float_sigma():
    run, data, p = gpu_run(MID_S)
    ref = og.GSGP(p, *data)
    ref.create_programs()
    S_R = run.semantics(pkg.POOL_RANDOM).astype(np.float64)
    v, e = oracle_semantics_with_bounds(ref.R, ref.X, p.protect_eps, logistic=True)
    want = oi.bf16_round(v)
    # every stored value is a bf16 number
    bits = S_R.astype(np.float32).view(np.uint32)
    assert np.all(bits & 0xFFFF == 0)
    fin = np.isfinite(e)
    exact = (S_R == want) & fin
    assert exact.sum() / fin.sum() > 0.995
    # the rest sit one bf16 step away: float32 and float64 sigma straddle a
    # rounding boundary
    off = fin & ~exact
    assert np.all(np.abs(S_R[off] - want[off]) <= _bf16_ulp(want[off]) * 1.0001)
    run.close()


def test_bf16_replay_with_the_same_rounded_sigma():
    run, data, p = gpu_run(MID_S)
    S_T0 = run.semantics(pkg.POOL_POPULATION)
    S_R = run.semantics(pkg.POOL_RANDOM)
    best_tr, _ = run.evolve(24)
    ref = og.GSGP(p, *data)
    ref.create_programs()
    ref.set_state(S_T0, S_R)
    checks = replay(ref, run.trace())
    assert not hard_failures(checks)
    ok, _, _ = semantics_close(run.semantics(pkg.POOL_POPULATION), ref.S_T)
    assert ok.all()
    F_tr, F_te = run.fitness()
    assert np.allclose(F_tr, ref.F_T, rtol=RMSE_RTOL)
    assert np.allclose(F_te, ref.F_T_te, rtol=RMSE_RTOL)
    assert np.allclose(best_tr, ref.best_train, rtol=RMSE_RTOL)
    run.close()


def test_bf16_predict_reproduces_training_semantics():
    run, data, p = gpu_run(MID_S)
    run.evolve(20)
    bt = run.best_trace()
    assert bt["sigma_dtype"] == pkg.SIGMA_BF16
    S = run.semantics(pkg.POOL_POPULATION)
    y = run.predict(np.concatenate([data[0], data[2]]))
    ok, _, _ = semantics_close(S[bt["best_slot"]], y)
    assert ok.all()
    run.close()


def test_bf16_error_against_exact_sigma_is_reported(capsys):
    """Float64 replay of the GPU lineage with exact sigma (not rounded):
    the difference measures what bf16 storage costs; it is reported and only
    loosely bounded (the tight parity check is the same-sigma replay)."""
    G = 60
    report = {}
    for bf in (False, True):
        w = MID_S.replace(sigma_bf16=bf)
        run, data, p = gpu_run(w)
        S_T0 = run.semantics(pkg.POOL_POPULATION)
        run.evolve(G)
        p_exact = og.Params(**{**p.__dict__, "sigma_bf16": False})
        ref = og.GSGP(p_exact, *data)
        ref.create_programs()
        ref.compute_semantics()                      # exact float64 sigma
        ref.set_state(S_T0, ref.S_R)
        par, r1, r2, ms = run.trace()
        for g in range(G):                           # follow the GPU's decisions
            ref.generation({"parent": par[g], "rt1": r1[g], "rt2": r2[g], "ms": ms[g]}, {})
        S = run.semantics(pkg.POOL_POPULATION).astype(np.float64)
        F_tr, _ = run.fitness()
        sem_err = np.max(np.abs(S - ref.S_T) / (1 + np.abs(ref.S_T)))
        fin = np.isfinite(ref.F_T)
        rmse_err = np.max(np.abs(F_tr[fin] - ref.F_T[fin]) / ref.F_T[fin])
        report["bf16" if bf else "f32"] = (sem_err, rmse_err)
        run.close()
    with capsys.disabled():
        for k, (a, b) in report.items():
            print(f"\n[{k} sigma] {G} generations, max |s - s64|/(1+|s64|) = {a:.3e}, "
                  f"max relative RMSE error = {b:.3e}")
    assert report["f32"][0] < 1e-4 and report["f32"][1] < 1e-5
    assert report["bf16"][0] < 2e-2 and report["bf16"][1] < 2e-2
