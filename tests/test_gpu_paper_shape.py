"""The paper's speed-up shape at full size (Sec. 3: linear genomes of
k = 2047 genes, l = 1,024 features, n = 81,920 + 20,480 cases,
m = r = 10,240), initialised exactly as the benchmark times it: sampled
genomes bit-exact against the oracle's generator, their semantics over every
case bit-exact against a float32 evaluation of the oracle's genome (skip
rule, register Out), sampled random trees' sigma within the float32
logistic's rounding, and the sampled individuals' initial RMSE."""
import numpy as np
import pytest

import workloads as W
from gpu_util import RMSE_RTOL, f32_program, gpu_run
from oracle import trees as ot
from oracle.philox import PURPOSE_POP, PURPOSE_RT

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2106_04034_gb300 as pkg  # noqa: E402

W_PAPER = W.PAPER_K2047
SAMPLE = [0, 1, 777, 5120, 9000, 10239]


def test_paper_shape_k2047_sampled():
    w = W_PAPER
    run, data, p = gpu_run(w)
    X = np.ascontiguousarray(np.concatenate([data[0], data[2]]).T, dtype=np.float32)
    t = np.concatenate([data[1], data[3]]).astype(np.float64)
    eps = np.float32(p.protect_eps)
    F_tr, F_te = run.fitness()
    for pool, purpose in ((pkg.POOL_POPULATION, PURPOSE_POP), (pkg.POOL_RANDOM, PURPOSE_RT)):
        for i in SAMPLE:
            genes, consts = ot.linear_genome(w.seed, w.run, purpose, i, w.max_genes,
                                             w.n_features, w.const_lo, w.const_hi)
            S = run.semantics(pool, i, 1)[0]
            v = f32_program(genes, consts, X, eps)
            if pool == pkg.POOL_POPULATION:
                assert np.array_equal(S.view(np.uint32), v.view(np.uint32)) or \
                    np.array_equal(S, v, equal_nan=True), i
                d = v.astype(np.float64) - t
                rm_tr = np.sqrt(np.mean(d[:w.n_train] ** 2))
                if np.isfinite(rm_tr) and rm_tr < 1e15:
                    assert np.isclose(F_tr[i], rm_tr, rtol=RMSE_RTOL, atol=0), i
            else:
                with np.errstate(over="ignore"):
                    sg = (np.float32(1) / (np.float32(1) + np.exp(-v))).astype(np.float32)
                assert np.allclose(S, sg, rtol=0, atol=1e-6, equal_nan=True), i
    run.close()
