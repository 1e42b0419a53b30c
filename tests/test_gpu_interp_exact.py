"""The interpreter's arithmetic, bit for bit.  Every operation of a program
is one IEEE float32 operation (protected division: 1 where |b| < eps), so a
float32 evaluation of the program as generated (skip rule and register Out
for linear genomes) gives the same bits case by case.  The GPU runs the
programs in another form (live code of genomes, "terminal, function" pairs
fused); this checks that the form changes no arithmetic."""
import numpy as np
import pytest

import workloads as W
from gpu_util import f32_program, gpu_run

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2106_04034_gb300 as pkg  # noqa: E402


CASES = {
    "trees": W.TINY,
    "deep trees": W.TINY.replace(name="deep trees", pop_size=96, n_random_trees=32,
                                 pop_min_depth=2, pop_max_depth=8, n_train=900, n_test=300),
    "genomes k127": W.TINY.replace(name="genomes", init_mode=1, max_genes=127),
    "genomes k1023": W.TINY.replace(name="long genomes", init_mode=1, max_genes=1023,
                                    pop_size=48, n_random_trees=16),
}


@pytest.mark.parametrize("case", list(CASES))
def test_population_semantics_bit_exact(case):
    w = CASES[case]
    run, data, p = gpu_run(w)
    X = np.ascontiguousarray(np.concatenate([data[0], data[2]]).T, dtype=np.float32)
    eps = np.float32(p.protect_eps)
    g, c, L = run.programs(pkg.POOL_POPULATION)
    S = run.semantics(pkg.POOL_POPULATION)
    for i in range(len(L)):
        want = f32_program(g[i, :L[i]], c[i, :L[i]], X, eps)
        assert np.array_equal(S[i].view(np.uint32), want.view(np.uint32)) or \
            np.array_equal(S[i], want, equal_nan=True), i
    run.close()


@pytest.mark.parametrize("case", ["deep trees", "genomes k127"])
def test_population_semantics_bit_exact_extreme_scales(case):
    """Cases whose features span every exponent (and subnormals): products
    and quotients overflow, underflow to subnormals and meet the protected
    division's threshold, with the same bits as a float32 evaluation."""
    w = CASES[case]
    Xtr, ytr, Xte, yte = W.make_data(w)
    rng = np.random.default_rng(20240611)

    def spread(X):
        k = rng.integers(-140, 128, size=X.shape)
        return (X.astype(np.float64) * np.exp2(k)).astype(np.float32)

    data = (spread(Xtr), ytr, spread(Xte), yte)
    assert np.all(np.isfinite(data[0])) and np.all(np.isfinite(data[2]))
    run, data, p = gpu_run(w, data=data)
    X = np.ascontiguousarray(np.concatenate([data[0], data[2]]).T, dtype=np.float32)
    eps = np.float32(p.protect_eps)
    g, c, L = run.programs(pkg.POOL_POPULATION)
    S = run.semantics(pkg.POOL_POPULATION)
    for i in range(len(L)):
        want = f32_program(g[i, :L[i]], c[i, :L[i]], X, eps)
        assert np.array_equal(S[i].view(np.uint32), want.view(np.uint32)) or \
            np.array_equal(S[i], want, equal_nan=True), i
    run.close()




@pytest.mark.parametrize("case", ["trees", "deep trees", "genomes k1023"])
def test_general_loop_bit_exact(case, monkeypatch):
    """The interpreter's general loop (stack pointer and skip rule, for
    programs that are not well-formed postfix, which the library does not
    generate) selected by its diagnostic switch: the same bits as a float32
    evaluation, for one chunk per thread (short trees) and two."""
    monkeypatch.setenv("GSGP_INTERP_GENERAL", "1")
    w = CASES[case]
    run, data, p = gpu_run(w)
    X = np.ascontiguousarray(np.concatenate([data[0], data[2]]).T, dtype=np.float32)
    eps = np.float32(p.protect_eps)
    g, c, L = run.programs(pkg.POOL_POPULATION)
    S = run.semantics(pkg.POOL_POPULATION)
    for i in range(len(L)):
        want = f32_program(g[i, :L[i]], c[i, :L[i]], X, eps)
        assert np.array_equal(S[i].view(np.uint32), want.view(np.uint32)) or \
            np.array_equal(S[i], want, equal_nan=True), i
    run.close()
