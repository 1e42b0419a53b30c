"""The command-line front end on the GPU: its per-generation fitness files
equal the library's best-of-generation logs for the same configuration (one
run after another, and batched), and its model files reproduce the run's
predictions bit for bit, as does gsgp_model_predict on the model that
gsgp_best_trace returns."""
import subprocess

import numpy as np
import pytest

import workloads as W
from gpu_util import gpu_run

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2106_04034_gb300 as pkg  # noqa: E402
from paper_2106_04034_gb300.build import CLI, build_library  # noqa: E402

G = 15


def write_cases(path, X, y=None):
    rows = X if y is None else np.concatenate([X, y[:, None]], axis=1)
    np.savetxt(path, rows, fmt="%.9g")


@pytest.mark.parametrize("batched", [False, True], ids=["sequential", "batched"])
@pytest.mark.parametrize("linear", [False, True], ids=["trees", "genomes"])
def test_cli_matches_the_library(tmp_path, batched, linear):
    build_library()
    w = W.TINY.replace(pop_size=64, n_random_trees=50)
    if linear:
        w = w.replace(init_mode=1, max_genes=63)
    Xtr, ytr, Xte, yte = W.make_data(w)
    # the files hold the cases exactly (float32 printed with 9 digits)
    write_cases(tmp_path / "train.txt", Xtr, ytr)
    write_cases(tmp_path / "test.txt", Xte, yte)
    data = tuple(np.loadtxt(tmp_path / f, dtype=np.float64).astype(np.float32)
                 for f in ("train.txt", "test.txt"))
    data = (data[0][:, :-1], data[0][:, -1], data[1][:, :-1], data[1][:, -1])
    (tmp_path / "config.ini").write_text(
        "[run]\n"
        f"pop_size = {w.pop_size}\nn_random_trees = {w.n_random_trees}\n"
        f"pop_max_depth = {w.pop_max_depth}\nrt_max_depth = {w.rt_max_depth}\n"
        f"init_mode = {w.init_mode}\nmax_genes = {w.max_genes}\n"
        f"generations = {G}\nruns = 2\n")
    args = [CLI, "-train_file", str(tmp_path / "train.txt"), "-test_file",
            str(tmp_path / "test.txt"), "-config", str(tmp_path / "config.ini"), "-output_dir",
            str(tmp_path)]
    if batched:
        args.append("-batch")
    r = subprocess.run(args, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    ftr = np.loadtxt(tmp_path / "fitness_train.txt", ndmin=2)
    fte = np.loadtxt(tmp_path / "fitness_test.txt", ndmin=2)
    assert ftr.shape == (G, 2) and fte.shape == (G, 2)
    for k in range(2):
        run, _, p = gpu_run(w.replace(run=k), data=data)
        tr, te = run.evolve(G)
        assert np.array_equal(ftr[:, k], tr) and np.array_equal(fte[:, k], te)
        # the model file reproduces the run's predictions
        out = tmp_path / f"y{k}.txt"
        r = subprocess.run([CLI, "-model", str(tmp_path / f"model_run{k}.txt"), "-predict_file",
                            str(_features_file(tmp_path, data[2])), "-output", str(out)],
                           capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr
        want = run.predict(data[2])
        assert np.array_equal(np.loadtxt(out), want)
        # and so does gsgp_model_predict on the model gsgp_best_trace returns
        assert np.array_equal(pkg.model_predict(run.best_trace(), data[2]), want)
        run.close()


def _features_file(tmp_path, X):
    f = tmp_path / "features.txt"
    np.savetxt(f, X, fmt="%.9g")
    return f


def test_cli_fitness_files_against_the_oracle(tmp_path):
    """The tool's per-generation best training and test RMSE (the paper's
    two output series, Sec. 3.3) against the float64 oracle run from the
    same seed on the same case files, independently (programs, semantics,
    selection and survival all its own): the oracle's best-of-generation
    series must agree within the RMSE tolerance."""
    from oracle import gsgp as og
    from gpu_util import RMSE_RTOL, oracle_params
    build_library()
    w = W.TINY.replace(pop_size=64, n_random_trees=50)
    Xtr, ytr, Xte, yte = W.make_data(w)
    write_cases(tmp_path / "train.txt", Xtr, ytr)
    write_cases(tmp_path / "test.txt", Xte, yte)
    tr_rows = np.loadtxt(tmp_path / "train.txt", dtype=np.float64).astype(np.float32)
    te_rows = np.loadtxt(tmp_path / "test.txt", dtype=np.float64).astype(np.float32)
    (tmp_path / "config.ini").write_text(
        "[run]\n"
        f"pop_size = {w.pop_size}\nn_random_trees = {w.n_random_trees}\n"
        f"pop_max_depth = {w.pop_max_depth}\nrt_max_depth = {w.rt_max_depth}\n"
        f"generations = {G}\nruns = 2\n")
    r = subprocess.run([CLI, "-train_file", str(tmp_path / "train.txt"), "-test_file",
                        str(tmp_path / "test.txt"), "-config", str(tmp_path / "config.ini"),
                        "-output_dir", str(tmp_path)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    ftr = np.loadtxt(tmp_path / "fitness_train.txt", ndmin=2)
    fte = np.loadtxt(tmp_path / "fitness_test.txt", ndmin=2)
    for k in range(2):
        ref = og.GSGP(oracle_params(w.replace(run=k)), tr_rows[:, :-1], tr_rows[:, -1],
                      te_rows[:, :-1], te_rows[:, -1])
        ref.init()
        ref.evolve(G)
        assert np.allclose(ftr[:, k], ref.best_train, rtol=RMSE_RTOL, atol=0)
        assert np.allclose(fte[:, k], ref.best_test, rtol=RMSE_RTOL, atol=0)
