"""Host-side accounting of the benchmark, on CPU: the algorithmic bytes of a
generation (every distinct parent row and random-tree row read once, every
offspring row written once, the targets read once) from a hand-made trace,
and the whole-job throughput and peak helpers."""
import numpy as np

import bench
import workloads as W


class FakeRun:
    """Stands in for a run: only the trace (parent, rt1, rt2, ms) per
    generation and slot."""

    def __init__(self, par, r1, r2):
        self._t = (np.array(par, np.int32), np.array(r1, np.int32), np.array(r2, np.int32),
                   np.zeros(np.shape(par), np.float32))

    def trace(self):
        return self._t


def test_unique_bytes_mutation_elite_and_crossover():
    n = 1000
    w = W.TINY.replace(pop_size=4, n_train=800, n_test=200)
    assert w.n_cases == n
    run = FakeRun(
        par=[[0, 0, 1, 2],        # mutation: parents {0, 1, 2}, trees {0, 1, 2, 3}
             [1, 1, 1, 0],        # slot 3 is the elite copy (-1, -1): reads nothing
             [0, 2, 2, 2]],       # slot 0 a crossover of parents 0 and 3 with tree 1
        r1=[[0, 1, 1, 3],
            [2, 2, 0, -1],
            [1, 0, 0, 0]],
        r2=[[1, 1, 2, 0],
            [3, 3, 1, -1],
            [-2 - 3, 0, 0, 0]])
    for sig in (4, 2):
        got = bench.unique_bytes_per_generation(run, w, sig)
        want = [(3 + 4) * n * 4 + 4 * n * sig + n * 4,
                (1 + 4) * n * 4 + 4 * n * sig + n * 4,
                (3 + 4) * n * 4 + 2 * n * sig + n * 4]   # parents {0, 2, 3}, trees {0, 1}
        assert np.array_equal(got, np.array(want, np.float64)), (sig, got, want)


def test_job_value_and_single_rank_max():
    assert bench.job_value(3.0e9, 1, 2.0) == 1.5e9
    assert bench.job_value(3.0e9, 4, 2.0) == 6.0e9     # whole job: all ranks' units
    assert bench.max_over_ranks(1.25, 1) == 1.25


def test_peaks():
    gbs, kind = bench.measured_peak_gbs()
    assert kind in ("measured", "fallback") and gbs > 1000.0
    tops = bench.alu_peak_tops()
    assert 152 * 128 * 1.0e9 / 1e12 < tops < 152 * 128 * 3.0e9 / 1e12
