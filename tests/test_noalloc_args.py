"""Host-side argument checks of the allocation-free mutation call
(binding.check_noalloc_args): every malformed tensor is refused with
E_INVALID before anything reaches the library.  The checks read only
dtype, shape, contiguity, device and address ranges, so they are exercised
here on CPU tensors with the CPU as the expected device."""
import pytest

torch = pytest.importorskip("torch")

from paper_2106_04034_gb300.binding import E_INVALID, GsgpError, check_noalloc_args  # noqa: E402

M, N_TRAIN, N_TEST, LD = 6, 40, 10, 52
CPU = torch.device("cpu")


def good():
    return dict(
        parents=torch.zeros((M, LD), dtype=torch.float32),
        sigma_r=torch.zeros((5, LD), dtype=torch.float32),
        target=torch.zeros(LD, dtype=torch.float32),
        n_train=N_TRAIN, n_test=N_TEST,
        parent=torch.zeros(M, dtype=torch.int32),
        rt1=torch.zeros(M, dtype=torch.int32),
        rt2=torch.zeros(M, dtype=torch.int32),
        ms=torch.zeros(M, dtype=torch.float32),
        offspring=torch.zeros((M, LD), dtype=torch.float32),
        rmse_train=torch.zeros(M, dtype=torch.float64),
        rmse_test=torch.zeros(M, dtype=torch.float64))


def check(a, device=CPU):
    return check_noalloc_args(a["parents"], a["sigma_r"], a["target"], a["n_train"],
                              a["n_test"], a["parent"], a["rt1"], a["rt2"], a["ms"],
                              a["offspring"], a["rmse_train"], a["rmse_test"], device)


def test_well_formed_arguments_pass():
    assert check(good()) == M


def _refused(a, words, device=CPU):
    with pytest.raises(GsgpError) as e:
        check(a, device)
    assert e.value.status == E_INVALID
    assert words in str(e.value)


BAD = {
    "parents float64": ("parents", lambda: torch.zeros((M, LD), dtype=torch.float64),
                        "parents must be a float32 matrix"),
    "parents 1-d": ("parents", lambda: torch.zeros(M * LD, dtype=torch.float32),
                    "parents must be a float32 matrix"),
    "parents too narrow": ("parents", lambda: torch.zeros((M, N_TRAIN), dtype=torch.float32),
                           "row stride"),
    "sigma_r other stride": ("sigma_r", lambda: torch.zeros((5, LD + 4), dtype=torch.float32),
                             "sigma_r must have"),
    "sigma_r bf16": ("sigma_r", lambda: torch.zeros((5, LD), dtype=torch.bfloat16),
                     "sigma_r must be a float32 matrix"),
    "target short": ("target", lambda: torch.zeros(LD - 1, dtype=torch.float32),
                     "target must be float32"),
    "target float64": ("target", lambda: torch.zeros(LD, dtype=torch.float64),
                       "target must be float32"),
    "parent int64": ("parent", lambda: torch.zeros(M, dtype=torch.int64),
                     "parent must be int32"),
    "rt1 short": ("rt1", lambda: torch.zeros(M - 1, dtype=torch.int32), "rt1 must be int32"),
    "rt2 float": ("rt2", lambda: torch.zeros(M, dtype=torch.float32), "rt2 must be int32"),
    "ms float64": ("ms", lambda: torch.zeros(M, dtype=torch.float64), "ms must be float32"),
    "ms long": ("ms", lambda: torch.zeros(M + 1, dtype=torch.float32), "ms must be float32"),
    "offspring too few rows": ("offspring", lambda: torch.zeros((1, LD), dtype=torch.float32),
                               "at least m"),
    "offspring other stride": ("offspring", lambda: torch.zeros((M, 4), dtype=torch.float32),
                               "offspring must have"),
    "rmse_train float32": ("rmse_train", lambda: torch.zeros(M, dtype=torch.float32),
                           "rmse_train must be float64"),
    "rmse_test short": ("rmse_test", lambda: torch.zeros(M - 1, dtype=torch.float64),
                        "rmse_test must be float64"),
    "offspring strided": ("offspring",
                          lambda: torch.zeros((LD, M), dtype=torch.float32).t(),
                          "offspring must be contiguous"),
    "parents not a tensor": ("parents", lambda: [[0.0] * LD] * M, "parents must be a torch"),
}


@pytest.mark.parametrize("case", sorted(BAD))
def test_each_malformed_argument_is_refused(case):
    name, make, words = BAD[case]
    a = good()
    a[name] = make()
    _refused(a, words)


def test_tensors_on_another_device_are_refused():
    _refused(good(), "expected meta", device=torch.device("meta"))


@pytest.mark.parametrize("other", ["parents", "sigma_r", "target"])
def test_offspring_may_not_overlap_its_inputs(other):
    a = good()
    if other == "target":
        a["offspring"] = torch.zeros((M + 1, LD), dtype=torch.float32)
        a["target"] = a["offspring"][M]          # the last offspring row
    elif other == "parents":
        a["offspring"] = a["parents"]            # in place
    else:
        big = torch.zeros((M + 5, LD), dtype=torch.float32)
        a["offspring"], a["sigma_r"] = big[:M], big[M - 1:M + 4]
    _refused(a, f"offspring overlaps {other}")
