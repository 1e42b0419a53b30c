"""The C ABI library loads, exports every declared symbol, and its host-side
logic (configuration checks, state machine, argument checks) works without a
GPU.  No call here reaches the device."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2106_04034_gb300 as pkg
from paper_2106_04034_gb300 import binding as B
from paper_2106_04034_gb300.build import INCLUDE, build_library


@pytest.fixture(scope="module")
def lib():
    build_library()
    return pkg.load_library()


def declared_functions():
    names = []
    for h in sorted(os.listdir(INCLUDE)):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(INCLUDE, h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(gsgp_\w+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    # the binding wraps exactly the declared functions
    assert sorted(B.exported_names()) == names


def test_struct_layouts_match_the_header(lib, tmp_path):
    src = tmp_path / "layout.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "gsgp.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(gsgp_config), sizeof(gsgp_trace),
         sizeof(gsgp_info), offsetof(gsgp_config, stream), offsetof(gsgp_trace, coef),
         offsetof(gsgp_trace, sigma_dtype), offsetof(gsgp_info, device_bytes),
         sizeof(gsgp_batch_info), offsetof(gsgp_batch_info, updates_per_generation));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", INCLUDE, str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    want = [C.sizeof(B.Config), C.sizeof(B.Trace), C.sizeof(B.Info), B.Config.stream.offset,
            B.Trace.coef.offset, B.Trace.sigma_dtype.offset, B.Info.device_bytes.offset,
            C.sizeof(B.BatchInfo), B.BatchInfo.updates_per_generation.offset]
    assert got == want


def test_default_config(lib):
    cfg = pkg.default_config()
    assert cfg.struct_size == C.sizeof(B.Config)
    assert (cfg.pop_size, cfg.n_random_trees, cfg.tournament_size, cfg.elitism) == (1024, 1024, 4, 1)
    assert cfg.ms == np.float32(0.1) and cfg.protect_eps == np.float32(1e-3)
    assert cfg.p_feature_given_terminal == np.float32(0.14 / 0.18)
    assert lib.gsgp_config_error(C.byref(cfg)) == b""


@pytest.mark.parametrize("field,value", [
    ("pop_size", 1), ("pop_size", 65537), ("n_random_trees", 0), ("pop_min_depth", 7),
    ("rt_max_depth", 11), ("p_grow_function", 1.5), ("p_feature_given_terminal", -0.1),
    ("protect_eps", -1.0), ("ms_mode", 2), ("tournament_size", 65), ("elitism", 2),
    ("sigma_dtype", 3), ("const_lo", 5.0), ("struct_size", 8), ("ms", float("nan")),
])
def test_bad_configs_are_rejected(lib, field, value):
    cfg = pkg.default_config()
    setattr(cfg, field, value)
    ctx = C.c_void_p()
    assert lib.gsgp_create(C.byref(cfg), C.byref(ctx)) == B.E_INVALID
    assert not ctx.value
    assert lib.gsgp_config_error(C.byref(cfg)) != b""


def test_state_machine_without_device(lib):
    r = pkg.Run(pop_size=8, n_random_trees=4)
    assert r.info().state == 0
    for call in (r.init, lambda: r.evolve(3), r.best_trace, lambda: r.predict(np.zeros((2, 3))),
                 r.fitness):
        with pytest.raises(pkg.GsgpError) as e:
            call()
        assert e.value.status == B.E_STATE
    r.close()
    r.close()   # idempotent


# Non-finite values are checked on the device once the cases are copied
# there (tests/test_gpu_parity.py); shapes are checked on the host first.
@pytest.mark.parametrize("args", [
    dict(X=np.zeros((0, 3)), y=np.zeros(0)),                  # no training case
    dict(X=np.zeros((2, 0)), y=np.zeros(2)),                  # no feature
])
def test_bad_shapes_are_rejected_on_the_host(lib, args):
    r = pkg.Run(pop_size=8, n_random_trees=4)
    with pytest.raises(pkg.GsgpError) as e:
        r.load(args["X"], args["y"])
    assert e.value.status == B.E_INVALID
    assert r.info().state == 0
    r.close()


def test_null_arguments(lib):
    ctx = C.c_void_p()
    assert lib.gsgp_create(None, C.byref(ctx)) == B.E_INVALID
    cfg = pkg.default_config()
    assert lib.gsgp_create(C.byref(cfg), None) == B.E_INVALID
    assert lib.gsgp_init(None) == B.E_INVALID
    assert lib.gsgp_last_error(None) == b""
    lib.gsgp_destroy(None)
    assert lib.gsgp_rng_words(1, 0, 0, 0, -1, None, None) == B.E_INVALID
    r = pkg.Run(pop_size=8, n_random_trees=4)
    assert lib.gsgp_load(r.ctx, None, None, 4, 2, None, None, 0) == B.E_INVALID
    assert lib.gsgp_evolve(r.ctx, -1, None, None) in (B.E_STATE, B.E_INVALID)
    t = B.Trace()
    t.struct_size = 3
    assert lib.gsgp_best_trace(r.ctx, C.byref(t)) == B.E_INVALID
    r.close()


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    monkeypatch.setattr(B, "_lib", None)
    with pytest.raises(ImportError):
        B.load_library(str(tmp_path / "libgsgp.so"))


def test_batch_arguments_and_state_without_device(lib):
    """gsgp_batch_create checks its arguments and the runs' state on the host
    before any device call."""
    out = C.c_void_p()
    runs = [pkg.Run(pop_size=8, n_random_trees=4) for _ in range(2)]
    arr = (C.c_void_p * 2)(runs[0].ctx.value, runs[1].ctx.value)
    assert lib.gsgp_batch_create(arr, 2, None) == B.E_INVALID
    assert lib.gsgp_batch_create(None, 2, C.byref(out)) == B.E_INVALID
    assert lib.gsgp_batch_create(arr, 0, C.byref(out)) == B.E_INVALID
    assert lib.gsgp_batch_create(arr, 1025, C.byref(out)) == B.E_INVALID
    dup = (C.c_void_p * 2)(runs[0].ctx.value, runs[0].ctx.value)
    assert lib.gsgp_batch_create(dup, 2, C.byref(out)) == B.E_INVALID
    with_null = (C.c_void_p * 2)(runs[0].ctx.value, None)
    assert lib.gsgp_batch_create(with_null, 2, C.byref(out)) == B.E_INVALID
    # runs that are not initialised
    assert lib.gsgp_batch_create(arr, 2, C.byref(out)) == B.E_STATE
    assert not out.value
    with pytest.raises(pkg.GsgpError) as e:
        pkg.Batch(runs)
    assert e.value.status == B.E_STATE
    assert lib.gsgp_batch_evolve(None, 1, None, None) == B.E_INVALID
    assert lib.gsgp_batch_set_shape(None, 1, 1) == B.E_INVALID
    assert lib.gsgp_batch_get_info(None, None) == B.E_INVALID
    assert lib.gsgp_batch_last_error(None) == b""
    lib.gsgp_batch_destroy(None)
    for r in runs:
        r.close()


def test_linear_genome_config_checks(lib):
    cfg = pkg.default_config()
    assert (cfg.init_mode, cfg.max_genes) == (pkg.INIT_RHH, 127)
    for mode, k, ok in ((pkg.INIT_LINEAR, 127, True), (pkg.INIT_LINEAR, 4095, True),
                        (pkg.INIT_LINEAR, 0, False), (pkg.INIT_LINEAR, 4096, False),
                        (2, 127, False), (pkg.INIT_RHH, 0, True)):
        cfg = pkg.default_config(init_mode=mode, max_genes=k)
        assert (lib.gsgp_config_error(C.byref(cfg)) == b"") == ok, (mode, k)
    # depths are not checked for linear genomes' programs, but stay valid fields
    cfg = pkg.default_config(init_mode=pkg.INIT_LINEAR, max_genes=2047)
    r = pkg.Run(cfg)
    assert r.info().pop_max_genes == 2047 and r.info().rt_max_genes == 2047
    r.close()


def test_checkpoint_needs_a_run(lib):
    r = pkg.Run(pop_size=8, n_random_trees=4)
    n = C.c_size_t(0)
    assert lib.gsgp_checkpoint(r.ctx, None, 0, C.byref(n)) == B.E_STATE
    buf = C.create_string_buffer(64)
    assert lib.gsgp_restore(r.ctx, buf, 64) == B.E_STATE
    assert lib.gsgp_restore(None, buf, 64) == B.E_INVALID
    r.close()


def test_barrier_fault_hook_checks_its_arguments(lib):
    """The timeout test hook validates on the host and only arms the next
    persistent launch (no device work here)."""
    r = pkg.Run(pop_size=8, n_random_trees=4)
    assert lib.gsgp_arm_barrier_fault(None, 4096) == B.E_INVALID
    for bad in (0, 1023, (1 << 24) + 1):
        assert lib.gsgp_arm_barrier_fault(r.ctx, bad) == B.E_INVALID, bad
    assert lib.gsgp_arm_barrier_fault(r.ctx, 4096) == B.OK
    assert lib.gsgp_arm_barrier_fault(r.ctx, 1 << 24) == B.OK
    r.close()
