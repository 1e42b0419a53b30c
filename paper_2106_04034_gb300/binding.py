"""ctypes binding of libgsgp.so (argument marshalling only).

Every function of include/gsgp.h is exposed under the same name on ``lib``;
``Run`` wraps one context.  No step of the method runs in Python: arrays
are handed to the library as pointers (numpy arrays for host buffers, torch
CUDA tensors for device buffers), and a non-OK status raises GsgpError.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libgsgp.so")

STATUS = {0: "GSGP_OK", 1: "GSGP_E_INVALID", 2: "GSGP_E_STATE", 3: "GSGP_E_OOM",
          4: "GSGP_E_CUDA", 5: "GSGP_E_TIMEOUT", 6: "GSGP_E_NUMERIC"}
OK, E_INVALID, E_STATE, E_OOM, E_CUDA, E_TIMEOUT, E_NUMERIC = range(7)
OP_ADD, OP_SUB, OP_MUL, OP_DIV, OP_CONST, OP_VAR, GENE_PAD = 0, 1, 2, 3, 4, 5, -1
SIGMA_F32, SIGMA_BF16 = 0, 1
INIT_RHH, INIT_LINEAR = 0, 1
POOL_POPULATION, POOL_RANDOM = 0, 1
PATH_AUTO, PATH_PERSISTENT, PATH_CHAINED = 0, 1, 2

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class GsgpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Config(C.Structure):
    _fields_ = [
        ("struct_size", C.c_uint32), ("seed", C.c_uint64), ("run", C.c_uint32),
        ("pop_size", C.c_int32), ("n_random_trees", C.c_int32),
        ("pop_min_depth", C.c_int32), ("pop_max_depth", C.c_int32),
        ("rt_min_depth", C.c_int32), ("rt_max_depth", C.c_int32),
        ("const_lo", C.c_float), ("const_hi", C.c_float),
        ("p_grow_function", C.c_float), ("p_feature_given_terminal", C.c_float),
        ("protect_eps", C.c_float), ("ms", C.c_float), ("ms_mode", C.c_int32),
        ("tournament_size", C.c_int32), ("elitism", C.c_int32), ("sigma_dtype", C.c_int32),
        ("init_mode", C.c_int32), ("max_genes", C.c_int32), ("p_crossover", C.c_float),
        ("stream", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN),
        ("alloc_user", C.c_void_p),
    ]


class Trace(C.Structure):
    _fields_ = [
        ("struct_size", C.c_uint32), ("best_slot", C.c_int32),
        ("best_train_rmse", C.c_double), ("best_test_rmse", C.c_double),
        ("ancestor", C.c_int32), ("ancestor_length", C.c_int32), ("max_genes", C.c_int32),
        ("ancestor_genes", C.POINTER(C.c_int32)), ("ancestor_consts", C.POINTER(C.c_float)),
        ("n_generations", C.c_int32),
        ("lineage_parent", C.POINTER(C.c_int32)), ("lineage_rt1", C.POINTER(C.c_int32)),
        ("lineage_rt2", C.POINTER(C.c_int32)), ("lineage_ms", C.POINTER(C.c_float)),
        ("n_random_trees", C.c_int32), ("coef", C.POINTER(C.c_double)),
        ("rt_max_genes", C.c_int32), ("rt_genes", C.POINTER(C.c_int32)),
        ("rt_consts", C.POINTER(C.c_float)), ("rt_lengths", C.POINTER(C.c_int32)),
        ("sigma_dtype", C.c_int32), ("n_features", C.c_int32), ("protect_eps", C.c_float),
        ("init_mode", C.c_int32),
    ]


class Info(C.Structure):
    _fields_ = [
        ("struct_size", C.c_uint32), ("state", C.c_int32), ("n_features", C.c_int32),
        ("n_train", C.c_int64), ("n_test", C.c_int64), ("n_cases", C.c_int64),
        ("n_cases_padded", C.c_int64), ("pop_size", C.c_int32), ("n_random_trees", C.c_int32),
        ("pop_max_genes", C.c_int32), ("rt_max_genes", C.c_int32), ("generation", C.c_int32),
        ("evolve_tile_cases", C.c_int32), ("evolve_offspring_per_cta", C.c_int32),
        ("evolve_path", C.c_int32), ("evolve_grid", C.c_int32),
        ("evolve_generations_per_launch", C.c_int32),
        ("kernel_launches", C.c_int64), ("device_bytes", C.c_int64),
        ("pop_evaluated_genes", C.c_int64), ("rt_evaluated_genes", C.c_int64),
    ]


class BatchInfo(C.Structure):
    _fields_ = [
        ("struct_size", C.c_uint32), ("runs", C.c_int32), ("tile_cases", C.c_int32),
        ("offspring_per_cta", C.c_int32), ("grid", C.c_int32),
        ("generations_per_launch", C.c_int32), ("graph", C.c_int32),
        ("offspring", C.c_int64), ("updates_per_generation", C.c_int64),
        ("items_per_generation", C.c_int64), ("kernel_launches", C.c_int64),
    ]


P = C.c_void_p
_SIGS = {
    "gsgp_config_default": (None, [C.POINTER(Config)]),
    "gsgp_config_error": (C.c_char_p, [C.POINTER(Config)]),
    "gsgp_create": (C.c_int, [C.POINTER(Config), C.POINTER(P)]),
    "gsgp_load": (C.c_int, [P, P, P, C.c_int64, C.c_int32, P, P, C.c_int64]),
    "gsgp_load_device": (C.c_int, [P, P, P, C.c_int64, C.c_int32, P, P, C.c_int64]),
    "gsgp_init": (C.c_int, [P]),
    "gsgp_evolve": (C.c_int, [P, C.c_int32, P, P]),
    "gsgp_best_trace": (C.c_int, [P, C.POINTER(Trace)]),
    "gsgp_predict": (C.c_int, [P, P, C.c_int64, P]),
    "gsgp_predict_device": (C.c_int, [P, P, C.c_int64, P]),
    "gsgp_last_error": (C.c_char_p, [P]),
    "gsgp_destroy": (None, [P]),
    "gsgp_get_info": (C.c_int, [P, C.POINTER(Info)]),
    "gsgp_get_programs": (C.c_int, [P, C.c_int32, P, P, P]),
    "gsgp_get_semantics": (C.c_int, [P, C.c_int32, C.c_int32, C.c_int32, P]),
    "gsgp_get_fitness": (C.c_int, [P, P, P]),
    "gsgp_get_trace": (C.c_int, [P, C.c_int32, C.c_int32, P, P, P, P]),
    "gsgp_set_evolve_shape": (C.c_int, [P, C.c_int32, C.c_int32, C.c_int32]),
    "gsgp_arm_barrier_fault": (C.c_int, [P, C.c_uint32]),
    "gsgp_shard_configure": (C.c_int, [P, C.c_int64, C.c_int64, C.c_int64]),
    "gsgp_shard_partials": (C.c_int, [P, C.POINTER(C.c_void_p), C.POINTER(C.c_int64),
                                      C.POINTER(C.c_int64)]),
    "gsgp_shard_generation": (C.c_int, [P]),
    "gsgp_shard_finish": (C.c_int, [P]),
    "gsgp_set_kernel_timing": (C.c_int, [P, C.c_int32]),
    "gsgp_kernel_times": (C.c_int, [P, P, C.c_int32, P]),
    "gsgp_init_kernel_times": (C.c_int, [P, P]),
    "gsgp_rng_words": (C.c_int, [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int32, P, P]),
    "gsgp_mutate_noalloc": (C.c_int, [P, P, C.c_int64, P, C.c_int64, C.c_int64, P, P, P, P,
                                      C.c_int32, P, P, P, P, C.c_char_p, C.c_size_t]),
    "gsgp_checkpoint": (C.c_int, [P, P, C.c_size_t, C.POINTER(C.c_size_t)]),
    "gsgp_restore": (C.c_int, [P, P, C.c_size_t]),
    "gsgp_model_predict": (C.c_int, [C.POINTER(Trace), P, C.c_int64, P, P, C.c_char_p,
                                     C.c_size_t]),
    "gsgp_batch_create": (C.c_int, [P, C.c_int32, C.POINTER(P)]),
    "gsgp_batch_evolve": (C.c_int, [P, C.c_int32, P, P]),
    "gsgp_batch_set_shape": (C.c_int, [P, C.c_int32, C.c_int32]),
    "gsgp_batch_set_kernel_timing": (C.c_int, [P, C.c_int32]),
    "gsgp_batch_kernel_times": (C.c_int, [P, P, C.c_int32, P]),
    "gsgp_batch_get_info": (C.c_int, [P, C.POINTER(BatchInfo)]),
    "gsgp_batch_last_error": (C.c_char_p, [P]),
    "gsgp_batch_destroy": (None, [P]),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libgsgp.so (raises when it has not been built: there is no
    fallback implementation)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libgsgp.so is not built ({path}); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_names():
    return list(_SIGS)


def _ptr(a) -> Optional[int]:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    if hasattr(a, "data_ptr"):        # torch tensor
        assert a.is_contiguous()
        return a.data_ptr()
    return int(a)


def default_config(**kw) -> Config:
    lib = load_library()
    cfg = Config()
    lib.gsgp_config_default(C.byref(cfg))
    for k, v in kw.items():
        if not hasattr(cfg, k):
            raise TypeError(f"unknown config field {k}")
        setattr(cfg, k, v)
    return cfg


class TorchAllocator:
    """Device allocator hooks backed by torch's caching allocator."""

    def __init__(self, device: int = 0):
        import torch
        self.torch = torch
        self.device = device

        def _alloc(user, nbytes, stream):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), self.device,
                                                              stream if stream else 0))
            except Exception:
                return None

        def _free(user, ptr, stream):
            if ptr:
                torch.cuda.caching_allocator_delete(ptr)

        self.alloc_fn = ALLOC_FN(_alloc)
        self.free_fn = FREE_FN(_free)


class _DeviceArray:
    """A device buffer owned by the library, described by the CUDA array
    interface so that torch can view it without a copy."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(int(s) for s in shape),
                                         "typestr": typestr, "data": (int(ptr), False),
                                         "version": 2}


class Run:
    """One GSGP run (one gsgp_ctx)."""

    def __init__(self, cfg: Optional[Config] = None, stream=None, torch_allocator=False, **kw):
        self.lib = load_library()
        self.cfg = cfg if cfg is not None else default_config(**kw)
        if stream is not None:
            self.cfg.stream = stream if isinstance(stream, int) else stream.cuda_stream
        self._allocator = None
        if torch_allocator:
            self._allocator = TorchAllocator()
            self.cfg.alloc = self._allocator.alloc_fn
            self.cfg.free = self._allocator.free_fn
        self.ctx = P()
        st = self.lib.gsgp_create(C.byref(self.cfg), C.byref(self.ctx))
        if st != OK:
            raise GsgpError(st, self.lib.gsgp_config_error(C.byref(self.cfg)).decode())

    def _check(self, st):
        if st != OK:
            raise GsgpError(st, self.lib.gsgp_last_error(self.ctx).decode())

    def close(self):
        if self.ctx:
            self.lib.gsgp_destroy(self.ctx)
            self.ctx = P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- data -------------------------------------------------------------
    def load(self, X_train, y_train, X_test=None, y_test=None):
        X_train = np.ascontiguousarray(X_train, dtype=np.float32)
        y_train = np.ascontiguousarray(y_train, dtype=np.float32)
        n_te = 0 if X_test is None else len(X_test)
        if n_te:
            X_test = np.ascontiguousarray(X_test, dtype=np.float32)
            y_test = np.ascontiguousarray(y_test, dtype=np.float32)
        self._check(self.lib.gsgp_load(self.ctx, _ptr(X_train), _ptr(y_train), len(X_train),
                                       X_train.shape[1] if X_train.ndim == 2 else 0,
                                       _ptr(X_test) if n_te else None,
                                       _ptr(y_test) if n_te else None, n_te))

    def load_device(self, X_train, y_train, X_test=None, y_test=None):
        """torch CUDA float32 tensors, row-major (cases x features)."""
        n_te = 0 if X_test is None else int(X_test.shape[0])
        self._check(self.lib.gsgp_load_device(
            self.ctx, _ptr(X_train), _ptr(y_train), int(X_train.shape[0]), int(X_train.shape[1]),
            _ptr(X_test) if n_te else None, _ptr(y_test) if n_te else None, n_te))

    def init(self):
        self._check(self.lib.gsgp_init(self.ctx))

    def evolve(self, generations: int, log: bool = True):
        if not log:
            self._check(self.lib.gsgp_evolve(self.ctx, generations, None, None))
            return None
        tr = np.zeros(generations, dtype=np.float64)
        te = np.zeros(generations, dtype=np.float64)
        self._check(self.lib.gsgp_evolve(self.ctx, generations, _ptr(tr), _ptr(te)))
        return tr, te

    # -- best individual ---------------------------------------------------
    def best_trace(self) -> dict:
        t = Trace()
        t.struct_size = C.sizeof(Trace)
        self._check(self.lib.gsgp_best_trace(self.ctx, C.byref(t)))
        G, r, K, Kr = t.n_generations, t.n_random_trees, t.max_genes, t.rt_max_genes
        out = {
            "anc_genes": np.zeros(K, np.int32), "anc_consts": np.zeros(K, np.float32),
            "parent": np.zeros(max(G, 1), np.int32), "rt1": np.zeros(max(G, 1), np.int32),
            "rt2": np.zeros(max(G, 1), np.int32), "ms": np.zeros(max(G, 1), np.float32),
            "coef": np.zeros(r, np.float64), "rt_genes": np.zeros((r, Kr), np.int32),
            "rt_consts": np.zeros((r, Kr), np.float32), "rt_lengths": np.zeros(r, np.int32),
        }

        def p(a, ct):
            return a.ctypes.data_as(C.POINTER(ct))

        t.ancestor_genes = p(out["anc_genes"], C.c_int32)
        t.ancestor_consts = p(out["anc_consts"], C.c_float)
        t.lineage_parent = p(out["parent"], C.c_int32)
        t.lineage_rt1 = p(out["rt1"], C.c_int32)
        t.lineage_rt2 = p(out["rt2"], C.c_int32)
        t.lineage_ms = p(out["ms"], C.c_float)
        t.coef = p(out["coef"], C.c_double)
        t.rt_genes = p(out["rt_genes"], C.c_int32)
        t.rt_consts = p(out["rt_consts"], C.c_float)
        t.rt_lengths = p(out["rt_lengths"], C.c_int32)
        self._check(self.lib.gsgp_best_trace(self.ctx, C.byref(t)))
        for k in ("parent", "rt1", "rt2", "ms"):
            out[k] = out[k][:G]
        out.update(best_slot=t.best_slot, best_train_rmse=t.best_train_rmse,
                   best_test_rmse=t.best_test_rmse, ancestor=t.ancestor,
                   ancestor_length=t.ancestor_length, n_generations=G,
                   sigma_dtype=t.sigma_dtype, n_features=t.n_features,
                   protect_eps=t.protect_eps, init_mode=t.init_mode)
        return out

    def predict(self, X) -> np.ndarray:
        X = np.ascontiguousarray(X, dtype=np.float32)
        y = np.zeros(len(X), dtype=np.float64)
        self._check(self.lib.gsgp_predict(self.ctx, _ptr(X), len(X), _ptr(y)))
        return y

    def predict_device(self, X, y):
        self._check(self.lib.gsgp_predict_device(self.ctx, _ptr(X), int(X.shape[0]), _ptr(y)))

    # -- introspection -----------------------------------------------------
    def info(self) -> Info:
        i = Info()
        i.struct_size = C.sizeof(Info)
        self._check(self.lib.gsgp_get_info(self.ctx, C.byref(i)))
        return i

    def programs(self, pool: int):
        i = self.info()
        cnt = i.pop_size if pool == POOL_POPULATION else i.n_random_trees
        K = i.pop_max_genes if pool == POOL_POPULATION else i.rt_max_genes
        g = np.zeros((cnt, K), np.int32)
        c = np.zeros((cnt, K), np.float32)
        L = np.zeros(cnt, np.int32)
        self._check(self.lib.gsgp_get_programs(self.ctx, pool, _ptr(g), _ptr(c), _ptr(L)))
        return g, c, L

    def semantics(self, pool: int, row0: int = 0, rows: Optional[int] = None) -> np.ndarray:
        i = self.info()
        cnt = i.pop_size if pool == POOL_POPULATION else i.n_random_trees
        rows = cnt - row0 if rows is None else rows
        out = np.zeros((rows, i.n_cases), np.float32)
        self._check(self.lib.gsgp_get_semantics(self.ctx, pool, row0, rows, _ptr(out)))
        return out

    def fitness(self):
        m = self.info().pop_size
        tr = np.zeros(m, np.float64)
        te = np.zeros(m, np.float64)
        self._check(self.lib.gsgp_get_fitness(self.ctx, _ptr(tr), _ptr(te)))
        return tr, te

    def trace(self, g0: int = 0, count: Optional[int] = None):
        i = self.info()
        count = i.generation - g0 if count is None else count
        m = i.pop_size
        a = [np.zeros((count, m), np.int32) for _ in range(3)]
        ms = np.zeros((count, m), np.float32)
        self._check(self.lib.gsgp_get_trace(self.ctx, g0, count, _ptr(a[0]), _ptr(a[1]),
                                            _ptr(a[2]), _ptr(ms)))
        return a[0], a[1], a[2], ms

    def checkpoint(self) -> bytes:
        """gsgp_checkpoint: the run's state as bytes."""
        n = C.c_size_t(0)
        self._check(self.lib.gsgp_checkpoint(self.ctx, None, 0, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self._check(self.lib.gsgp_checkpoint(self.ctx, buf, n.value, C.byref(n)))
        return buf.raw[:n.value]

    def restore(self, data: bytes):
        """gsgp_restore: resume from checkpoint bytes (same config and data loaded)."""
        buf = C.create_string_buffer(data, len(data))
        self._check(self.lib.gsgp_restore(self.ctx, buf, len(data)))

    def set_evolve_shape(self, path: int, vec: int = 0, opb: int = 0):
        self._check(self.lib.gsgp_set_evolve_shape(self.ctx, path, vec, opb))

    # -- case sharding (gsgp_shard_*) ----------------------------------------
    def shard_configure(self, case0: int, n_train_all: int, n_test_all: int):
        """Make this (not yet loaded) run the shard holding the problem's
        cases from case0 on; load() then gets exactly that slice."""
        self._check(self.lib.gsgp_shard_configure(self.ctx, case0, n_train_all, n_test_all))

    def shard_partials(self):
        """The pending exchange's partial sums as a torch CUDA float64 tensor
        of shape (pop_size, chunks, 2) viewing the library's device array
        (valid until the next init)."""
        import torch
        ptr, rows, chunks = C.c_void_p(), C.c_int64(), C.c_int64()
        self._check(self.lib.gsgp_shard_partials(self.ctx, C.byref(ptr), C.byref(rows),
                                                 C.byref(chunks)))
        return torch.as_tensor(_DeviceArray(ptr.value, (rows.value, chunks.value, 2), "<f8"),
                               device="cuda")

    def shard_generation(self):
        self._check(self.lib.gsgp_shard_generation(self.ctx))

    def shard_finish(self):
        self._check(self.lib.gsgp_shard_finish(self.ctx))

    def arm_barrier_fault(self, spin_limit: int):
        """Test hook of the timeout path (gsgp_arm_barrier_fault)."""
        self._check(self.lib.gsgp_arm_barrier_fault(self.ctx, spin_limit))

    def set_kernel_timing(self, enabled: bool):
        self._check(self.lib.gsgp_set_kernel_timing(self.ctx, int(enabled)))

    def kernel_times(self, cap: int = 1 << 16) -> np.ndarray:
        out = np.zeros(cap, np.float32)
        n = C.c_int32(0)
        self._check(self.lib.gsgp_kernel_times(self.ctx, _ptr(out), cap, C.byref(n)))
        return out[:n.value].copy()

    def init_kernel_times(self) -> np.ndarray:
        """ms of the last init's two interpreter launches (population, random trees)."""
        out = np.zeros(2, np.float32)
        self._check(self.lib.gsgp_init_kernel_times(self.ctx, _ptr(out)))
        return out


class Batch:
    """Independent runs evolved together (one gsgp_batch).  The runs must
    be initialised and must outlive the batch; they stay usable as Run
    objects (best_trace, predict, semantics, ...)."""

    def __init__(self, runs):
        self.lib = load_library()
        self.runs = list(runs)
        arr = (P * len(self.runs))(*[r.ctx.value for r in self.runs])
        self.handle = P()
        st = self.lib.gsgp_batch_create(arr, len(self.runs), C.byref(self.handle))
        if st != OK:
            raise GsgpError(st, "gsgp_batch_create failed")

    def _check(self, st):
        if st != OK:
            raise GsgpError(st, self.lib.gsgp_batch_last_error(self.handle).decode())

    def close(self):
        if self.handle:
            self.lib.gsgp_batch_destroy(self.handle)
            self.handle = P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def evolve(self, generations: int, log: bool = True):
        """Advance every run; with log, (train, test) arrays of shape
        (runs, generations) of the best RMSE per generation."""
        if not log:
            self._check(self.lib.gsgp_batch_evolve(self.handle, generations, None, None))
            return None
        tr = np.zeros((len(self.runs), generations), dtype=np.float64)
        te = np.zeros((len(self.runs), generations), dtype=np.float64)
        self._check(self.lib.gsgp_batch_evolve(self.handle, generations, _ptr(tr), _ptr(te)))
        return tr, te

    def set_shape(self, vec: int = 0, opb: int = 0):
        self._check(self.lib.gsgp_batch_set_shape(self.handle, vec, opb))

    def set_kernel_timing(self, enabled: bool):
        self._check(self.lib.gsgp_batch_set_kernel_timing(self.handle, int(enabled)))

    def kernel_times(self, cap: int = 1 << 16) -> np.ndarray:
        out = np.zeros(cap, np.float32)
        n = C.c_int32(0)
        self._check(self.lib.gsgp_batch_kernel_times(self.handle, _ptr(out), cap, C.byref(n)))
        return out[:n.value].copy()

    def info(self) -> BatchInfo:
        i = BatchInfo()
        i.struct_size = C.sizeof(BatchInfo)
        self._check(self.lib.gsgp_batch_get_info(self.handle, C.byref(i)))
        return i


def model_predict(model: dict, X, stream=None) -> np.ndarray:
    """gsgp_model_predict: evaluate a model (the dict Run.best_trace returns)
    on HOST cases X (n x n_features), with no run context."""
    lib = load_library()
    X = np.ascontiguousarray(X, dtype=np.float32)
    n = X.shape[0]
    keep = {k: np.ascontiguousarray(model[k]) for k in
            ("anc_genes", "anc_consts", "coef", "rt_genes", "rt_consts", "rt_lengths")}
    t = Trace()
    t.struct_size = C.sizeof(Trace)
    t.ancestor_length = int(model["ancestor_length"])
    t.max_genes = int(keep["anc_genes"].shape[0])
    t.ancestor_genes = keep["anc_genes"].ctypes.data_as(C.POINTER(C.c_int32))
    t.ancestor_consts = keep["anc_consts"].ctypes.data_as(C.POINTER(C.c_float))
    t.n_random_trees = int(keep["coef"].shape[0])
    t.coef = keep["coef"].ctypes.data_as(C.POINTER(C.c_double))
    t.rt_max_genes = int(keep["rt_genes"].shape[1])
    t.rt_genes = keep["rt_genes"].ctypes.data_as(C.POINTER(C.c_int32))
    t.rt_consts = keep["rt_consts"].ctypes.data_as(C.POINTER(C.c_float))
    t.rt_lengths = keep["rt_lengths"].ctypes.data_as(C.POINTER(C.c_int32))
    t.sigma_dtype = int(model["sigma_dtype"])
    t.n_features = int(model["n_features"])
    t.protect_eps = float(model["protect_eps"])
    t.init_mode = int(model["init_mode"])
    y = np.zeros(n, np.float64)
    msg = C.create_string_buffer(256)
    s = None if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    st = lib.gsgp_model_predict(C.byref(t), _ptr(X), n, _ptr(y), s, msg, 256)
    if st != OK:
        raise GsgpError(st, msg.value.decode())
    return y


def rng_words(seed: int, run: int, gen_or_purpose: int, individual: int, n_words: int,
              stream=None) -> np.ndarray:
    lib = load_library()
    out = np.zeros(n_words, np.uint32)
    st = lib.gsgp_rng_words(seed, run, gen_or_purpose, individual, n_words, _ptr(out),
                            stream.cuda_stream if stream is not None and not isinstance(stream, int)
                            else stream)
    if st != OK:
        raise GsgpError(st, "gsgp_rng_words failed")
    return out


def check_noalloc_args(parents, sigma_r, target, n_train, n_test, parent, rt1, rt2, ms,
                       offspring, rmse_train, rmse_test, device) -> int:
    """Validate the tensors of gsgp_mutate_noalloc before any launch: every
    tensor on ``device`` and contiguous; parents / sigma_r / offspring float32
    matrices with the common row stride ld = parents.shape[1] >= n_train +
    n_test; offspring with at least m rows and not the same memory as parents,
    sigma_r or target (the call reads those while it writes offspring);
    target float32 with at least ld elements; parent / rt1 / rt2 int32 and ms
    float32 with m = parent.numel() elements each; rmse outputs float64 with
    at least m elements.  The library itself checks sizes, alignment and the
    scratch limit but cannot see dtypes or buffer extents.  Returns m; raises
    GsgpError(E_INVALID) on the first violation."""
    import torch

    def bad(text):
        raise GsgpError(E_INVALID, f"mutate_noalloc: {text}")

    named = (("parents", parents), ("sigma_r", sigma_r), ("target", target), ("parent", parent),
             ("rt1", rt1), ("rt2", rt2), ("ms", ms), ("offspring", offspring),
             ("rmse_train", rmse_train), ("rmse_test", rmse_test))
    for name, t in named:
        if not isinstance(t, torch.Tensor):
            bad(f"{name} must be a torch tensor")
        if t.device != device:
            bad(f"{name} is on {t.device}, expected {device}")
        if not t.is_contiguous():
            bad(f"{name} must be contiguous")
    for name, t in (("parents", parents), ("sigma_r", sigma_r), ("offspring", offspring)):
        if t.dtype != torch.float32 or t.dim() != 2:
            bad(f"{name} must be a float32 matrix")
    ld = int(parents.shape[1])
    if ld < int(n_train) + int(n_test):
        bad("the row stride parents.shape[1] is below n_train + n_test")
    for name, t in (("sigma_r", sigma_r), ("offspring", offspring)):
        if int(t.shape[1]) != ld:
            bad(f"{name} must have parents.shape[1] = {ld} columns")
    if target.dtype != torch.float32 or target.numel() < ld:
        bad(f"target must be float32 with at least {ld} elements")
    m = int(parent.numel())
    for name, t in (("parent", parent), ("rt1", rt1), ("rt2", rt2)):
        if t.dtype != torch.int32 or t.numel() != m:
            bad(f"{name} must be int32 with m = {m} elements")
    if ms.dtype != torch.float32 or ms.numel() != m:
        bad(f"ms must be float32 with m = {m} elements")
    if int(offspring.shape[0]) < m:
        bad(f"offspring must have at least m = {m} rows")
    for name, t in (("rmse_train", rmse_train), ("rmse_test", rmse_test)):
        if t.dtype != torch.float64 or t.numel() < m:
            bad(f"{name} must be float64 with at least m = {m} elements")
    o0 = offspring.data_ptr()
    o1 = o0 + offspring.numel() * 4
    for name, t in (("parents", parents), ("sigma_r", sigma_r), ("target", target)):
        a0 = t.data_ptr()
        a1 = a0 + t.numel() * t.element_size()
        if a0 < o1 and o0 < a1:
            bad(f"offspring overlaps {name}")
    return m


def mutate_noalloc(parents, sigma_r, target, n_train, n_test, parent, rt1, rt2, ms, offspring,
                   rmse_train, rmse_test, stream=None):
    """gsgp_mutate_noalloc on torch CUDA tensors (row-major, common row
    stride = parents.shape[1]); queued on `stream` (default: torch's current
    stream).  The tensors are validated first (check_noalloc_args); raises
    GsgpError with the library's message on failure."""
    import torch
    lib = load_library()
    device = torch.device("cuda", torch.cuda.current_device())
    m = check_noalloc_args(parents, sigma_r, target, n_train, n_test, parent, rt1, rt2, ms,
                           offspring, rmse_train, rmse_test, device)
    if stream is None:
        stream = torch.cuda.current_stream()
    s = stream if isinstance(stream, int) else stream.cuda_stream
    msg = C.create_string_buffer(256)
    st = lib.gsgp_mutate_noalloc(_ptr(parents), _ptr(sigma_r), int(parents.shape[1]),
                                 _ptr(target), n_train, n_test, _ptr(parent), _ptr(rt1),
                                 _ptr(rt2), _ptr(ms), m, _ptr(offspring),
                                 _ptr(rmse_train), _ptr(rmse_test), s, msg, 256)
    if st != OK:
        raise GsgpError(st, msg.value.decode())
