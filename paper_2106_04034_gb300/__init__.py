"""GB300-native Geometric Semantic GP (symbolic regression) hot path.

The compute runs in the sm_103a CUDA library libgsgp.so (C ABI in
include/gsgp.h); this package only builds and binds it.
"""
from .binding import (GENE_PAD, INIT_LINEAR, INIT_RHH, OP_ADD, OP_CONST, OP_DIV, OP_MUL, OP_SUB, OP_VAR,
                      PATH_AUTO, PATH_CHAINED, PATH_PERSISTENT,
                      POOL_POPULATION, POOL_RANDOM, SIGMA_BF16, SIGMA_F32, Batch, BatchInfo,
                      Config, GsgpError, Run, default_config, load_library, model_predict,
                      rng_words)

__all__ = ["Run", "Batch", "BatchInfo", "Config", "GsgpError", "default_config",
           "load_library", "model_predict", "rng_words",
           "OP_ADD", "OP_SUB", "OP_MUL", "OP_DIV", "OP_CONST", "OP_VAR", "GENE_PAD",
           "SIGMA_F32", "SIGMA_BF16", "INIT_RHH", "INIT_LINEAR", "POOL_POPULATION", "POOL_RANDOM",
           "PATH_AUTO", "PATH_PERSISTENT", "PATH_CHAINED"]
