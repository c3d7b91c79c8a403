"""GB300-native sparse-matrix fixpoint of logic programs (liblp + Python binding).

The compute path is liblp.so (CUDA for sm_103a, C ABI in include/lp.h); this package only
loads it and marshals arguments. Nothing here falls back to a CPU implementation.
"""
from .lp import (ERR_INVALID, ERR_NO_FIXPOINT, EXPORTS, LP_COMPILE_HOST_ONLY, LP_COMPILE_ON_DEVICE,  # noqa: F401
                 LP_COMPILE_ON_HOST, LP_ROWS, LP_TIMING, LP_TUNE_LEAST, LP_TUNE_STABLE, Batch, LPError, Program,
                 check_grid_barrier, debug_fail_alloc, launch_count, least_model_static,
                 library_path, load, words)


def build(force: bool = False) -> str:
    from . import _build
    return _build.build(force=force)
