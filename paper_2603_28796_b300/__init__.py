"""GaloisSAT's differentiable solving stage (arXiv 2603.28796) as a B300-native library.

The compute path is ``libgaloissat.so`` (C ABI in ``include/gs.h``, sm_103a kernels); this
package holds its Python binding (``_abi``, same function names as the C entry points), the
training engine built on it (``engine``: autograd.Function, fused Adam step, CUDA-graph loop),
candidate sharding over ranks (``shard``), the seeded input generators (``synth``) and the
in-tree build (``build``).

Names of the binding are resolved on first use, so that importing the package (e.g. for the
input generators) does not load the CUDA library.
"""
import importlib

__version__ = "0.1.0"

_ABI_NAMES = (
    "GS_BF16", "GS_F16", "GS_F32", "GSError", "Problem", "gs_adam_default", "gs_backward", "gs_check_bits",
    "gs_forward", "gs_free", "gs_info_get", "gs_inspect_cnf", "gs_last_error", "gs_load_batch", "gs_load_cnf",
    "gs_load_dimacs", "gs_relax", "gs_reserve", "gs_set_tuning", "gs_get_tuning", "gs_autotune", "gs_forward_noalloc", "gs_round_check", "gs_status_str", "gs_step", "gs_sync_status", "gs_wait_selftest", "gs_st_noise",
    "gs_st_sample", "gs_st_step", "gs_tseitin3", "gs_pool_sample",
    "gs_branch_vars",
)


def __getattr__(name):
    if name in _ABI_NAMES:
        return getattr(importlib.import_module("._abi", __name__), name)
    raise AttributeError(name)
