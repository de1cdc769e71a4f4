"""GB300 (sm_103a) screened ACE exchange build: C-ABI CUDA library and its Python binding.

The compute path is libace_gb300.so (csrc/, declared in include/ace.h); ``ace`` is a ctypes
binding with the same entry-point names, and ``build`` compiles the library with nvcc.
"""

from . import ace  # noqa: F401
from .ace import (  # noqa: F401
    ACE_COULOMB_PERIODIC,
    ACE_COULOMB_TRUNCATED,
    ACE_FP64,
    ACE_MIXED,
    AceDesc,
    AceError,
    AceGraph,
    AceOp,
    ace_apply,
    ace_build,
    ace_build_batched,
    ace_build_pairs,
    ace_destroy,
    ace_get,
    ace_graph_create,
    ace_grid_supported,
    ace_last_error,
    ace_pair_count,
    ace_scdm,
    ace_stage_times,
    exchange_energy,
    make_desc,
)
