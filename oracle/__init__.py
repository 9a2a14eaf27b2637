"""Sequential CPU oracle for GSP-Louvain (arXiv 2402.11454).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  The product path (the
CUDA library and its binding) never imports this package, and this package
imports nothing from the product.

The arithmetic lives in ``oracle.c`` (plain C, FP64, one thread); this module
compiles it with gcc and marshals numpy arrays through ctypes.  Every
function cites the passage of the paper it follows; see ``oracle.c``.
"""
from .oracle import (  # noqa: F401
    build_oracle,
    Graph,
    vertex_weights,
    modularity,
    delta_modularity,
    move_sweep_sync,
    move,
    split_lp,
    split_bfs,
    renumber,
    lookup,
    aggregate,
    disconnected,
    louvain,
    louvain_trace,
    wave_hash,
    refine,
    refine_uniform,
    splitmix64,
    TRACE_FIELDS,
    LouvainOptions,
)
