"""ctypes declarations of libgsp.so (include/gsp.h).  No fallback: importing
this module without the compiled library raises."""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgsp.so")

c_u32 = ctypes.c_uint32
c_u64 = ctypes.c_uint64
c_int = ctypes.c_int
c_dbl = ctypes.c_double
c_flt = ctypes.c_float
P = ctypes.c_void_p

GSP_MAX_PASS_STATS = 32
GSP_NOT_COUNTED = 0xFFFFFFFF
STATUS = {0: "ok", -1: "invalid argument", -2: "out of device memory", -3: "CUDA error",
          -4: "device wait timed out", -5: "capacity exceeded", -6: "graph not symmetric"}


class GspOpts(ctypes.Structure):
    _fields_ = [("max_passes", c_int), ("max_iterations", c_int), ("tolerance", c_dbl),
                ("tolerance_drop", c_dbl), ("aggregation_tolerance", c_dbl), ("split", c_int),
                ("split_when", c_int), ("move", c_int), ("waves", c_int), ("wave_repeats", c_int),
                ("no_return_from", c_int), ("precision", c_int),
                ("singleton_rule", c_int), ("prune", c_int), ("mlp_params", P),
                ("full_sweep_every", c_int), ("prune_threshold", c_flt), ("count_disconnected", c_int),
                ("refine", c_int), ("refine_theta", c_dbl), ("seed", c_u64),
                ("workspace", P), ("workspace_bytes", ctypes.c_size_t), ("stream", P)]


_N = GSP_MAX_PASS_STATS


class GspStats(ctypes.Structure):
    _fields_ = [("passes", c_int), ("iterations", c_int * _N), ("vertices", c_u32 * _N),
                ("communities", c_u32 * _N), ("edges", c_u64 * _N), ("ms_move", c_flt * _N),
                ("ms_split", c_flt * _N), ("ms_aggregate", c_flt * _N), ("ms_other", c_flt * _N),
                ("vertices_processed", c_u64 * _N), ("edges_scanned", c_u64 * _N),
                ("vertices_skipped", c_u64 * _N), ("move_bytes", c_dbl * _N),
                ("ms_move_kernels", c_flt * _N), ("final_communities", c_u32),
                ("modularity", c_dbl), ("ms_total", c_flt), ("disconnected", c_u32),
                ("workspace_bytes", c_u64), ("refined", c_u32 * _N), ("ms_refine", c_flt * _N)]


class GspDeviceGraph(ctypes.Structure):
    _fields_ = [("n", c_u32), ("nnz", c_u64), ("offsets", P), ("targets", P), ("weights", P)]


class GspTuning(ctypes.Structure):
    _fields_ = [("groups_blocks_per_sm", c_int), ("w512_blocks_per_sm", c_int), ("block_blocks_per_sm", c_int),
                ("hub_blocks_per_sm", c_int), ("persist_max_vertices", c_u32), ("group_max_degree", c_u32),
                ("warp_max_degree", c_u32), ("block_max_degree", c_u32), ("big_max_degree", c_u32)]


_SIGS = {
    "gsp_default_opts": (None, [P]),
    "gsp_status_string": (ctypes.c_char_p, [c_int]),
    "gsp_last_error": (ctypes.c_char_p, []),
    "gsp_louvain": (c_int, [P, P, P, c_u32, c_u64, P, P, P, P]),
    "gsp_louvain_host": (c_int, [P, P, P, c_u32, c_u64, P, P, P, P]),
    "gsp_louvain_batched": (c_int, [c_u32, P, P, P, P, c_u32, c_u64, P, P, P, P]),
    "gsp_vertex_weights": (c_int, [P, P, P, c_int, c_u32, c_u64, P, P, P]),
    "gsp_modularity": (c_int, [P, P, P, c_int, c_u32, c_u64, P, P, P]),
    "gsp_move_sweep": (c_int, [P, P, P, c_int, c_u32, c_u64, P, P, P, c_dbl, P, c_int, c_int, P, P,
                               P, P]),
    "gsp_local_move": (c_int, [P, P, P, c_int, c_u32, c_u64, P, P, P, c_dbl, c_dbl, c_int, c_int,
                               c_int, c_int, c_int, c_int, c_int, P, P]),
    "gsp_louvain_trace": (c_int, [P, P, P, c_u32, c_u64, P, P, P, P, c_u32, c_u32, P]),
    "gsp_split": (c_int, [P, P, c_u32, c_u64, P, c_int, P, P, P]),
    "gsp_refine": (c_int, [P, P, P, c_int, c_u32, c_u64, P, P, c_dbl, c_u64, c_u32, c_int, c_int, P, P]),
    "gsp_renumber": (c_int, [c_u32, P, P, P, P]),
    "gsp_lookup": (c_int, [c_u32, P, P, P]),
    "gsp_aggregate": (c_int, [P, P, P, c_int, c_u32, c_u64, P, c_u32, P, P, P, P, P]),
    "gsp_count_disconnected": (c_int, [P, P, c_u32, c_u64, P, P, P, P]),
    "gsp_mlp_param_count": (c_int, []),
    "gsp_mlp_forward": (c_int, [P, P, c_u32, P, P]),
    "gsp_mlp_backward": (c_int, [P, P, P, c_u32, P, P, P]),
    "gsp_mlp_sgd": (c_int, [P, P, c_flt, P]),
    "gsp_mlp_adam": (c_int, [P, P, P, P, c_flt, c_flt, c_flt, c_flt, c_int, P]),
    "gsp_get_tuning": (c_int, [P]),
    "gsp_set_tuning": (c_int, [P]),
    "gsp_autotune": (c_int, [P, P, P, c_u32, c_u64, P, P, P, P]),
    "gsp_autotune_batched": (c_int, [c_u32, P, P, P, P, c_u32, c_u64, P, P, P, P]),
    "gsp_gen_rmat": (c_int, [c_u32, c_u32, c_u64, c_u64, c_u64, c_u64, P, P]),
    "gsp_gen_planted_batch": (c_int, [c_u32, P, P, P, P, P, P, P]),
    "gsp_gen_grid": (c_int, [c_u32, c_u32, c_u64, c_u64, c_flt, c_flt, c_u64, P, P]),
    "gsp_release_graph": (None, []),
    "gsp_kernel_launches": (c_u64, []),
    "gsp_workspace_reserved": (c_u64, []),
    "gsp_release_workspace": (None, []),
    "gsp_modularity_static": (c_int, [P, P, P, c_int, c_u32, c_u64, P, P, P]),
}

_lib = None


def load():
    """Load libgsp.so (raises OSError when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError("libgsp.so not found at %s: run paper_2402_11454_gb300.build.build()" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


class GspError(RuntimeError):
    pass


def check(status):
    if status != 0:
        msg = load().gsp_last_error().decode(errors="replace")
        raise GspError("%s (%d): %s" % (STATUS.get(status, "unknown"), status, msg))
