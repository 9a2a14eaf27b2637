"""Python binding of libgsp (include/gsp.h): argument marshalling only.

Tensors are CUDA tensors: offsets int64 (read as uint64), targets and
memberships int32 (read as uint32), weights float32 or float64.  Every step
of the computation runs in the CUDA library; there is no CPU fallback.
"""
import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import GspOpts, GspStats, GspDeviceGraph, GspTuning, check

SPLIT = {"none": 0, "lp": 1, "lpp": 2, "bfs": 3, "sv": 4}
SPLIT_WHEN = {"pass": 0, "last": 1}
MOVE = {"async": 0, "sync": 1}
PRECISION = {"mixed": 0, "fp64": 1}
PRUNE = {"flags": 0, "learned": 1}
W_F32, W_F64 = 0, 1


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _cuda(t, dtype, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return t


def _wt(w):
    if w.dtype == torch.float32:
        return W_F32
    if w.dtype == torch.float64:
        return W_F64
    raise TypeError("weights must be float32 or float64")


def _graph(off, tgt, w=None):
    _cuda(off, torch.int64, "offsets")
    _cuda(tgt, torch.int32, "targets")
    if w is not None:
        if not (w.is_cuda and w.is_contiguous()):
            raise TypeError("weights must be a contiguous CUDA tensor")
    n = off.numel() - 1
    nnz = tgt.numel()
    return n, nnz


def make_opts(max_passes=10, max_iterations=20, tolerance=1e-2, tolerance_drop=10.0,
              aggregation_tolerance=0.8, split="lpp", split_when="pass", move="sync", waves=0,
              wave_repeats=3, no_return_from=3, precision="mixed", singleton_rule=True, prune="flags", mlp_params=None,
              full_sweep_every=4, prune_threshold=0.5, count_disconnected=False, refine=False, refine_theta=0.01,
              seed=0, workspace=None, stream=None):
    o = GspOpts()
    _lib.load().gsp_default_opts(ctypes.byref(o))
    o.max_passes = max_passes
    o.max_iterations = max_iterations
    o.tolerance = tolerance
    o.tolerance_drop = tolerance_drop
    o.aggregation_tolerance = aggregation_tolerance
    o.split = SPLIT[split]
    o.split_when = SPLIT_WHEN[split_when]
    o.move = MOVE[move]
    o.waves = waves
    o.wave_repeats = wave_repeats
    o.no_return_from = no_return_from
    o.precision = PRECISION[precision]
    o.singleton_rule = int(bool(singleton_rule))
    o.prune = PRUNE[prune]
    o.mlp_params = None if mlp_params is None else _cuda(mlp_params, torch.float32, "mlp_params").data_ptr()
    o.full_sweep_every = full_sweep_every
    o.prune_threshold = prune_threshold
    o.count_disconnected = int(bool(count_disconnected))
    o.refine = int(bool(refine))
    o.refine_theta = refine_theta
    o.seed = seed
    if workspace is not None:
        _cuda(workspace, torch.uint8, "workspace")
        o.workspace = workspace.data_ptr()
        o.workspace_bytes = workspace.numel()
    o.stream = _stream(stream).value
    return o


def stats_dict(st):
    p = min(st.passes, _lib.GSP_MAX_PASS_STATS)
    return dict(passes=st.passes, iterations=list(st.iterations[:p]), vertices=list(st.vertices[:p]),
                communities=list(st.communities[:p]), edges=list(st.edges[:p]),
                ms_move=list(st.ms_move[:p]), ms_split=list(st.ms_split[:p]),
                ms_aggregate=list(st.ms_aggregate[:p]), ms_other=list(st.ms_other[:p]),
                vertices_processed=list(st.vertices_processed[:p]),
                edges_scanned=list(st.edges_scanned[:p]),
                vertices_skipped=list(st.vertices_skipped[:p]),
                move_bytes=list(st.move_bytes[:p]), ms_move_kernels=list(st.ms_move_kernels[:p]),
                final_communities=st.final_communities, modularity=st.modularity,
                ms_total=st.ms_total,
                disconnected=None if st.disconnected == _lib.GSP_NOT_COUNTED else st.disconnected,
                workspace_bytes=st.workspace_bytes, refined=list(st.refined[:p]),
                ms_refine=list(st.ms_refine[:p]))


def louvain(offsets, targets, weights, membership=None, **kw):
    """GSP-Louvain (Algorithm 1) on a device CSR; returns (membership, Q, stats)."""
    n, nnz = _graph(offsets, targets, weights)
    _cuda(weights, torch.float32, "weights")
    o = make_opts(**kw)
    if membership is None:
        membership = torch.empty(n, dtype=torch.int32, device=offsets.device)
    q = ctypes.c_double()
    st = GspStats()
    check(_lib.load().gsp_louvain(_p(offsets), _p(targets), _p(weights), n, nnz, ctypes.byref(o),
                                  _p(membership), ctypes.byref(q), ctypes.byref(st)))
    return membership, q.value, stats_dict(st)


def louvain_host(offsets, targets, weights, membership=None, **kw):
    """As louvain, on HOST (CPU, ideally pinned) tensors; copies inside the call."""
    for t, nm in ((offsets, "offsets"), (targets, "targets"), (weights, "weights")):
        if t.is_cuda or not t.is_contiguous():
            raise TypeError("%s must be a contiguous CPU tensor" % nm)
    n = offsets.numel() - 1
    nnz = targets.numel()
    o = make_opts(**kw)
    if membership is None:
        membership = torch.empty(n, dtype=torch.int32, pin_memory=True)
    q = ctypes.c_double()
    st = GspStats()
    check(_lib.load().gsp_louvain_host(_p(offsets), _p(targets), _p(weights), n, nnz, ctypes.byref(o),
                                       _p(membership), ctypes.byref(q), ctypes.byref(st)))
    return membership, q.value, stats_dict(st)


def louvain_batched(graph_vertex_offsets, offsets, targets, weights, membership=None, **kw):
    """Batched GSP-Louvain over concatenated independent graphs; returns
    (membership (graph-local ids), per-graph modularity tensor, stats)."""
    n, nnz = _graph(offsets, targets, weights)
    gvo = np.ascontiguousarray(np.asarray(graph_vertex_offsets, dtype=np.uint64))
    G = len(gvo) - 1
    o = make_opts(**kw)
    if membership is None:
        membership = torch.empty(n, dtype=torch.int32, device=offsets.device)
    q = torch.empty(G, dtype=torch.float64, device=offsets.device)
    st = GspStats()
    check(_lib.load().gsp_louvain_batched(G, gvo.ctypes.data_as(ctypes.c_void_p), _p(offsets), _p(targets),
                                          _p(weights), n, nnz, ctypes.byref(o), _p(membership), _p(q),
                                          ctypes.byref(st)))
    return membership, q, stats_dict(st)


def vertex_weights(offsets, targets, weights, stream=None):
    n, nnz = _graph(offsets, targets, weights)
    K = torch.empty(n, dtype=torch.float64, device=offsets.device)
    m = ctypes.c_double()
    check(_lib.load().gsp_vertex_weights(_p(offsets), _p(targets), _p(weights), _wt(weights), n, nnz,
                                         _p(K), ctypes.byref(m), _stream(stream)))
    return K, m.value


def modularity(offsets, targets, weights, C, stream=None):
    n, nnz = _graph(offsets, targets, weights)
    _cuda(C, torch.int32, "membership")
    q = ctypes.c_double()
    check(_lib.load().gsp_modularity(_p(offsets), _p(targets), _p(weights), _wt(weights), n, nnz, _p(C),
                                     ctypes.byref(q), _stream(stream)))
    return q.value


def modularity_static(offsets, targets, weights, C, stream=None):
    """Equation 1 without device allocation (fixed internal scratch; n <= 2^20)."""
    n, nnz = _graph(offsets, targets, weights)
    _cuda(C, torch.int32, "membership")
    q = ctypes.c_double()
    check(_lib.load().gsp_modularity_static(_p(offsets), _p(targets), _p(weights), _wt(weights), n, nnz, _p(C),
                                            ctypes.byref(q), _stream(stream)))
    return q.value


def move_sweep(offsets, targets, weights, C, K, Sigma, m, active=None, precision="fp64",
               singleton_rule=True, stream=None):
    """One frozen-state local-moving sweep; returns (choice, dq, moved)."""
    n, nnz = _graph(offsets, targets, weights)
    choice = torch.empty(n, dtype=torch.int32, device=offsets.device)
    dq = ctypes.c_double()
    moved = ctypes.c_uint32()
    if active is not None:
        _cuda(active, torch.uint8, "active")
    check(_lib.load().gsp_move_sweep(_p(offsets), _p(targets), _p(weights), _wt(weights), n, nnz, _p(C),
                                     _p(K), _p(Sigma), m, _p(active), PRECISION[precision],
                                     int(bool(singleton_rule)), _p(choice), ctypes.byref(dq),
                                     ctypes.byref(moved), _stream(stream)))
    return choice, dq.value, moved.value


def local_move(offsets, targets, weights, C, K, Sigma, m, tolerance=1e-2, max_iterations=20,
               move="sync", waves=17, wave_repeats=3, no_return_from=3, precision="fp64", singleton_rule=True,
               stream=None):
    """louvainMove (Algorithm 4); C and Sigma are updated in place; returns l_i."""
    n, nnz = _graph(offsets, targets, weights)
    it = ctypes.c_int()
    check(_lib.load().gsp_local_move(_p(offsets), _p(targets), _p(weights), _wt(weights), n, nnz, _p(C),
                                     _p(K), _p(Sigma), m, tolerance, max_iterations, MOVE[move], waves,
                                     wave_repeats, no_return_from, PRECISION[precision], int(bool(singleton_rule)),
                                     ctypes.byref(it), _stream(stream)))
    return it.value


def louvain_trace(offsets, targets, weights, capacity, sample_every=8, with_keys=False, **kw):
    """Run the plain method and record move/no-move trace rows:
    (features [rows, 6] float32, labels [rows] uint8), plus the visit keys
    [rows] int64 (pass << 56 | iteration << 48 | repeat << 40 | vertex) when
    with_keys is set."""
    n, nnz = _graph(offsets, targets, weights)
    o = make_opts(**kw)
    x = torch.empty((capacity, 6), dtype=torch.float32, device=offsets.device)
    y = torch.empty(capacity, dtype=torch.uint8, device=offsets.device)
    keys = torch.empty(capacity, dtype=torch.int64, device=offsets.device) if with_keys else None
    rows = ctypes.c_uint32()
    check(_lib.load().gsp_louvain_trace(_p(offsets), _p(targets), _p(weights), n, nnz, ctypes.byref(o),
                                        _p(x), _p(y), _p(keys), capacity, sample_every, ctypes.byref(rows)))
    if with_keys:
        return x[:rows.value], y[:rows.value], keys[:rows.value]
    return x[:rows.value], y[:rows.value]


def split(offsets, targets, C, mode="bfs", stream=None):
    """Split step (Algorithms 2, 3): (labels, number of components)."""
    n, nnz = _graph(offsets, targets)
    labels = torch.empty(n, dtype=torch.int32, device=offsets.device)
    k = ctypes.c_uint32()
    check(_lib.load().gsp_split(_p(offsets), _p(targets), n, nnz, _p(C), SPLIT[mode], _p(labels),
                                ctypes.byref(k), _stream(stream)))
    return labels, k.value


def refine(offsets, targets, weights, B, theta=0.01, seed=0, pass_index=0, waves=0, precision="fp64", stream=None):
    """Leiden refinement (Section 3.5) of the bound membership B: (refined
    membership named by member vertex ids, number of vertices that joined)."""
    n, nnz = _graph(offsets, targets, weights)
    _cuda(B, torch.int32, "bound membership")
    R = torch.empty(n, dtype=torch.int32, device=offsets.device)
    moves = ctypes.c_uint32()
    check(_lib.load().gsp_refine(_p(offsets), _p(targets), _p(weights), _wt(weights), n, nnz, _p(B), _p(R),
                                 float(theta), int(seed), int(pass_index), int(waves), PRECISION[precision],
                                 ctypes.byref(moves),
                                 _stream(stream)))
    return R, moves.value


def renumber(C, stream=None):
    _cuda(C, torch.int32, "membership")
    out = torch.empty_like(C)
    k = ctypes.c_uint32()
    check(_lib.load().gsp_renumber(C.numel(), _p(C), _p(out), ctypes.byref(k), _stream(stream)))
    return out, k.value


def lookup(C_top, C_pass, stream=None):
    check(_lib.load().gsp_lookup(C_top.numel(), _p(C_top), _p(C_pass), _stream(stream)))
    return C_top


def aggregate(offsets, targets, weights, C, k, stream=None):
    """louvainAggregate (Algorithm 5): (offsets, targets, float64 weights)."""
    n, nnz = _graph(offsets, targets, weights)
    dev = offsets.device
    o2 = torch.empty(k + 1, dtype=torch.int64, device=dev)
    t2 = torch.empty(max(nnz, 1), dtype=torch.int32, device=dev)
    w2 = torch.empty(max(nnz, 1), dtype=torch.float64, device=dev)
    e = ctypes.c_uint64()
    check(_lib.load().gsp_aggregate(_p(offsets), _p(targets), _p(weights), _wt(weights), n, nnz, _p(C), k,
                                    _p(o2), _p(t2), _p(w2), ctypes.byref(e), _stream(stream)))
    return o2, t2[:e.value], w2[:e.value]


def count_disconnected(offsets, targets, C, stream=None):
    n, nnz = _graph(offsets, targets)
    flags = torch.empty(n, dtype=torch.uint8, device=offsets.device)
    c = ctypes.c_uint32()
    check(_lib.load().gsp_count_disconnected(_p(offsets), _p(targets), n, nnz, _p(C), _p(flags),
                                             ctypes.byref(c), _stream(stream)))
    return c.value, flags


_TUNING_FIELDS = ("groups_blocks_per_sm", "w512_blocks_per_sm", "block_blocks_per_sm", "hub_blocks_per_sm",
                  "persist_max_vertices", "group_max_degree", "warp_max_degree", "block_max_degree",
                  "big_max_degree")


def get_tuning():
    """Grid caps (blocks per SM) of the local-moving kernels, as a dict."""
    t = GspTuning()
    check(_lib.load().gsp_get_tuning(ctypes.byref(t)))
    return {f: getattr(t, f) for f in _TUNING_FIELDS}


def set_tuning(**caps):
    """Install grid caps; fields not given keep their current values."""
    cur = get_tuning()
    cur.update(caps)
    t = GspTuning(*[int(cur[f]) for f in _TUNING_FIELDS])
    check(_lib.load().gsp_set_tuning(ctypes.byref(t)))
    return get_tuning()


def autotune(offsets, targets, weights, graph_vertex_offsets=None, **kw):
    """Pick and install the grid caps and class boundaries for this graph (or,
    with graph_vertex_offsets, for this batch through the batched call);
    returns (settings, ms of a call before, ms after)."""
    n, nnz = _graph(offsets, targets, weights)
    o = make_opts(**kw)
    t = GspTuning()
    before, after = ctypes.c_float(), ctypes.c_float()
    if graph_vertex_offsets is None:
        check(_lib.load().gsp_autotune(_p(offsets), _p(targets), _p(weights), n, nnz, ctypes.byref(o),
                                       ctypes.byref(t), ctypes.byref(before), ctypes.byref(after)))
    else:
        gvo = np.ascontiguousarray(np.asarray(graph_vertex_offsets, dtype=np.uint64))
        check(_lib.load().gsp_autotune_batched(len(gvo) - 1, gvo.ctypes.data_as(ctypes.c_void_p), _p(offsets),
                                               _p(targets), _p(weights), n, nnz, ctypes.byref(o),
                                               ctypes.byref(t), ctypes.byref(before), ctypes.byref(after)))
    return {f: getattr(t, f) for f in _TUNING_FIELDS}, before.value, after.value


def kernel_launches():
    """Kernels launched by libgsp so far (process-wide counter)."""
    return _lib.load().gsp_kernel_launches()


def workspace_reserved():
    """Bytes of device memory held by libgsp's internal workspaces."""
    return _lib.load().gsp_workspace_reserved()


def release_workspace():
    """Free libgsp's internal workspace on the current device."""
    _lib.load().gsp_release_workspace()


# ------------------------------------------------------------------ MLP
def mlp_param_count():
    return _lib.load().gsp_mlp_param_count()


def mlp_forward(params, x, stream=None):
    rows = x.shape[0]
    p = torch.empty(rows, dtype=torch.float32, device=x.device)
    check(_lib.load().gsp_mlp_forward(_p(params), _p(x), rows, _p(p), _stream(stream)))
    return p


def mlp_backward(params, x, y, stream=None):
    grad = torch.empty(mlp_param_count(), dtype=torch.float32, device=x.device)
    loss = ctypes.c_double()
    check(_lib.load().gsp_mlp_backward(_p(params), _p(x), _p(y), x.shape[0], _p(grad), ctypes.byref(loss),
                                       _stream(stream)))
    return grad, loss.value


def mlp_sgd(params, grad, lr, stream=None):
    check(_lib.load().gsp_mlp_sgd(_p(params), _p(grad), lr, _stream(stream)))
    return params


def mlp_adam(params, grad, m, v, lr, t, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    check(_lib.load().gsp_mlp_adam(_p(params), _p(grad), _p(m), _p(v), lr, beta1, beta2, eps, t,
                                   _stream(stream)))
    return params


# ------------------------------------------------------------ generators
class _DevArray:
    """Wraps a device pointer for torch.as_tensor (no copy)."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False),
                                         "version": 3}


def _take_graph(g):
    """Copy the library-owned generated CSR into torch tensors."""
    n, nnz = g.n, g.nnz
    torch.cuda.synchronize()
    off = torch.as_tensor(_DevArray(g.offsets, n + 1, "<i8"), device="cuda").clone()
    tgt = torch.as_tensor(_DevArray(g.targets, max(nnz, 1), "<i4"), device="cuda")[:nnz].clone()
    w = torch.as_tensor(_DevArray(g.weights, max(nnz, 1), "<f4"), device="cuda")[:nnz].clone()
    torch.cuda.synchronize()
    _lib.load().gsp_release_graph()
    return off, tgt, w


def gen_rmat(scale, edge_factor=16, a=0.57, b=0.19, c=0.19, seed=2):
    from .graphgen import rmat_thresholds
    t1, t2, t3 = rmat_thresholds(a, b, c)
    g = GspDeviceGraph()
    check(_lib.load().gsp_gen_rmat(scale, edge_factor, t1, t2, t3, seed, ctypes.byref(g), _stream()))
    return _take_graph(g)


def gen_planted_batch(n_g, k_g, edges_g, p_g, seeds_g):
    from .graphgen import threshold53
    G = len(n_g)
    arrs = [np.ascontiguousarray(np.asarray(a, dtype=np.uint64)) for a in
            (n_g, k_g, edges_g, [threshold53(float(p)) for p in p_g], seeds_g)]
    g = GspDeviceGraph()
    check(_lib.load().gsp_gen_planted_batch(G, *[a.ctypes.data_as(ctypes.c_void_p) for a in arrs],
                                            ctypes.byref(g), _stream()))
    return _take_graph(g)


def gen_planted(n=10000, k=64, mean_degree=16, p_intra=0.8, seed=1):
    return gen_planted_batch([n], [k], [(n * mean_degree) // 2], [p_intra], [seed])


def gen_grid(R=4096, Cc=4096, p_remove=0.05, p_long=0.001, wlo=1.0, whi=10.0, seed=3):
    from .graphgen import threshold53
    E = R * (Cc - 1) + (R - 1) * Cc
    g = GspDeviceGraph()
    check(_lib.load().gsp_gen_grid(R, Cc, threshold53(p_remove), int(p_long * E), wlo, whi, seed,
                                   ctypes.byref(g), _stream()))
    return _take_graph(g)
