"""ctypes marshalling for the C oracle (oracle.c).  Test infrastructure only.

Nothing here computes the method: every call forwards numpy arrays to the C
functions, which follow the paper step by step in FP64.
"""
import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build_oracle(force=False):
    """Compile oracle.c with gcc (-O2, no FP contraction) into liboracle.so."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


class _OgGraph(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("nnz", ctypes.c_uint64),
                ("off", ctypes.c_void_p), ("tgt", ctypes.c_void_p), ("w", ctypes.c_void_p)]


class _OgOpts(ctypes.Structure):
    _fields_ = [("max_passes", ctypes.c_int), ("max_iterations", ctypes.c_int),
                ("tolerance", ctypes.c_double), ("tolerance_drop", ctypes.c_double),
                ("aggregation_tolerance", ctypes.c_double), ("split", ctypes.c_int),
                ("split_last", ctypes.c_int), ("sync", ctypes.c_int), ("waves", ctypes.c_int),
                ("wave_hash", ctypes.c_int), ("wave_repeats", ctypes.c_int), ("no_return_from", ctypes.c_int),
                ("singleton_rule", ctypes.c_int), ("refine", ctypes.c_int), ("refine_theta", ctypes.c_double),
                ("seed", ctypes.c_uint64)]


class _OgStats(ctypes.Structure):
    _fields_ = [("passes", ctypes.c_int), ("iterations", ctypes.c_int * 64),
                ("vertices", ctypes.c_uint32 * 64), ("communities", ctypes.c_uint32 * 64),
                ("modularity", ctypes.c_double), ("final_communities", ctypes.c_uint32)]


def _load():
    global _lib
    if _lib is None:
        build_oracle()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        G = ctypes.POINTER(_OgGraph)
        lib.og_vertex_weights.argtypes = [G, P]
        lib.og_vertex_weights.restype = ctypes.c_double
        lib.og_modularity.argtypes = [G, P]
        lib.og_modularity.restype = ctypes.c_double
        lib.og_delta_modularity.argtypes = [ctypes.c_double] * 6
        lib.og_delta_modularity.restype = ctypes.c_double
        lib.og_move_sweep_sync.argtypes = [G, P, P, P, P, ctypes.c_int, ctypes.c_double, P, P, P, P]
        lib.og_move_sweep_sync.restype = None
        lib.og_move.argtypes = [G, P, P, P, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                ctypes.c_int, P]
        lib.og_wave_hash.argtypes = [ctypes.c_uint32]
        lib.og_wave_hash.restype = ctypes.c_uint32
        lib.og_move.restype = ctypes.c_int
        lib.og_split_lp.argtypes = [G, P, P, ctypes.c_int]
        lib.og_split_lp.restype = ctypes.c_int
        lib.og_split_bfs.argtypes = [G, P, P]
        lib.og_split_bfs.restype = None
        lib.og_renumber.argtypes = [ctypes.c_uint32, P]
        lib.og_renumber.restype = ctypes.c_uint32
        lib.og_lookup.argtypes = [ctypes.c_uint64, P, P]
        lib.og_lookup.restype = None
        lib.og_aggregate.argtypes = [G, P, ctypes.c_uint32, P, P, P]
        lib.og_aggregate.restype = ctypes.c_uint64
        lib.og_splitmix64.argtypes = [ctypes.c_uint64]
        lib.og_splitmix64.restype = ctypes.c_uint64
        lib.og_refine_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32]
        lib.og_refine_uniform.restype = ctypes.c_double
        lib.og_refine.argtypes = [G, P, P, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                                  ctypes.c_int]
        lib.og_refine.restype = ctypes.c_uint32
        lib.og_disconnected.argtypes = [G, P, P]
        lib.og_disconnected.restype = ctypes.c_uint32
        lib.og_louvain.argtypes = [G, ctypes.POINTER(_OgOpts), P, ctypes.POINTER(_OgStats)]
        lib.og_louvain.restype = ctypes.c_int
        lib.og_louvain_trace.argtypes = [G, ctypes.POINTER(_OgOpts), P, ctypes.POINTER(_OgStats), P,
                                         ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]
        lib.og_louvain_trace.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


class Graph:
    """Symmetric CSR held as numpy arrays (offsets u64, targets u32, weights f64)."""

    def __init__(self, offsets, targets, weights):
        self.offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        self.targets = np.ascontiguousarray(targets, dtype=np.uint32)
        self.weights = np.ascontiguousarray(weights, dtype=np.float64)
        self.n = len(self.offsets) - 1
        self.nnz = int(self.offsets[-1]) if self.n >= 0 else 0
        self._s = _OgGraph(self.n, self.nnz, _p(self.offsets), _p(self.targets), _p(self.weights))

    @property
    def ref(self):
        return ctypes.byref(self._s)


def _u32(a):
    return np.ascontiguousarray(a, dtype=np.uint32)


def vertex_weights(g):
    """Section 3: K_i and m."""
    K = np.zeros(g.n, dtype=np.float64)
    m = _load().og_vertex_weights(g.ref, _p(K))
    return K, m


def modularity(g, C):
    """Equation 1 (per-community form)."""
    C = _u32(C)
    return _load().og_modularity(g.ref, _p(C))


def delta_modularity(Kic, Kid, Ki, Sc, Sd, m):
    """Equation 2."""
    return _load().og_delta_modularity(Kic, Kid, Ki, Sc, Sd, m)


def move_sweep_sync(g, C, K, Sigma, m, active=None, singleton_rule=True):
    """One frozen-state local-moving sweep (Algorithm 4): per-vertex choice,
    best and runner-up delta-modularity."""
    C = _u32(C)
    K = np.ascontiguousarray(K, dtype=np.float64)
    Sigma = np.ascontiguousarray(Sigma, dtype=np.float64)
    size = np.bincount(C, minlength=g.n).astype(np.uint32)
    act = None if active is None else np.ascontiguousarray(active, dtype=np.uint8)
    choice = np.zeros(g.n, dtype=np.uint32)
    best = np.zeros(g.n, dtype=np.float64)
    second = np.zeros(g.n, dtype=np.float64)
    _load().og_move_sweep_sync(g.ref, _p(C), _p(K), _p(Sigma), _p(size), int(bool(singleton_rule)),
                               m, _p(act), _p(choice), _p(best), _p(second))
    return choice, best, second


def move(g, C, K, Sigma, m, tau, max_iterations=20, sync=True, singleton_rule=True, waves=1, wave_repeats=1,
         wave_hash=True, no_return_from=0):
    """louvainMove (Algorithm 4); returns (C, Sigma, l_i, dq per iteration).
    sync=True runs frozen-state waves (vertex i in wave hash(i) mod waves, or
    i mod waves without wave_hash); in the first iteration each wave runs
    wave_repeats times (a repeat takes the wave's vertices re-marked by the
    previous repeat's moves); from iteration no_return_from on (0: never) a
    vertex does not move back to the community it left the iteration before."""
    C = _u32(C).copy()
    K = np.ascontiguousarray(K, dtype=np.float64)
    Sigma = np.ascontiguousarray(Sigma, dtype=np.float64).copy()
    dq = np.zeros(max(max_iterations, 1), dtype=np.float64)
    li = _load().og_move(g.ref, _p(C), _p(K), _p(Sigma), m, tau, max_iterations, int(bool(sync)),
                         int(waves), int(bool(wave_hash)), int(wave_repeats), int(no_return_from),
                         int(bool(singleton_rule)), _p(dq))
    return C, Sigma, li, dq[:li]


def split_lp(g, C, prune=False):
    """splitDisconnectedLp (Algorithm 2); prune=True is LPP."""
    C = _u32(C)
    Cp = np.zeros(g.n, dtype=np.uint32)
    iters = _load().og_split_lp(g.ref, _p(C), _p(Cp), int(bool(prune)))
    return Cp, iters


def split_bfs(g, C):
    """splitDisconnectedBfs (Algorithm 3)."""
    C = _u32(C)
    Cp = np.zeros(g.n, dtype=np.uint32)
    _load().og_split_bfs(g.ref, _p(C), _p(Cp))
    return Cp


def renumber(C):
    """Renumber communities (Algorithm 1) by increasing id."""
    C = _u32(C).copy()
    k = _load().og_renumber(len(C), _p(C))
    return C, k


def lookup(C, Cp):
    """Dendrogram lookup (Algorithm 1)."""
    C = _u32(C).copy()
    Cp = _u32(Cp)
    _load().og_lookup(len(C), _p(C), _p(Cp))
    return C


def aggregate(g, C, k):
    """louvainAggregate (Algorithm 5) -> Graph with sorted rows."""
    C = _u32(C)
    off = np.zeros(k + 1, dtype=np.uint64)
    tgt = np.zeros(max(g.nnz, 1), dtype=np.uint32)
    w = np.zeros(max(g.nnz, 1), dtype=np.float64)
    nnz2 = _load().og_aggregate(g.ref, _p(C), k, _p(off), _p(tgt), _p(w))
    return Graph(off, tgt[:nnz2].copy(), w[:nnz2].copy())


def disconnected(g, C):
    """disconnectedCommunities (Algorithm 6): (count, per-community flags)."""
    C = _u32(C)
    D = np.zeros(max(g.n, 1), dtype=np.uint8)
    cnt = _load().og_disconnected(g.ref, _p(C), _p(D))
    return cnt, D[:g.n]


def splitmix64(x):
    """SplitMix64's output for generator state x (og_splitmix64)."""
    return int(_load().og_splitmix64(int(x) & 0xFFFFFFFFFFFFFFFF))


def refine_uniform(seed, pass_index, v, c):
    """The uniform draw in (0,1) of the refinement choice (og_refine_uniform)."""
    return _load().og_refine_uniform(int(seed), int(pass_index), int(v), int(c))


def refine(g, B, theta=0.01, seed=0, pass_index=0, waves=17, wave_hash=True):
    """Leiden refinement (Section 3.5) of the bound membership B: (refined
    membership named by member vertex ids, number of vertices that joined)."""
    B = _u32(B)
    R = np.zeros(g.n, dtype=np.uint32)
    moves = _load().og_refine(g.ref, _p(B), _p(R), float(theta), int(seed), int(pass_index), int(waves),
                              int(bool(wave_hash)))
    return R, int(moves)


SPLIT_MODES = {"none": 0, "lp": 1, "lpp": 2, "bfs": 3}


@dataclass
class LouvainOptions:
    max_passes: int = 10
    max_iterations: int = 20
    tolerance: float = 1e-2
    tolerance_drop: float = 10.0
    aggregation_tolerance: float = 0.8
    split: str = "bfs"
    split_last: bool = False
    sync: bool = True
    waves: int = 17
    wave_hash: bool = True
    wave_repeats: int = 3
    no_return_from: int = 3
    singleton_rule: bool = True
    refine: bool = False
    refine_theta: float = 0.01
    seed: int = 0


def louvain(g, opts=None):
    """louvain (Algorithm 1): (membership, stats dict)."""
    o = opts or LouvainOptions()
    co = _OgOpts(o.max_passes, o.max_iterations, o.tolerance, o.tolerance_drop,
                 o.aggregation_tolerance, SPLIT_MODES[o.split], int(o.split_last), int(o.sync),
                 int(o.waves), int(bool(o.wave_hash)), int(o.wave_repeats), int(o.no_return_from),
                 int(o.singleton_rule), int(bool(o.refine)), float(o.refine_theta), int(o.seed))
    C = np.zeros(g.n, dtype=np.uint32)
    st = _OgStats()
    _load().og_louvain(g.ref, ctypes.byref(co), _p(C), ctypes.byref(st))
    p = st.passes
    stats = dict(passes=p, iterations=list(st.iterations[:p]), vertices=list(st.vertices[:p]),
                 communities=list(st.communities[:p]), modularity=st.modularity,
                 final_communities=st.final_communities)
    return C, stats


TRACE_FIELDS = ("pass", "iteration", "repeat", "vertex", "degree", "K", "kept", "gain", "moved_last", "moved",
                "max_K")


def louvain_trace(g, opts=None, capacity=1 << 20):
    """louvain (Algorithm 1) recording every local-moving visit: returns
    (membership, stats, records) with records a dict of arrays named by
    TRACE_FIELDS (the vertex's state before the visit; see og_trace in
    oracle.c).  Raises if the run made more than `capacity` visits."""
    o = opts or LouvainOptions()
    co = _OgOpts(o.max_passes, o.max_iterations, o.tolerance, o.tolerance_drop,
                 o.aggregation_tolerance, SPLIT_MODES[o.split], int(o.split_last), int(o.sync),
                 int(o.waves), int(bool(o.wave_hash)), int(o.wave_repeats), int(o.no_return_from),
                 int(o.singleton_rule), int(bool(o.refine)), float(o.refine_theta), int(o.seed))
    C = np.zeros(g.n, dtype=np.uint32)
    st = _OgStats()
    rec = np.zeros((capacity, len(TRACE_FIELDS)), dtype=np.float64)
    n = ctypes.c_uint64()
    _load().og_louvain_trace(g.ref, ctypes.byref(co), _p(C), ctypes.byref(st), _p(rec), capacity,
                             ctypes.byref(n))
    if n.value > capacity:
        raise ValueError("trace needs %d records, capacity %d" % (n.value, capacity))
    rec = rec[:n.value]
    return C, {"passes": st.passes, "modularity": st.modularity}, {k: rec[:, j] for j, k in
                                                                   enumerate(TRACE_FIELDS)}


def wave_hash(i):
    """The wave hash of vertex ids (og_wave_hash): MurmurHash3's 32-bit
    finaliser."""
    f = _load().og_wave_hash
    return np.array([f(int(x)) for x in np.atleast_1d(i)], dtype=np.uint32)
