"""Seeded synthetic graph generators (host side, numpy).

This module holds no arithmetic of the community-detection method: it only
draws graphs.  Both the CUDA path and the CPU oracle consume its output, and
the library carries a GPU twin of each generator (``gsp_gen_*``) that draws
the same edges from the same counter-based stream, for sizes numpy cannot
handle in reasonable time.

Random numbers: SplitMix64 (Steele, Lea and Flood, "Fast Splittable
Pseudorandom Number Generators", OOPSLA 2014) used counter-style: the value
for counter t of a stream is mix64(key + (t + 1) * GAMMA), with the stream key
mix64(seed * GAMMA + stream * STREAM_MUL).  Every draw is an integer
operation, so host and device agree bit for bit:
  * Bernoulli(p):   (r >> 11) < floor(p * 2^53)
  * uniform [0, N): ((r >> 32) * N) >> 32
  * weight in [lo, hi): float32(lo + (hi - lo) * (r >> 40) * 2^-24)

Graphs are returned as symmetric CSR (offsets u64, targets u32, weights f32)
with self-loops dropped and duplicate pairs merged (the smallest weight wins).
"""
import math

import numpy as np

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
STREAM_MUL = 0xD1B54A32D192ED03
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB

STREAM_RMAT = 1
STREAM_PLANTED = 2
STREAM_GRID_KEEP = 3
STREAM_GRID_WEIGHT = 4
STREAM_GRID_LONG = 5
STREAM_BATCH = 6

_U64 = np.uint64


def mix64_int(z):
    """SplitMix64 finaliser on a Python int."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * MIX1) & MASK64
    z = ((z ^ (z >> 27)) * MIX2) & MASK64
    return z ^ (z >> 31)


def stream_key(seed, stream):
    return mix64_int((seed * GAMMA + stream * STREAM_MUL) & MASK64)


def mix64(z):
    """SplitMix64 finaliser on a uint64 numpy array (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> _U64(30))) * _U64(MIX1)
        z = (z ^ (z >> _U64(27))) * _U64(MIX2)
        return z ^ (z >> _U64(31))


def rand_u64(key, ctr):
    """Counter-based draw: mix64(key + (ctr + 1) * GAMMA); ctr is a uint64 array."""
    with np.errstate(over="ignore"):
        return mix64(_U64(key) + (ctr + _U64(1)) * _U64(GAMMA))


def threshold53(p):
    """Integer threshold for Bernoulli(p) on the top 53 bits."""
    return int(p * (1 << 53))


def uniform_int(r, N):
    """((r >> 32) * N) >> 32 for N < 2^32 (elementwise; N may be an array)."""
    return (((r >> _U64(32)) * np.asarray(N, dtype=np.uint64)) >> _U64(32))


def weight_from(r, lo, hi):
    x = (r >> _U64(40)).astype(np.float64) * (2.0 ** -24)
    return (lo + (hi - lo) * x).astype(np.float32)


def edges_to_csr(n, u, v, w=None):
    """Undirected edge list -> symmetric CSR.  Self-loops are dropped; a pair
    seen more than once keeps its smallest weight."""
    u = np.asarray(u, dtype=np.uint64)
    v = np.asarray(v, dtype=np.uint64)
    if w is None:
        w = np.ones(len(u), dtype=np.float32)
    w = np.asarray(w, dtype=np.float32)
    keep = u != v
    u, v, w = u[keep], v[keep], w[keep]
    src = np.concatenate([u, v])
    dst = np.concatenate([v, u])
    ww = np.concatenate([w, w])
    key = (src << _U64(32)) | dst
    order = np.lexsort((ww, key))
    key = key[order]
    ww = ww[order]
    first = np.ones(len(key), dtype=bool)
    first[1:] = key[1:] != key[:-1]
    key = key[first]
    ww = ww[first]
    src = (key >> _U64(32)).astype(np.int64)
    tgt = (key & _U64(0xFFFFFFFF)).astype(np.uint32)
    counts = np.bincount(src, minlength=n)
    off = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(counts, out=off[1:])
    return off, tgt, ww.astype(np.float32)


def rmat_thresholds(a, b, c):
    return threshold53(a), threshold53(a + b), threshold53(a + b + c)


def rmat_edges(scale, edge_factor, a=0.57, b=0.19, c=0.19, seed=2, chunk=1 << 22):
    """R-MAT (Chakrabarti et al. 2004) edge samples: edge_factor * 2^scale
    draws; at level l (most significant bit first) one draw picks a quadrant
    with probabilities a, b, c, d = 1 - a - b - c.  No noise, no relabelling."""
    S = edge_factor << scale
    key = stream_key(seed, STREAM_RMAT)
    t1, t2, t3 = (_U64(t) for t in rmat_thresholds(a, b, c))
    us, vs = [], []
    for s0 in range(0, S, chunk):
        e = np.arange(s0, min(S, s0 + chunk), dtype=np.uint64)
        u = np.zeros(len(e), dtype=np.uint64)
        v = np.zeros(len(e), dtype=np.uint64)
        for lvl in range(scale):
            r = rand_u64(key, e * _U64(scale) + _U64(lvl)) >> _U64(11)
            bit = _U64(1) << _U64(scale - 1 - lvl)
            src1 = r >= t2                     # quadrants c, d
            dst1 = ((r >= t1) & (r < t2)) | (r >= t3)   # quadrants b, d
            u |= np.where(src1, bit, _U64(0))
            v |= np.where(dst1, bit, _U64(0))
        us.append(u)
        vs.append(v)
    return np.concatenate(us), np.concatenate(vs)


def rmat(scale, edge_factor=16, a=0.57, b=0.19, c=0.19, seed=2):
    u, v = rmat_edges(scale, edge_factor, a, b, c, seed)
    return edges_to_csr(1 << scale, u, v)


def planted_edges(n, k, num_edges, p_intra, seed, stream=STREAM_PLANTED):
    """Planted partition: vertex v belongs to community v mod k.  Each of the
    num_edges samples is, with probability p_intra, a uniform pair inside one
    uniformly chosen community, else a uniform pair over all vertices.
    Four draws per sample: intra test, community, two endpoints."""
    key = stream_key(seed, stream)
    e = np.arange(num_edges, dtype=np.uint64)
    r0 = rand_u64(key, _U64(4) * e) >> _U64(11)
    r1 = rand_u64(key, _U64(4) * e + _U64(1))
    r2 = rand_u64(key, _U64(4) * e + _U64(2))
    r3 = rand_u64(key, _U64(4) * e + _U64(3))
    intra = r0 < _U64(threshold53(p_intra))
    c = uniform_int(r1, k)
    size_c = (_U64(n) - c + _U64(k - 1)) // _U64(k)
    ui = c + _U64(k) * uniform_int(r2, size_c)
    vi = c + _U64(k) * uniform_int(r3, size_c)
    uo = uniform_int(r2, n)
    vo = uniform_int(r3, n)
    return np.where(intra, ui, uo), np.where(intra, vi, vo)


def planted(n=10000, k=64, mean_degree=16, p_intra=0.8, seed=1):
    """Planted-partition graph with n * mean_degree / 2 edge samples."""
    u, v = planted_edges(n, k, (n * mean_degree) // 2, p_intra, seed)
    return edges_to_csr(n, u, v)


def planted_truth(n, k):
    return (np.arange(n) % k).astype(np.uint32)


def grid_edges(R, Cc, p_remove=0.05, p_long=0.001, wlo=1.0, whi=10.0, seed=3):
    """R x Cc 4-neighbour grid (vertex r*Cc + c).  Horizontal edge e = r*(Cc-1)+c,
    vertical edge e = R*(Cc-1) + r*Cc + c.  Each grid edge is removed with
    probability p_remove; floor(p_long * #grid edges) uniform long-range pairs
    are added.  Weights are uniform in [wlo, whi): grid edge e uses weight draw
    e, long-range pair t uses weight draw #grid_edges + t."""
    nh = R * (Cc - 1)
    nv = (R - 1) * Cc
    E = nh + nv
    e = np.arange(E, dtype=np.uint64)
    kk = stream_key(seed, STREAM_GRID_KEEP)
    kw = stream_key(seed, STREAM_GRID_WEIGHT)
    kl = stream_key(seed, STREAM_GRID_LONG)
    keep = (rand_u64(kk, e) >> _U64(11)) >= _U64(threshold53(p_remove))
    w = weight_from(rand_u64(kw, e), wlo, whi)
    eh = e[:nh]
    r = eh // _U64(Cc - 1)
    c = eh % _U64(Cc - 1)
    hu = r * _U64(Cc) + c
    hv = hu + _U64(1)
    ev = e[nh:] - _U64(nh)
    vu = ev
    vv = ev + _U64(Cc)
    u = np.concatenate([hu, vu])[keep]
    v = np.concatenate([hv, vv])[keep]
    w = w[keep]
    L = int(p_long * E)
    t = np.arange(L, dtype=np.uint64)
    N = R * Cc
    lu = uniform_int(rand_u64(kl, _U64(2) * t), N)
    lv = uniform_int(rand_u64(kl, _U64(2) * t + _U64(1)), N)
    lw = weight_from(rand_u64(kw, _U64(E) + t), wlo, whi)
    return np.concatenate([u, lu]), np.concatenate([v, lv]), np.concatenate([w, lw])


def grid(R=4096, Cc=4096, p_remove=0.05, p_long=0.001, wlo=1.0, whi=10.0, seed=3):
    u, v, w = grid_edges(R, Cc, p_remove, p_long, wlo, whi, seed)
    return edges_to_csr(R * Cc, u, v, w)


def batch_params(num_graphs=4096, nmin=64, nmax=65536, kmin=4, kmax=64, dmin=4.0, dmax=64.0,
                 pmin=0.7, pmax=0.9, seed=4):
    """Per-graph parameters of the batched planted-partition set (host only):
    n log-uniform in [nmin, nmax], k uniform in {kmin..kmax} (capped at n),
    mean degree uniform in [dmin, dmax], intra fraction uniform in [pmin, pmax]."""
    key = stream_key(seed, STREAM_BATCH)
    g = np.arange(num_graphs, dtype=np.uint64)
    u0 = (rand_u64(key, _U64(4) * g) >> _U64(11)).astype(np.float64) * 2.0 ** -53
    u2 = (rand_u64(key, _U64(4) * g + _U64(2)) >> _U64(11)).astype(np.float64) * 2.0 ** -53
    u3 = (rand_u64(key, _U64(4) * g + _U64(3)) >> _U64(11)).astype(np.float64) * 2.0 ** -53
    n = np.floor(np.exp(math.log(nmin) + u0 * (math.log(nmax) - math.log(nmin)))).astype(np.int64)
    n = np.clip(n, nmin, nmax)
    k = kmin + uniform_int(rand_u64(key, _U64(4) * g + _U64(1)), kmax - kmin + 1).astype(np.int64)
    k = np.minimum(k, n)
    deg = dmin + (dmax - dmin) * u2
    p = pmin + (pmax - pmin) * u3
    edges = np.floor(n * deg / 2.0).astype(np.int64)
    return n, k, edges, p


def batch_graph_seed(seed, g):
    return (seed * 1000003 + g) & MASK64


def batch(num_graphs=4096, seed=4, **kw):
    """Concatenated batch of planted-partition graphs: returns the per-graph
    vertex offsets and one CSR over the union (no edge crosses graphs)."""
    n, k, edges, p = batch_params(num_graphs, seed=seed, **kw)
    voff = np.zeros(num_graphs + 1, dtype=np.uint64)
    np.cumsum(n, out=voff[1:])
    us, vs = [], []
    for g in range(num_graphs):
        u, v = planted_edges(int(n[g]), int(k[g]), int(edges[g]), float(p[g]),
                             batch_graph_seed(seed, g))
        us.append(u + voff[g])
        vs.append(v + voff[g])
    off, tgt, w = edges_to_csr(int(voff[-1]), np.concatenate(us), np.concatenate(vs))
    eoff = off[voff.astype(np.int64)]
    return voff, eoff, off, tgt, w
