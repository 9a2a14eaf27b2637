"""Batched GSP-Louvain (many independent graphs in one run) through the C ABI.

Each graph of a batch must get exactly the result it gets when run alone:
the same membership (graph-local ids ordered by smallest vertex) and the
same Equation 1 value, in every deterministic mode (frozen-state sweeps).
In FP64 mode that is also the oracle's membership.  The batches mix the
planted-partition recipe of the batched workload (uneven sizes, community
counts, degrees and mixing) with degenerate members: empty graphs, edgeless
graphs, a single vertex, a self-loop, two cliques and a star."""
import numpy as np
import pytest
import torch

import oracle
from paper_2402_11454_gb300 import graphgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gsp():
    from paper_2402_11454_gb300 import build
    build.build()
    from paper_2402_11454_gb300 import gsp as g
    return g


def csr_from_edges(n, edges):
    if not edges:
        return np.zeros(n + 1, np.uint64), np.zeros(0, np.uint32), np.zeros(0, np.float32)
    u = np.array([a for a, b in edges], dtype=np.uint64)
    v = np.array([b for a, b in edges], dtype=np.uint64)
    return graphgen.edges_to_csr(n, u, v)


def members():
    out = []
    voff, eoff, off, tgt, w = graphgen.batch(num_graphs=20, nmax=3000, seed=4)
    for g in range(20):
        a, b = int(voff[g]), int(voff[g + 1])
        lo, hi = int(off[a]), int(off[b])
        out.append((off[a:b + 1] - off[a], (tgt[lo:hi] - a).astype(np.uint32), w[lo:hi]))
    n = 300
    star = [(0, i) for i in range(1, n)] + [(i, i + 1) for i in range(1, n - 1)]
    cliques = [(a, b) for a in range(4) for b in range(4) if a < b] + \
              [(a, b) for a in range(4, 8) for b in range(4, 8) if a < b]
    extra = [csr_from_edges(5, []), csr_from_edges(1, []), csr_from_edges(3, [(1, 1)]),
             csr_from_edges(8, cliques), csr_from_edges(n, star)]
    # interleave, with empty graphs at the front, middle and end
    res = [None]
    for i, g in enumerate(out):
        res.append(g)
        if i % 4 == 1 and extra:
            res.append(extra.pop())
        if i == 10:
            res.append(None)
    res += extra + [None]
    return res


def concat(gs):
    gvo = [0]
    offs, tgts, ws = [np.zeros(1, np.uint64)], [], []
    base_e = 0
    for g in gs:
        if g is None:
            gvo.append(gvo[-1])
            continue
        off, tgt, w = g
        n = len(off) - 1
        offs.append(off[1:].astype(np.uint64) + np.uint64(base_e))
        tgts.append(tgt.astype(np.uint32) + np.uint32(gvo[-1]))
        ws.append(w.astype(np.float32))
        base_e += int(off[-1])
        gvo.append(gvo[-1] + n)
    return (np.array(gvo, np.uint64), np.concatenate(offs), np.concatenate(tgts) if tgts else np.zeros(0, np.uint32),
            np.concatenate(ws) if ws else np.zeros(0, np.float32))


MEMBERS = members()
BATCH = concat(MEMBERS)


def dev(off, tgt, w):
    return (torch.from_numpy(np.asarray(off).astype(np.int64)).cuda(),
            torch.from_numpy(np.asarray(tgt).astype(np.int32)).cuda(),
            torch.from_numpy(np.asarray(w).astype(np.float32)).cuda())


def run_batched(gsp, **kw):
    gvo, off, tgt, w = BATCH
    C, q, st = gsp.louvain_batched(gvo, *dev(off, tgt, w), **kw)
    return gvo, C.cpu().numpy().astype(np.int64), q.cpu().numpy(), st


def run_single(gsp, g, **kw):
    off, tgt, w = g
    C, q, st = gsp.louvain(*dev(off, tgt, w), **kw)
    return C.cpu().numpy().astype(np.int64), q


DETERMINISTIC = [
    {"precision": "fp64"},
    {},  # mixed precision, LPP split
    {"split": "bfs", "precision": "fp64"},
    {"split": "lp"},
    {"split_when": "last"},
    {"split": "none"},
    {"waves": 1},
    {"waves": 4, "precision": "fp64"},
    {"max_passes": 1},
    {"max_passes": 2, "aggregation_tolerance": 0.95},
]


@pytest.mark.parametrize("kw", DETERMINISTIC, ids=lambda kw: ",".join(f"{k}={v}" for k, v in kw.items()) or "default")
def test_batched_equals_single_runs(gsp, kw):
    gvo, C, q, st = run_batched(gsp, **kw)
    assert C.shape[0] == int(gvo[-1]) and q.shape[0] == len(MEMBERS)
    for gi, g in enumerate(MEMBERS):
        a, b = int(gvo[gi]), int(gvo[gi + 1])
        if g is None:
            assert a == b and q[gi] == 0.0
            continue
        Cs, qs = run_single(gsp, g, **kw)
        assert np.array_equal(C[a:b], Cs), f"graph {gi}"
        assert q[gi] == pytest.approx(qs, rel=1e-12, abs=1e-15), f"graph {gi}"
    assert st["modularity"] == pytest.approx(float(np.mean(q)), rel=1e-12)


def test_batched_fp64_equals_oracle(gsp):
    gvo, C, q, st = run_batched(gsp, precision="fp64")
    for gi, g in enumerate(MEMBERS):
        if g is None:
            continue
        a, b = int(gvo[gi]), int(gvo[gi + 1])
        off, tgt, w = g
        og = oracle.Graph(off, tgt, w.astype(np.float64))
        Co, ost = oracle.louvain(og, oracle.LouvainOptions(sync=True))
        assert np.array_equal(C[a:b].astype(np.uint32), Co), f"graph {gi}"
        assert q[gi] == pytest.approx(ost["modularity"], rel=1e-9, abs=1e-12)


def test_batched_invariants(gsp):
    for kw in ({}, {"move": "async"}):
        gvo, C, q, st = run_batched(gsp, **kw)
        for gi, g in enumerate(MEMBERS):
            if g is None:
                continue
            a, b = int(gvo[gi]), int(gvo[gi + 1])
            off, tgt, w = g
            og = oracle.Graph(off, tgt, w.astype(np.float64))
            Cg = C[a:b].astype(np.uint32)
            assert q[gi] == pytest.approx(oracle.modularity(og, Cg), rel=1e-9, abs=1e-12)
            assert oracle.disconnected(og, Cg)[0] == 0
            first = np.unique(Cg, return_index=True)[1]
            assert Cg.min() == 0 and np.all(np.diff(first) > 0) and len(first) == Cg.max() + 1


def test_batched_single_graph_equals_louvain(gsp):
    off, tgt, w = MEMBERS[1]
    n = len(off) - 1
    C, q, st = gsp.louvain_batched(np.array([0, n], np.uint64), *dev(off, tgt, w))
    Cs, qs = run_single(gsp, MEMBERS[1])
    assert np.array_equal(C.cpu().numpy(), Cs) and q.cpu().item() == pytest.approx(qs, rel=1e-12)


def test_batched_rejects_bad_input(gsp):
    from paper_2402_11454_gb300._lib import GspError
    off, tgt, w = csr_from_edges(6, [(0, 1), (2, 3), (4, 5)])
    d = dev(off, tgt, w)
    with pytest.raises(GspError):  # edge (2, 3) crosses graphs [0, 3) and [3, 6)
        gsp.louvain_batched(np.array([0, 3, 6], np.uint64), *d)
    with pytest.raises(GspError):  # offsets must end at n
        gsp.louvain_batched(np.array([0, 4], np.uint64), *d)
    with pytest.raises(GspError):  # offsets must not decrease
        gsp.louvain_batched(np.array([0, 4, 2, 6], np.uint64), *d)
    C, q, _ = gsp.louvain_batched(np.array([0, 2, 4, 6], np.uint64), *d)
    assert np.array_equal(C.cpu().numpy(), [0, 0, 0, 0, 0, 0])
    assert np.allclose(q.cpu().numpy(), 0.0)  # one edge per graph: Q = 1/2 - 1/2
