"""Parity of the GPU refinement (Section 3.5, the GSP-Leiden variant) with
the oracle, through the C ABI.

The refined membership is integer work decided by float64 scores whose sums
are exact for these inputs (integer and float32-exact weights), so the GPU
must reproduce the oracle's refined partition bit for bit in every wave
count, for the greedy limit and for random choices (the Gumbel draws use the
same counter-based generator on both sides; the logarithms may differ in the
last bit, which could only matter at a near-tie of two noisy scores).  Whole
GSP-Leiden runs in frozen-state FP64 mode must equal the oracle's."""
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


def dev(off, tgt, w, wdtype=None):
    d_off = torch.from_numpy(np.asarray(off).astype(np.int64)).cuda()
    d_tgt = torch.from_numpy(np.asarray(tgt).astype(np.int32)).cuda()
    w = np.asarray(w) if wdtype is None else np.asarray(w).astype(wdtype)
    return d_off, d_tgt, torch.from_numpy(w).cuda()


def star_with_ring(n):
    """A hub joined to every other vertex (degree n - 1, beyond the 8192 edges
    of the shared-memory tables), the others in a path."""
    u = np.zeros(n - 1, dtype=np.uint64)
    v = np.arange(1, n, dtype=np.uint64)
    return graphgen.edges_to_csr(n, np.concatenate([u, v[:-1]]), np.concatenate([v, v[1:]]))


def graphs():
    """Inputs spanning the degree classes: planted (small degrees), R-MAT 14
    and 16 (warp, block and 16384-slot classes), a weighted grid, and a hub
    of 11999 edges (the pool class)."""
    return {
        "planted": graphgen.planted(n=10000, k=64, mean_degree=16, p_intra=0.8, seed=1),
        "rmat14": graphgen.rmat(14, 16, seed=2),
        "rmat16": graphgen.rmat(16, 16, seed=5),
        "grid": graphgen.grid(60, 70, seed=3),
        "hub": star_with_ring(12000),
    }


GRAPHS = graphs()


def og(name):
    off, tgt, w = GRAPHS[name]
    return oracle.Graph(off, tgt, w.astype(np.float64))


def bound_membership(name):
    """Local moving (the default frozen-state schedule) and the split, by the
    oracle: the input the refinement gets inside a run."""
    g = og(name)
    if name == "hub":
        # one bound community: the hub's table then holds every refined community
        return np.zeros(g.n, dtype=np.uint32)
    K, m = oracle.vertex_weights(g)
    C, _, _, _ = oracle.move(g, np.arange(g.n), K, K.copy(), m, 1e-2, waves=17, wave_repeats=3, no_return_from=3)
    return oracle.split_bfs(g, C)


BOUND = {name: bound_membership(name) for name in GRAPHS}


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("theta,seed", [(0.0, 0), (0.01, 3), (0.7, 11)])
@pytest.mark.parametrize("waves", [1, 5, 17])
def test_refine_matches_oracle(gsp, name, theta, seed, waves):
    off, tgt, w = GRAPHS[name]
    B = BOUND[name]
    R, moves = gsp.refine(*dev(off, tgt, w), torch.from_numpy(B.astype(np.int32)).cuda(), theta=theta, seed=seed,
                          pass_index=2, waves=waves)
    Ro, mo = oracle.refine(og(name), B, theta=theta, seed=seed, pass_index=2, waves=waves, wave_hash=True)
    R = R.cpu().numpy().astype(np.uint32)
    assert moves == mo
    assert mo > 0
    np.testing.assert_array_equal(R, Ro)


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("theta", [0.0, 0.01])
def test_refine_mixed_precision_invariants(gsp, name, theta):
    """Float32 sums and scores (the default mode): the refined partition
    nests in the bound one, every target keeps its own member, refined
    communities are connected, and the number of merges stays within 2 %
    of the float64 evaluation's."""
    off, tgt, w = GRAPHS[name]
    B = BOUND[name]
    R, moves = gsp.refine(*dev(off, tgt, w), torch.from_numpy(B.astype(np.int32)).cuda(), theta=theta, seed=3,
                          waves=17, precision="mixed")
    R = R.cpu().numpy().astype(np.uint32)
    Ro, mo = oracle.refine(og(name), B, theta=theta, seed=3, waves=17, wave_hash=True)
    assert np.all(B[R] == B)
    assert np.all(R[R] == R)
    assert oracle.disconnected(og(name), R)[0] == 0
    assert moves == int((R != np.arange(len(R))).sum())
    assert abs(moves - mo) <= max(2, 0.02 * mo)


def test_refine_float64_weights_and_default_waves(gsp):
    """float64 weights take the same path; waves = 0 is 17."""
    off, tgt, w = GRAPHS["grid"]
    B = BOUND["grid"]
    R, moves = gsp.refine(*dev(off, tgt, w, np.float64), torch.from_numpy(B.astype(np.int32)).cuda(), theta=0.01,
                          seed=9, waves=0)
    Ro, mo = oracle.refine(og("grid"), B, theta=0.01, seed=9, waves=17, wave_hash=True)
    np.testing.assert_array_equal(R.cpu().numpy().astype(np.uint32), Ro)
    assert moves == mo


def test_refine_edgeless_and_isolated_vertices(gsp):
    """No edges: every vertex stays alone.  Isolated vertices beside a
    path stay alone too (no candidate); in one wave the path's vertices pick
    each other in pairs (0-1, 2-3), every one is targeted and all stay; in 17
    waves the pairs merge."""
    off = torch.zeros(5, dtype=torch.int64, device="cuda")
    tgt = torch.zeros(0, dtype=torch.int32, device="cuda")
    w = torch.zeros(0, dtype=torch.float32, device="cuda")
    R, moves = gsp.refine(off, tgt, w, torch.zeros(4, dtype=torch.int32, device="cuda"), theta=0.0)
    assert R.cpu().tolist() == [0, 1, 2, 3] and moves == 0
    n = 8
    off, tgt, w = graphgen.edges_to_csr(n, np.array([0, 1, 2], np.uint64), np.array([1, 2, 3], np.uint64))
    B = np.zeros(n, np.uint32)
    for waves, expect in ((1, [0, 1, 2, 3]), (17, [1, 1, 3, 3])):
        R, moves = gsp.refine(*dev(off, tgt, w), torch.zeros(n, dtype=torch.int32, device="cuda"), theta=0.0,
                              waves=waves)
        Ro, mo = oracle.refine(oracle.Graph(off, tgt, w.astype(np.float64)), B, theta=0.0, waves=waves,
                               wave_hash=True)
        np.testing.assert_array_equal(R.cpu().numpy().astype(np.uint32), Ro)
        assert moves == mo
        assert R.cpu().tolist() == expect + [4, 5, 6, 7]


def test_refine_rejects_bad_arguments(gsp):
    off, tgt, w = GRAPHS["planted"]
    B = BOUND["planted"].astype(np.int64)
    bad = B.copy()
    bad[3] = len(B) + 5
    with pytest.raises(RuntimeError, match="bound membership"):
        gsp.refine(*dev(off, tgt, w), torch.from_numpy(bad.astype(np.int32)).cuda())
    with pytest.raises(RuntimeError, match="theta"):
        gsp.refine(*dev(off, tgt, w), torch.from_numpy(B.astype(np.int32)).cuda(), theta=-1.0)


@pytest.mark.parametrize("name", ["planted", "rmat14", "grid"])
@pytest.mark.parametrize("theta,seed", [(0.0, 0), (0.01, 4)])
def test_gsp_leiden_fp64_equals_oracle(gsp, name, theta, seed):
    """The whole GSP-Leiden run (local moving, split, refinement, aggregation
    of the refined partition, the next pass from the bound communities) in
    frozen-state FP64 mode reproduces the oracle's run bit for bit."""
    off, tgt, w = GRAPHS[name]
    g = og(name)
    C, q, st = gsp.louvain(*dev(off, tgt, w), move="sync", precision="fp64", refine=True, refine_theta=theta,
                           seed=seed, count_disconnected=True)
    Co, ost = oracle.louvain(g, oracle.LouvainOptions(sync=True, refine=True, refine_theta=theta, seed=seed))
    assert st["passes"] == ost["passes"]
    assert st["iterations"] == ost["iterations"]
    np.testing.assert_array_equal(C.cpu().numpy().astype(np.uint32), Co)
    assert q == pytest.approx(ost["modularity"], rel=1e-9)
    assert st["disconnected"] == 0
    assert any(r > 0 for r in st["refined"])


@pytest.mark.parametrize("name", ["planted", "rmat16", "grid"])
def test_gsp_leiden_default_mode_quality(gsp, name):
    """The default (mixed-precision) GSP-Leiden run stays within 0.002 of the
    oracle's GSP-Leiden modularity and leaves no community disconnected."""
    off, tgt, w = GRAPHS[name]
    g = og(name)
    C, q, st = gsp.louvain(*dev(off, tgt, w), refine=True, count_disconnected=True)
    _, ost = oracle.louvain(g, oracle.LouvainOptions(refine=True))
    assert q >= ost["modularity"] - 0.002
    assert st["disconnected"] == 0
    assert q == pytest.approx(oracle.modularity(g, C.cpu().numpy().astype(np.uint32)), rel=1e-9)


def _concat(graphs):
    offs, tgts, ws, gvo = [], [], [], [0]
    base_v, base_e = 0, 0
    for off, tgt, w in graphs:
        off = np.asarray(off, dtype=np.int64)
        offs.append(off[:-1] + base_e)
        tgts.append(np.asarray(tgt, dtype=np.int64) + base_v)
        ws.append(np.asarray(w))
        base_v += len(off) - 1
        base_e += int(off[-1])
        gvo.append(base_v)
    off = np.concatenate(offs + [np.array([base_e], dtype=np.int64)])
    return off, np.concatenate(tgts), np.concatenate(ws), np.array(gvo, dtype=np.uint64)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batched_gsp_leiden_equals_solo_runs(gsp, precision):
    """In a batch each graph refines as it does alone (its own 2m, draws keyed
    by its own vertex indices, waves by index within it): the batched
    GSP-Leiden membership and modularity of every graph equal its solo run,
    and in FP64 the oracle's."""
    graphs = [graphgen.planted(n=3000 + 997 * k, k=8 + 5 * k, mean_degree=10 + 3 * k, p_intra=0.75, seed=20 + k)
              for k in range(4)] + [graphgen.rmat(12, 8, seed=7), graphgen.grid(30, 40, seed=5)]
    off, tgt, w, gvo = _concat(graphs)
    kw = dict(move="sync", precision=precision, refine=True, refine_theta=0.01, seed=3)
    C, qg, st = gsp.louvain_batched(gvo, *dev(off, tgt, w), **kw)
    C = C.cpu().numpy()
    qg = qg.cpu().numpy()
    assert any(r > 0 for r in st["refined"])
    for k, (o1, t1, w1) in enumerate(graphs):
        Cs, qs, _ = gsp.louvain(*dev(o1, t1, w1), **kw)
        np.testing.assert_array_equal(C[gvo[k]:gvo[k + 1]], Cs.cpu().numpy())
        assert qg[k] == pytest.approx(qs, rel=1e-9)
        if precision == "fp64":
            Co, ost = oracle.louvain(oracle.Graph(o1, t1, w1.astype(np.float64)),
                                     oracle.LouvainOptions(sync=True, refine=True, refine_theta=0.01, seed=3))
            np.testing.assert_array_equal(Cs.cpu().numpy().astype(np.uint32), Co)


@pytest.mark.parametrize("name", ["planted", "rmat14"])
@pytest.mark.parametrize("variant", ["split_last", "no_split", "hooking"])
def test_gsp_leiden_split_variants_fp64_equal_oracle(gsp, name, variant):
    """Refinement combined with Split Last (Section 4.1), with no split at all
    (GVE-Louvain's passes plus the refinement) and with the hooking split
    reproduces the oracle's run of the same variant in frozen-state FP64
    mode, the disconnected-community count included."""
    off, tgt, w = GRAPHS[name]
    g = og(name)
    kw, okw = {"split_last": (dict(split="lpp", split_when="last"), dict(split="lp", split_last=True)),
               "no_split": (dict(split="none"), dict(split="none")),
               "hooking": (dict(split="sv"), dict(split="bfs"))}[variant]
    C, q, st = gsp.louvain(*dev(off, tgt, w), move="sync", precision="fp64", refine=True, refine_theta=0.01, seed=2,
                           count_disconnected=True, **kw)
    Co, ost = oracle.louvain(g, oracle.LouvainOptions(sync=True, refine=True, refine_theta=0.01, seed=2, **okw))
    assert st["passes"] == ost["passes"]
    assert st["iterations"] == ost["iterations"]
    np.testing.assert_array_equal(C.cpu().numpy().astype(np.uint32), Co)
    assert q == pytest.approx(ost["modularity"], rel=1e-9)
    assert st["disconnected"] == oracle.disconnected(g, Co)[0]
