"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer work (split labels, renumbering, lookup, aggregation targets and
offsets, disconnected counts, generated graphs) must match bit for bit;
float64 sums of float32-exact weights (K, m, aggregated weights) must match
exactly too.  Local moving in frozen-state FP64 mode must pick the oracle's
community except where the top two candidates' delta-modularity differ by
less than 1e-12 relative, or the best gain is that close to zero."""
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


def dev(off, tgt, w=None):
    d_off = torch.from_numpy(np.asarray(off).astype(np.int64)).cuda()
    d_tgt = torch.from_numpy(np.asarray(tgt).astype(np.int32)).cuda()
    if w is None:
        return d_off, d_tgt
    return d_off, d_tgt, torch.from_numpy(np.asarray(w)).cuda()


def host(t):
    return t.cpu().numpy()


def graphs():
    """Small inputs spanning the degree classes: planted (config-1 shape),
    R-MAT with hubs above 4096, a weighted grid, and a star."""
    out = {}
    out["planted"] = graphgen.planted(n=10000, k=64, mean_degree=16, p_intra=0.8, seed=1)
    out["rmat14"] = graphgen.rmat(14, 16, seed=2)
    out["grid"] = graphgen.grid(60, 70, seed=3)
    n = 9000
    u = np.zeros(n - 1, dtype=np.uint64)
    v = np.arange(1, n, dtype=np.uint64)
    out["star"] = graphgen.edges_to_csr(n, np.concatenate([u, v[:-1]]), np.concatenate([v, v[1:]]))
    return out


GRAPHS = graphs()


def og(name):
    off, tgt, w = GRAPHS[name]
    return oracle.Graph(off, tgt, w.astype(np.float64))


# --------------------------------------------------------------- generators
def test_device_generators_match_host(gsp):
    off, tgt, w = gsp.gen_planted(n=10000, k=64, mean_degree=16, p_intra=0.8, seed=1)
    ho, ht, hw = GRAPHS["planted"]
    assert np.array_equal(host(off).astype(np.uint64), ho)
    assert np.array_equal(host(tgt).astype(np.uint32), ht)
    assert np.array_equal(host(w), hw)
    off, tgt, w = gsp.gen_rmat(14, 16, seed=2)
    ho, ht, hw = GRAPHS["rmat14"]
    assert np.array_equal(host(off).astype(np.uint64), ho)
    assert np.array_equal(host(tgt).astype(np.uint32), ht)
    off, tgt, w = gsp.gen_grid(60, 70, seed=3)
    ho, ht, hw = GRAPHS["grid"]
    assert np.array_equal(host(off).astype(np.uint64), ho)
    assert np.array_equal(host(tgt).astype(np.uint32), ht)
    assert np.array_equal(host(w), hw)
    n, k, e, p = graphgen.batch_params(10, seed=4, nmax=3000)
    seeds = [graphgen.batch_graph_seed(4, g) for g in range(10)]
    off, tgt, w = gsp.gen_planted_batch(n, k, e, p, seeds)
    voff, eoff, ho, ht, hw = graphgen.batch(10, seed=4, nmax=3000)
    assert np.array_equal(host(off).astype(np.uint64), ho)
    assert np.array_equal(host(tgt).astype(np.uint32), ht)


# ------------------------------------------------------------ weights / Q
@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_vertex_weights_exact(gsp, name):
    off, tgt, w = GRAPHS[name]
    K, m = gsp.vertex_weights(*dev(off, tgt, w))
    Ko, mo = oracle.vertex_weights(og(name))
    assert m == mo
    assert np.array_equal(host(K), Ko)


@pytest.mark.parametrize("name", ["rmat14", "grid"])
def test_vertex_weights_float64_sum_path(gsp, name):
    """Weights scaled by 2^-1010 have no integer unit the library accepts
    (it needs one of at least 2^-1000), so their row sums run in float64;
    those sums stay exact here, so they equal the oracle's on the scaled
    graph and, scaled back, the integer-unit sums of the original weights."""
    off, tgt, w = GRAPHS[name]
    w64 = np.ldexp(w.astype(np.float64), -1010)
    K, m = gsp.vertex_weights(*dev(off, tgt, w64))
    Ko, mo = oracle.vertex_weights(oracle.Graph(off, tgt, w64))
    assert m == mo
    assert np.array_equal(host(K), Ko)
    K1, m1 = gsp.vertex_weights(*dev(off, tgt, w))
    assert np.ldexp(m, 1010) == m1
    assert np.array_equal(np.ldexp(host(K), 1010), host(K1))


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_modularity_matches(gsp, name):
    off, tgt, w = GRAPHS[name]
    n = len(off) - 1
    rng = np.random.default_rng(1)
    d = dev(off, tgt, w)
    for C in (np.arange(n), rng.integers(0, max(1, n // 50), n), np.zeros(n, np.int64),
              np.arange(n) % 64):
        C = C.astype(np.uint32)
        q = gsp.modularity(*d, torch.from_numpy(C.astype(np.int32)).cuda())
        qo = oracle.modularity(og(name), C)
        assert q == pytest.approx(qo, rel=1e-12, abs=1e-14)


# -------------------------------------------------------------- local move
def near_tie(best, second, Ki, m):
    scale = max(abs(best), abs(second) if np.isfinite(second) else 0.0, Ki / m, 1e-300)
    return (np.isfinite(second) and abs(best - second) <= 1e-12 * scale) or abs(best) <= 1e-12 * scale


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("start", ["identity", "random", "coarse"])
def test_sync_sweep_fp64_matches_oracle(gsp, name, start):
    off, tgt, w = GRAPHS[name]
    n = len(off) - 1
    rng = np.random.default_rng(5)
    if start == "identity":
        C = np.arange(n)
    elif start == "random":
        C = rng.integers(0, n, n)
    else:
        C = rng.integers(0, max(2, n // 200), n)
    C = C.astype(np.uint32)
    g = og(name)
    K, m = oracle.vertex_weights(g)
    Sigma = np.bincount(C, weights=K, minlength=n)
    active = (rng.random(n) < 0.9).astype(np.uint8)
    choice_o, best, second = oracle.move_sweep_sync(g, C, K, Sigma, m, active=active)
    d = dev(off, tgt, w)
    choice, dq, moved = gsp.move_sweep(*d, torch.from_numpy(C.astype(np.int32)).cuda(),
                                       torch.from_numpy(K).cuda(), torch.from_numpy(Sigma).cuda(), m,
                                       active=torch.from_numpy(active).cuda(), precision="fp64")
    choice = host(choice).astype(np.uint32)
    diff = np.nonzero(choice != choice_o)[0]
    bad = [i for i in diff if not near_tie(best[i], second[i], K[i], m)]
    assert not bad, (len(bad), bad[:10])
    assert moved == int(np.sum(choice != C))


@pytest.mark.parametrize("name", ["planted", "rmat14", "grid"])
def test_sync_sweep_mixed_precision_close(gsp, name):
    """Float32 K_{i->c} and scores: choices agree with the FP64 oracle except
    where the top two gains are within the float32 error of the terms."""
    off, tgt, w = GRAPHS[name]
    n = len(off) - 1
    C = np.arange(n, dtype=np.uint32) // 3
    g = og(name)
    K, m = oracle.vertex_weights(g)
    Sigma = np.bincount(C, weights=K, minlength=n)
    choice_o, best, second = oracle.move_sweep_sync(g, C, K, Sigma, m)
    choice, _, _ = gsp.move_sweep(*dev(off, tgt, w), torch.from_numpy(C.astype(np.int32)).cuda(),
                                  torch.from_numpy(K).cuda(), torch.from_numpy(Sigma).cuda(), m,
                                  precision="mixed")
    choice = host(choice).astype(np.uint32)
    diff = np.nonzero(choice != choice_o)[0]
    eps = 2.0 ** -22
    for i in diff:
        # float32 terms: K_{i->c} <= K_i and K_i * Sigma_c / 2m <= K_i, so the
        # scaled scores carry an error below ~4 eps K_i; in units of Q, / m
        tol = 8 * eps * K[i] / m
        gap = best[i] - (second[i] if np.isfinite(second[i]) else -np.inf)
        assert gap <= tol or abs(best[i]) <= tol, (i, best[i], second[i], tol)
    assert len(diff) <= max(5, 0.001 * n)


@pytest.mark.parametrize("name", ["planted", "grid", "rmat14"])
@pytest.mark.parametrize("waves,repeats,no_return", [(1, 1, 0), (16, 1, 0), (17, 3, 3), (5, 2, 1)])
def test_sync_local_move_fp64_matches_oracle(gsp, name, waves, repeats, no_return):
    off, tgt, w = GRAPHS[name]
    n = len(off) - 1
    g = og(name)
    K, m = oracle.vertex_weights(g)
    C0 = np.arange(n, dtype=np.uint32)
    Co, So, li_o, _ = oracle.move(g, C0, K, K.copy(), m, tau=1e-4, max_iterations=20, sync=True,
                                  waves=waves, wave_repeats=repeats, no_return_from=no_return)
    dC = torch.from_numpy(C0.astype(np.int32)).cuda()
    dS = torch.from_numpy(K.copy()).cuda()
    li = gsp.local_move(*dev(off, tgt, w), dC, torch.from_numpy(K).cuda(), dS, m, tolerance=1e-4,
                        max_iterations=20, move="sync", waves=waves, wave_repeats=repeats, no_return_from=no_return,
                        precision="fp64")
    assert li == li_o
    assert np.array_equal(host(dC).astype(np.uint32), Co)
    assert np.array_equal(host(dS), So)


# -------------------------------------------------------------------- split
@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("mode", ["lp", "lpp", "bfs", "sv"])
def test_split_bit_exact(gsp, name, mode):
    off, tgt, w = GRAPHS[name]
    n = len(off) - 1
    rng = np.random.default_rng(7)
    g = og(name)
    for C in (rng.integers(0, max(2, n // 20), n), rng.integers(0, 4, n), np.arange(n)):
        C = C.astype(np.uint32)
        lab_o = oracle.split_bfs(g, C)
        lab, k = gsp.split(*dev(off, tgt), torch.from_numpy(C.astype(np.int32)).cuda(), mode=mode)
        assert np.array_equal(host(lab).astype(np.uint32), lab_o)
        assert k == len(np.unique(lab_o))


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_count_disconnected_matches(gsp, name):
    off, tgt, w = GRAPHS[name]
    n = len(off) - 1
    rng = np.random.default_rng(8)
    C = rng.integers(0, max(2, n // 10), n).astype(np.uint32)
    cnt_o, D_o = oracle.disconnected(og(name), C)
    cnt, flags = gsp.count_disconnected(*dev(off, tgt), torch.from_numpy(C.astype(np.int32)).cuda())
    assert cnt == cnt_o
    assert np.array_equal(host(flags), D_o)


def test_renumber_lookup(gsp):
    rng = np.random.default_rng(9)
    C = rng.integers(0, 5000, 100000).astype(np.uint32)
    Cd, k = gsp.renumber(torch.from_numpy(C.astype(np.int32)).cuda())
    R, ko = oracle.renumber(C)
    assert k == ko and np.array_equal(host(Cd).astype(np.uint32), R)
    top = rng.integers(0, 100000, 300000).astype(np.uint32)
    dtop = torch.from_numpy(top.astype(np.int32)).cuda()
    gsp.lookup(dtop, Cd)
    assert np.array_equal(host(dtop).astype(np.uint32), oracle.lookup(top, R))


# -------------------------------------------------------------- aggregate
@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("start", ["identity", "random", "coarse", "few"])
def test_aggregate_bit_exact(gsp, name, start):
    off, tgt, w = GRAPHS[name]
    n = len(off) - 1
    rng = np.random.default_rng(10)
    C = {"identity": np.arange(n), "random": rng.integers(0, n // 2, n),
         "coarse": rng.integers(0, max(2, n // 300), n), "few": rng.integers(0, 3, n)}[start]
    Cd, k = oracle.renumber(C.astype(np.uint32))
    h = oracle.aggregate(og(name), Cd, k)
    o2, t2, w2 = gsp.aggregate(*dev(off, tgt, w), torch.from_numpy(Cd.astype(np.int32)).cuda(), k)
    assert np.array_equal(host(o2).astype(np.uint64), h.offsets)
    assert np.array_equal(host(t2).astype(np.uint32), h.targets)
    assert np.array_equal(host(w2), h.weights)


def test_aggregate_of_aggregate_f64_weights(gsp):
    off, tgt, w = GRAPHS["rmat14"]
    n = len(off) - 1
    C1, k1 = oracle.renumber((np.arange(n) // 7).astype(np.uint32))
    h1 = oracle.aggregate(og("rmat14"), C1, k1)
    C2, k2 = oracle.renumber((np.arange(k1) // 5).astype(np.uint32))
    h2 = oracle.aggregate(h1, C2, k2)
    d1 = dev(h1.offsets, h1.targets, h1.weights)
    o2, t2, w2 = gsp.aggregate(*d1, torch.from_numpy(C2.astype(np.int32)).cuda(), k2)
    assert np.array_equal(host(o2).astype(np.uint64), h2.offsets)
    assert np.array_equal(host(t2).astype(np.uint32), h2.targets)
    assert np.array_equal(host(w2), h2.weights)


@pytest.mark.parametrize("name", ["rmat14", "grid"])
def test_aggregate_float64_table_path(gsp, name):
    """Weights whose common unit is below 2^-1000 take the float64 table path
    instead of the integer one; scaled by 2^-1010 the input weights keep
    every sum exact, so the result still equals the oracle's bit for bit."""
    off, tgt, w = GRAPHS[name]
    n = len(off) - 1
    w64 = np.ldexp(w.astype(np.float64), -1010)
    C, k = oracle.renumber(np.random.default_rng(13).integers(0, max(2, n // 50), n).astype(np.uint32))
    h = oracle.aggregate(oracle.Graph(off, tgt, w64), C, k)
    o2, t2, w2 = gsp.aggregate(*dev(off, tgt, w64), torch.from_numpy(C.astype(np.int32)).cuda(), k)
    assert np.array_equal(host(o2).astype(np.uint64), h.offsets)
    assert np.array_equal(host(t2).astype(np.uint32), h.targets)
    assert np.array_equal(host(w2), h.weights)


# ------------------------------------------------------------- full runs
@pytest.mark.parametrize("split", ["bfs", "lp", "lpp"])
@pytest.mark.parametrize("move", ["sync", "async"])
def test_louvain_planted_against_oracle(gsp, split, move):
    off, tgt, w = GRAPHS["planted"]
    g = og("planted")
    C, q, st = gsp.louvain(*dev(off, tgt, w), split=split, move=move)
    C = host(C).astype(np.uint32)
    q_re = oracle.modularity(g, C)
    assert q == pytest.approx(q_re, rel=1e-9)
    assert oracle.disconnected(g, C)[0] == 0
    _, ost = oracle.louvain(g, oracle.LouvainOptions(split=split, sync=False))
    if move == "sync":  # the paper's in-place loop on a GPU is timing-dependent
        assert q >= ost["modularity"] - 0.002
    first = np.unique(C, return_index=True)[1]
    assert np.all(np.diff(first) > 0) and C.max() + 1 == st["final_communities"]


@pytest.mark.parametrize("name", ["planted", "grid", "rmat14"])
def test_louvain_sync_fp64_equals_oracle(gsp, name):
    """Frozen-state sweeps in FP64 are deterministic: the whole run (moves,
    split, aggregation, passes) reproduces the oracle's membership."""
    off, tgt, w = GRAPHS[name]
    g = og(name)
    C, q, st = gsp.louvain(*dev(off, tgt, w), move="sync", precision="fp64")
    Co, ost = oracle.louvain(g, oracle.LouvainOptions(sync=True))
    assert st["passes"] == ost["passes"]
    assert np.array_equal(host(C).astype(np.uint32), Co)
    assert q == pytest.approx(ost["modularity"], rel=1e-9)


@pytest.mark.parametrize("name", ["planted", "grid", "rmat14"])
@pytest.mark.parametrize("variant", ["split_last", "no_split"])
def test_louvain_split_variants_fp64_equal_oracle(gsp, name, variant):
    """Split Last (Section 4.1, Fig. 3) and no split at all (GVE-Louvain,
    Appendix A.3) reproduce the oracle's runs of the same variant bit for bit
    in frozen-state FP64 mode, including the disconnected communities that
    the unsplit run leaves."""
    off, tgt, w = GRAPHS[name]
    g = og(name)
    if variant == "split_last":
        kw, okw = dict(split="lpp", split_when="last"), dict(split="lp", split_last=True)
    else:
        kw, okw = dict(split="none"), dict(split="none")
    C, q, st = gsp.louvain(*dev(off, tgt, w), move="sync", precision="fp64", count_disconnected=True, **kw)
    Co, ost = oracle.louvain(g, oracle.LouvainOptions(sync=True, **okw))
    assert st["passes"] == ost["passes"]
    assert st["iterations"] == ost["iterations"]
    assert np.array_equal(host(C).astype(np.uint32), Co)
    assert q == pytest.approx(ost["modularity"], rel=1e-9)
    assert st["disconnected"] == oracle.disconnected(g, Co)[0]


@pytest.mark.parametrize("name", ["planted", "grid"])
def test_louvain_hooking_split_equals_oracle(gsp, name):
    """The hooking split (not in the paper) yields the same canonical labels
    as the paper's techniques, so a whole FP64 run still equals the oracle."""
    off, tgt, w = GRAPHS[name]
    g = og(name)
    C, q, st = gsp.louvain(*dev(off, tgt, w), move="sync", precision="fp64", split="sv")
    Co, ost = oracle.louvain(g, oracle.LouvainOptions(sync=True))
    assert np.array_equal(host(C).astype(np.uint32), Co)


@pytest.mark.parametrize("name", ["rmat14", "grid", "star"])
def test_louvain_invariants(gsp, name):
    off, tgt, w = GRAPHS[name]
    g = og(name)
    for kw in ({}, {"split_when": "last"}, {"precision": "fp64"}, {"split": "none"}, {"move": "async"},
               {"waves": 1}, {"split": "lp"}, {"split": "sv"}, {"split": "sv", "split_when": "last"}):
        C, q, st = gsp.louvain(*dev(off, tgt, w), **kw)
        C = host(C).astype(np.uint32)
        assert -0.5 <= q <= 1.0
        assert q == pytest.approx(oracle.modularity(g, C), rel=1e-9, abs=1e-12)
        if kw.get("split", "bfs") != "none":
            assert oracle.disconnected(g, C)[0] == 0


def test_louvain_edge_cases(gsp):
    # single vertex, edgeless graph, self-loop only, two cliques
    for n, edges in ((1, []), (5, []), (3, [(1, 1)]), (8, [(a, b) for a in range(4) for b in range(4) if a < b]
                                                       + [(a, b) for a in range(4, 8) for b in range(4, 8) if a < b])):
        A = np.zeros((n, n))
        for a, b in edges:
            A[a, b] = A[b, a] = 1.0
        rows, cols = np.nonzero(A)
        off = np.zeros(n + 1, dtype=np.uint64)
        np.cumsum(np.bincount(rows, minlength=n), out=off[1:])
        w = A[rows, cols].astype(np.float32)
        C, q, st = gsp.louvain(*dev(off, cols.astype(np.uint32), w))
        C = host(C)
        if not edges or edges == [(1, 1)]:
            assert np.array_equal(C, np.arange(n)) and q == 0.0
        else:
            assert np.array_equal(C, np.repeat([0, 1], 4))
            assert q == pytest.approx(0.5, abs=1e-12)  # 2 * (12/24 - (12/24)^2)


def test_input_check_sparse_rows_hub_and_tail(gsp):
    """The entry check walks the entries in contiguous ranges and finds each
    entry's row by search: a graph whose rows are mostly empty, with a hub
    of 6000 entries and the last entries in the last row, is accepted when
    valid, and a defect at the first entry, inside the hub or at the very last
    entry is caught."""
    from paper_2402_11454_gb300._lib import GspError
    n = 60000
    rng = np.random.default_rng(3)
    nb = rng.choice(np.arange(10, n - 1), size=6000, replace=False)
    u = np.concatenate([np.full(6000, 3), [0, n - 2, 17]]).astype(np.uint64)
    v = np.concatenate([nb, [n - 1, n - 1, 18]]).astype(np.uint64)
    off, tgt, w = graphgen.edges_to_csr(n, u, v)
    C, q, st = gsp.louvain(*dev(off, tgt, w), precision="fp64")
    g = oracle.Graph(off, tgt, w.astype(np.float64))
    assert q == pytest.approx(oracle.modularity(g, C.cpu().numpy()), abs=1e-12)
    hub = 3
    for e, what in ((0, "first"), (int(off[hub]) + 2999, "hub"), (len(tgt) - 1, "last")):
        t2 = tgt.copy()
        t2[e] = n  # target out of range
        with pytest.raises(GspError, match="violations"):
            gsp.louvain(*dev(off, t2, w))
        w2 = w.copy()
        w2[e] = np.nan
        with pytest.raises(GspError, match="violations"):
            gsp.louvain(*dev(off, tgt, w2))
        w3 = w.copy()
        w3[e] = 3.0  # its mirror keeps weight 1
        with pytest.raises(GspError, match="not symmetric"):
            gsp.louvain(*dev(off, tgt, w3))


def test_asymmetric_graph_rejected(gsp):
    """Section 3's graph is undirected (w_ij = w_ji): a CSR entry without its
    mirror, or with a different weight on the mirror, is GSP_ERR_NOT_SYMMETRIC
    (-6), not a silently wrong m.  Duplicate entries stored on both sides and
    self-loops stay valid."""
    from paper_2402_11454_gb300._lib import GspError
    off, tgt, w = GRAPHS["rmat14"]
    n = len(off) - 1
    # drop one direction of the edge stored at entry e (row i)
    rows = np.repeat(np.arange(n), np.diff(off.astype(np.int64)))
    e = int(off[5])
    i, j = int(rows[e]), int(tgt[e])
    assert i != j
    keep = np.ones(len(tgt), bool)
    keep[e] = False
    off2 = off.copy()
    off2[i + 1:] -= 1
    assert off2[i + 1] >= off2[i]
    with pytest.raises(GspError, match="not symmetric"):
        gsp.louvain(*dev(off2, tgt[keep], w[keep]))
    # same structure, one weight changed on one side
    w3 = w.copy()
    w3[e] = 2.0
    with pytest.raises(GspError, match="not symmetric"):
        gsp.louvain(*dev(off, tgt, w3))
    # a long row (hub) loses an entry
    hub = int(np.argmax(np.diff(off.astype(np.int64))))
    assert off[hub + 1] - off[hub] > 64
    e = int(off[hub]) + 7
    keep = np.ones(len(tgt), bool)
    keep[e] = False
    off4 = off.copy()
    off4[hub + 1:] -= 1
    with pytest.raises(GspError, match="not symmetric"):
        gsp.louvain(*dev(off4, tgt[keep], w[keep]))
    # the mirror of the changed weight changed too: symmetric again
    back = np.nonzero((rows == j) & (tgt == i))[0]
    assert len(back) == 1
    w3[back] = 2.0
    C, q, st = gsp.louvain(*dev(off, tgt, w3))
    assert -0.5 <= q <= 1.0
    # duplicates stored on both sides and a self-loop
    u = np.array([0, 0, 1, 2, 3], np.uint64)
    v = np.array([1, 1, 2, 2, 0], np.uint64)
    src = np.concatenate([u, v[u != v]])
    dst = np.concatenate([v, u[u != v]])
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    offd = np.zeros(5, np.uint64)
    np.cumsum(np.bincount(src.astype(np.int64), minlength=4), out=offd[1:])
    C, q, st = gsp.louvain(*dev(offd, dst.astype(np.uint32), np.ones(len(dst), np.float32)))
    assert -0.5 <= q <= 1.0


def test_caller_workspace(gsp):
    """With gsp_opts.workspace the run takes its scratch from the caller's
    buffer: same result as the internal workspace, no growth of the internal
    one, and GSP_ERR_CAPACITY when the buffer is too small."""
    from paper_2402_11454_gb300 import _lib
    from paper_2402_11454_gb300._lib import GspError
    off, tgt, w = GRAPHS["rmat14"]
    d = dev(off, tgt, w)
    C0, q0, st0 = gsp.louvain(*d, precision="fp64")
    need = st0["workspace_bytes"]
    assert need > 0
    before = _lib.load().gsp_workspace_reserved()
    ws = torch.empty(need + 4096, dtype=torch.uint8, device="cuda")
    C1, q1, st1 = gsp.louvain(*d, precision="fp64", workspace=ws)
    assert _lib.load().gsp_workspace_reserved() == before
    assert torch.equal(C0, C1) and q0 == q1
    assert st1["workspace_bytes"] <= ws.numel()
    small = torch.empty(need // 4, dtype=torch.uint8, device="cuda")
    with pytest.raises(GspError, match="capacity"):
        gsp.louvain(*d, precision="fp64", workspace=small)


def test_invalid_graph_rejected(gsp):
    from paper_2402_11454_gb300._lib import GspError
    off = np.array([0, 1, 2], dtype=np.uint64)
    with pytest.raises(GspError):
        gsp.louvain(*dev(off, np.array([1, 5], dtype=np.uint32), np.ones(2, np.float32)))
    with pytest.raises(GspError):
        gsp.louvain(*dev(off, np.array([1, 0], dtype=np.uint32), np.array([1.0, -1.0], np.float32)))
    with pytest.raises(GspError):
        gsp.louvain(*dev(off, np.array([1, 0], dtype=np.uint32), np.array([1.0, np.nan], np.float32)))
