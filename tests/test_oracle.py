"""Pins for the CPU oracle: each check compares the oracle with something
other than itself -- a hand-computed example, a closed form, brute force over
a dense matrix, a library routine (scipy connected components, numpy matmul),
or an invariant of the mathematics.  CPU only."""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

import oracle
from paper_2402_11454_gb300 import graphgen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- helpers
def random_graph(rng, n, p, self_loops=True, weighted=True):
    """Dense symmetric weight matrix -> oracle Graph (weights exact in f32)."""
    A = np.zeros((n, n))
    iu = np.triu_indices(n, 1)
    mask = rng.random(len(iu[0])) < p
    w = (rng.integers(1, 9, size=mask.sum()) / 4.0) if weighted else np.ones(mask.sum())
    A[iu[0][mask], iu[1][mask]] = w
    A = A + A.T
    if self_loops:
        d = rng.random(n) < 0.3
        A[np.arange(n)[d], np.arange(n)[d]] = rng.integers(1, 5, size=d.sum()) / 2.0
    return dense_to_graph(A), A


def dense_to_graph(A):
    n = A.shape[0]
    rows, cols = np.nonzero(A)
    off = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(np.bincount(rows, minlength=n), out=off[1:])
    return oracle.Graph(off, cols.astype(np.uint32), A[rows, cols])


def brute_modularity(A, C):
    """Equation 1 with the null-model term over all ordered vertex pairs:
    Q = 1/2m sum_{i,j} [A_ij - K_i K_j / 2m] delta(C_i, C_j)."""
    K = A.sum(axis=1)
    two_m = K.sum()
    if two_m == 0:
        return 0.0
    same = (C[:, None] == C[None, :])
    return float(((A - np.outer(K, K) / two_m) * same).sum() / two_m)


def ring_of_cliques(k, s):
    n = k * s
    A = np.zeros((n, n))
    for c in range(k):
        idx = np.arange(c * s, (c + 1) * s)
        A[np.ix_(idx, idx)] = 1
        A[idx, idx] = 0
        a, b = c * s, ((c + 1) % k) * s + 1
        A[a, b] = A[b, a] = 1
    return A


# ---------------------------------------------------------- Equation 1 pins
def read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, *vals = line.split()
            out[key] = vals
    return out


def test_golden_path4_modularity_and_delta():
    gd = read_golden("path4_modularity.txt")
    A = np.zeros((4, 4))
    for e in gd["edges"]:
        a, b = map(int, e.split("-"))
        A[a, b] = A[b, a] = 1
    g = dense_to_graph(A)
    C = np.array(list(map(int, gd["membership"])), dtype=np.uint32)
    q = oracle.modularity(g, C)
    assert q == pytest.approx(float(Fraction(gd["q_before"][0])), abs=1e-15)
    K, m = oracle.vertex_weights(g)
    i = int(gd["move_vertex"][0])
    c = int(gd["move_to"][0])
    d = int(C[i])
    Kic = sum(A[i, j] for j in range(4) if j != i and C[j] == c)
    Kid = sum(A[i, j] for j in range(4) if j != i and C[j] == d)
    Sc = K[C == c].sum()
    Sd = K[C == d].sum()
    dq = oracle.delta_modularity(Kic, Kid, K[i], Sc, Sd, m)
    assert dq == pytest.approx(float(Fraction(gd["delta_q"][0])), abs=1e-15)
    C2 = C.copy()
    C2[i] = c
    assert oracle.modularity(g, C2) == pytest.approx(float(Fraction(gd["q_after"][0])), abs=1e-15)


@pytest.mark.parametrize("seed", range(12))
def test_modularity_matches_all_pairs_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 30))
    g, A = random_graph(rng, n, rng.uniform(0.05, 0.6))
    for _ in range(4):
        C = rng.integers(0, max(1, n // 3), size=n).astype(np.uint32)
        assert oracle.modularity(g, C) == pytest.approx(brute_modularity(A, C), abs=1e-12)


def test_modularity_closed_forms():
    rng = np.random.default_rng(7)
    g, A = random_graph(rng, 25, 0.2, self_loops=False)
    K = A.sum(axis=1)
    two_m = K.sum()
    single = np.arange(25, dtype=np.uint32)
    assert oracle.modularity(g, single) == pytest.approx(-((K / two_m) ** 2).sum(), abs=1e-14)
    assert oracle.modularity(g, np.zeros(25, dtype=np.uint32)) == pytest.approx(0.0, abs=1e-14)
    # ring of k cliques K_s joined by single edges, cliques as communities
    for k, s in [(4, 5), (8, 5), (6, 4)]:
        Ar = ring_of_cliques(k, s)
        gr = dense_to_graph(Ar)
        C = (np.arange(k * s) // s).astype(np.uint32)
        m = k * s * (s - 1) / 2 + k
        closed = k * (s * (s - 1) / (2 * m) - ((s * (s - 1) + 2) / (2 * m)) ** 2)
        assert oracle.modularity(gr, C) == pytest.approx(closed, abs=1e-14)


def test_modularity_range_and_edgeless():
    rng = np.random.default_rng(3)
    for _ in range(20):
        n = int(rng.integers(2, 40))
        g, A = random_graph(rng, n, rng.uniform(0.02, 0.9))
        C = rng.integers(0, n, size=n).astype(np.uint32)
        q = oracle.modularity(g, C)
        assert -0.5 - 1e-12 <= q <= 1.0
    empty = oracle.Graph(np.zeros(6, dtype=np.uint64), np.zeros(0, np.uint32), np.zeros(0))
    assert oracle.modularity(empty, np.arange(5, dtype=np.uint32)) == 0.0


# ---------------------------------------------------------- Equation 2 pins
@pytest.mark.parametrize("seed", range(10))
def test_delta_modularity_equals_difference_of_modularity(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(3, 25))
    g, A = random_graph(rng, n, rng.uniform(0.1, 0.6))
    K, m = oracle.vertex_weights(g)
    if m == 0:
        return
    for _ in range(10):
        C = rng.integers(0, max(2, n // 2), size=n).astype(np.uint32)
        i = int(rng.integers(0, n))
        c = int(rng.integers(0, max(2, n // 2)))
        d = int(C[i])
        if c == d:
            continue
        nb = [j for j in range(n) if j != i]
        Kic = sum(A[i, j] for j in nb if C[j] == c)
        Kid = sum(A[i, j] for j in nb if C[j] == d)
        Sc = K[C == c].sum()
        Sd = K[C == d].sum()
        dq = oracle.delta_modularity(Kic, Kid, K[i], Sc, Sd, m)
        C2 = C.copy()
        C2[i] = c
        assert dq == pytest.approx(brute_modularity(A, C2) - brute_modularity(A, C), abs=1e-12)


# ------------------------------------------------------- Algorithm 4 pins
@pytest.mark.parametrize("seed", range(8))
def test_sync_sweep_is_brute_force_argmax(seed):
    """Each vertex of a frozen-state sweep picks the neighbouring community
    whose single move raises Eq.1 the most (ties -> lowest id), and moves only
    on a strictly positive gain; the lower-id rule for singleton pairs holds."""
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(4, 22))
    g, A = random_graph(rng, n, rng.uniform(0.15, 0.5))
    K, m = oracle.vertex_weights(g)
    if m == 0:
        return
    C = rng.integers(0, n, size=n).astype(np.uint32)
    Sigma = np.bincount(C, weights=K, minlength=n)
    size = np.bincount(C, minlength=n)
    choice, best, second = oracle.move_sweep_sync(g, C, K, Sigma, m)
    q0 = brute_modularity(A, C)
    for i in range(n):
        cands = sorted({int(C[j]) for j in range(n) if A[i, j] > 0 and j != i} - {int(C[i])})
        gains = []
        for c in cands:
            C2 = C.copy()
            C2[i] = c
            gains.append((brute_modularity(A, C2) - q0, c))
        expect = int(C[i])
        if gains:
            top = max(gn for gn, _ in gains)
            cbest = min(c for gn, c in gains if abs(gn - top) <= 1e-12)
            assert best[i] == pytest.approx(top, abs=1e-12)
            if top > 1e-12:
                expect = cbest
                d = int(C[i])
                if size[d] == 1 and size[cbest] == 1 and cbest > d:
                    expect = d
            elif top > -1e-12:
                continue  # zero gain: move decided by rounding, exempt
        assert choice[i] == expect, (i, gains)


@pytest.mark.parametrize("seed", range(6))
def test_async_move_telescopes(seed):
    """Asynchronous local moving: each applied move's Eq.2 gain is exact for
    the state it sees, so the gains summed over all iterations equal the
    change of Eq.1; Sigma stays the per-community sum of K."""
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(10, 60))
    g, A = random_graph(rng, n, rng.uniform(0.05, 0.3))
    K, m = oracle.vertex_weights(g)
    C0 = np.arange(n, dtype=np.uint32)
    C, Sigma, li, dq = oracle.move(g, C0, K, K.copy(), m, tau=0.0, max_iterations=50, sync=False)
    assert brute_modularity(A, C) - brute_modularity(A, C0) == pytest.approx(dq.sum(), abs=1e-10)
    assert np.all(dq[:-1] > 0)
    np.testing.assert_allclose(Sigma, np.bincount(C, weights=K, minlength=n), atol=1e-12)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("repeats", [1, 3])
def test_waves_of_one_vertex_equal_the_sequential_loop(seed, repeats):
    """Frozen-state waves with one vertex per wave (waves = |V|, vertex i in
    wave i) see every earlier move, which is the one-thread in-place loop of
    Algorithm 4: both forms must give the same result bit for bit.  A vertex
    never re-marks itself, so repeats of a one-vertex wave find nothing
    to do."""
    rng = np.random.default_rng(350 + seed)
    n = int(rng.integers(10, 80))
    g, A = random_graph(rng, n, rng.uniform(0.05, 0.3))
    K, m = oracle.vertex_weights(g)
    C0 = np.arange(n, dtype=np.uint32)
    Ca, Sa, la, dqa = oracle.move(g, C0, K, K.copy(), m, tau=1e-3, max_iterations=30, sync=False)
    Cw, Sw, lw, dqw = oracle.move(g, C0, K, K.copy(), m, tau=1e-3, max_iterations=30, sync=True,
                                  singleton_rule=False, waves=n, wave_repeats=repeats, wave_hash=False)
    assert la == lw
    np.testing.assert_array_equal(Ca, Cw)
    np.testing.assert_array_equal(Sa, Sw)
    np.testing.assert_array_equal(dqa, dqw)


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("repeats", [2, 3, 5])
def test_repeats_of_one_wave_equal_iterations(seed, repeats):
    """With one wave, the repeats of an iteration are exactly consecutive
    frozen-state iterations: after a pass that visited every unprocessed
    vertex, the next takes those its moves re-marked, as the next iteration
    would.  C and Sigma must agree bit for bit and the gains in total."""
    rng = np.random.default_rng(370 + seed)
    n = int(rng.integers(20, 90))
    g, A = random_graph(rng, n, rng.uniform(0.05, 0.3))
    K, m = oracle.vertex_weights(g)
    C0 = np.arange(n, dtype=np.uint32)
    Cr, Sr, lr, dqr = oracle.move(g, C0, K, K.copy(), m, tau=-np.inf, max_iterations=1, sync=True,
                                  waves=1, wave_repeats=repeats)
    Ci, Si, li, dqi = oracle.move(g, C0, K, K.copy(), m, tau=-np.inf, max_iterations=repeats, sync=True,
                                  waves=1, wave_repeats=1)
    assert lr == 1 and li == repeats
    np.testing.assert_array_equal(Cr, Ci)
    np.testing.assert_array_equal(Sr, Si)
    assert dqr[0] == pytest.approx(dqi.sum(), abs=1e-12)


@pytest.mark.parametrize("repeats", [1, 3])
def test_wave_repeats_keep_sigma_exact(repeats):
    """Every repeat applies moves as Algorithm 4 does: Sigma stays the
    per-community sum of K and the first iteration gains."""
    off, tgt, w = graphgen.rmat(12, 16, seed=9)
    g = oracle.Graph(off, tgt, w)
    n = g.n
    K, m = oracle.vertex_weights(g)
    C, S, li, dq = oracle.move(g, np.arange(n, dtype=np.uint32), K, K.copy(), m, tau=1e-2, sync=True,
                               waves=17, wave_repeats=repeats)
    np.testing.assert_array_equal(S, np.bincount(C, weights=K, minlength=n))
    assert dq[0] > 0


def test_wave_hash_is_a_balanced_bijection():
    """The wave hash (MurmurHash3's 32-bit finaliser) permutes 32-bit ids:
    distinct ids get distinct hashes, and taken mod 17 it spreads
    consecutive ids and ids of one residue class over all waves evenly."""
    ids = np.arange(1 << 16, dtype=np.uint64) * np.uint64(65537) % np.uint64(1 << 32)
    h = oracle.wave_hash(ids)
    assert len(np.unique(h)) == len(ids)
    assert oracle.wave_hash([0])[0] == 0  # the finaliser fixes zero
    for sample in (np.arange(20000), np.arange(20000) * 17, np.arange(20000) * 64):
        cnt = np.bincount(oracle.wave_hash(sample) % 17, minlength=17)
        expect = len(sample) / 17
        assert np.all(np.abs(cnt - expect) < 6 * np.sqrt(expect)), cnt


def test_no_return_rule_ends_two_iteration_cycles():
    """Simultaneous frozen-state decisions can cycle (a vertex leaves a
    community and comes back the next iteration, the claimed gains staying
    above tau): on a 64 x 64 grid one pass then runs to MAX_ITERATIONS.
    Forbidding the return from the fourth iteration on ends every pass early,
    at the one-thread loop's modularity (within 0.002)."""
    off, tgt, w = graphgen.grid(64, 64, seed=3)
    g = oracle.Graph(off, tgt, w)
    _, free = oracle.louvain(g, oracle.LouvainOptions(sync=True, no_return_from=0))
    _, rule = oracle.louvain(g, oracle.LouvainOptions(sync=True, no_return_from=3))
    _, seq = oracle.louvain(g, oracle.LouvainOptions(sync=False))
    assert max(free["iterations"]) == 20
    assert max(rule["iterations"]) < 20
    assert rule["modularity"] >= seq["modularity"] - 0.002


@pytest.mark.parametrize("scale,seed", [(16, 2), (17, 2), (18, 2)])
def test_default_schedule_reaches_the_one_thread_modularity(scale, seed):
    """The frozen-state reading (17 hashed waves, each run 3 times in a
    pass's first iteration) is a schedule for Algorithm 4's parallel loop;
    on R-MAT it must end within 0.002 of the one-thread loop's modularity."""
    off, tgt, w = graphgen.rmat(scale, 16, seed=seed)
    g = oracle.Graph(off, tgt, w)
    _, seq = oracle.louvain(g, oracle.LouvainOptions(sync=False, split="lpp"))
    _, wav = oracle.louvain(g, oracle.LouvainOptions(sync=True, waves=17, wave_repeats=3, split="lpp"))
    assert wav["modularity"] >= seq["modularity"] - 0.002, (wav["modularity"], seq["modularity"])


def test_hashed_waves_on_planted_graphs_with_k_a_multiple_of_17():
    """With waves taken as i mod 17, every community of a planted graph
    whose community count is a multiple of 17 (vertex v in community v mod k)
    falls into a single wave and decides all at once; on graph 2778 of the
    4096-graph batch (26 422 vertices, 17 communities) the run cycles and
    collapses to modularity 0.07 against 0.78 for the one-thread loop.
    Hashed waves keep it within 0.002, with or without the no-return rule."""
    n, k, e, p = graphgen.batch_params(4096, seed=4)
    gi = 2778
    assert k[gi] == 17
    u, v = graphgen.planted_edges(int(n[gi]), int(k[gi]), int(e[gi]), float(p[gi]), graphgen.batch_graph_seed(4, gi))
    off, tgt, w = graphgen.edges_to_csr(int(n[gi]), u, v)
    g = oracle.Graph(off, tgt, w)
    _, seq = oracle.louvain(g, oracle.LouvainOptions(sync=False))
    _, mod = oracle.louvain(g, oracle.LouvainOptions(sync=True, wave_hash=False, no_return_from=0))
    _, hsh = oracle.louvain(g, oracle.LouvainOptions(sync=True, no_return_from=0))
    _, dflt = oracle.louvain(g, oracle.LouvainOptions(sync=True))
    assert mod["modularity"] < seq["modularity"] - 0.1
    assert hsh["modularity"] >= seq["modularity"] - 0.002
    assert dflt["modularity"] >= seq["modularity"] - 0.002


@pytest.mark.parametrize("waves", [1, 4, 16])
def test_waves_keep_sigma_and_gain_positive_first_sweep(waves):
    off, tgt, w = graphgen.planted(n=2000, k=16, mean_degree=12, p_intra=0.8, seed=5)
    g = oracle.Graph(off, tgt, w)
    K, m = oracle.vertex_weights(g)
    C, S, li, dq = oracle.move(g, np.arange(2000, dtype=np.uint32), K, K.copy(), m, tau=1e-2,
                               sync=True, waves=waves)
    np.testing.assert_allclose(S, np.bincount(C, weights=K, minlength=2000), atol=1e-9)
    assert dq[0] > 0


def test_sync_move_keeps_sigma_and_finds_cliques():
    A = ring_of_cliques(8, 5)
    g = dense_to_graph(A)
    K, m = oracle.vertex_weights(g)
    C, Sigma, li, dq = oracle.move(g, np.arange(40, dtype=np.uint32), K, K.copy(), m, tau=0.0,
                                   max_iterations=50, sync=True)
    np.testing.assert_allclose(Sigma, np.bincount(C, weights=K, minlength=40), atol=1e-12)
    # every clique ends in one community
    for c in range(8):
        assert len(set(C[c * 5:(c + 1) * 5].tolist())) == 1


# ------------------------------------------------- Algorithms 2, 3, 6 pins
def scipy_split(A, C):
    """Components of the intra-community subgraph (library routine)."""
    same = C[:, None] == C[None, :]
    B = sp.csr_matrix((A != 0) & same)
    _, lab = connected_components(B, directed=False)
    return lab


@pytest.mark.parametrize("seed", range(10))
def test_split_matches_connected_components(seed):
    rng = np.random.default_rng(400 + seed)
    n = int(rng.integers(2, 80))
    g, A = random_graph(rng, n, rng.uniform(0.01, 0.2))
    C = rng.integers(0, max(1, n // 4), size=n).astype(np.uint32)
    lab = scipy_split(A, C)
    lp, _ = oracle.split_lp(g, C)
    lpp, _ = oracle.split_lp(g, C, prune=True)
    bfs = oracle.split_bfs(g, C)
    np.testing.assert_array_equal(lp, lpp)
    np.testing.assert_array_equal(lp, bfs)
    # same partition as the library, label = smallest vertex of the component
    for comp in np.unique(lab):
        members = np.nonzero(lab == comp)[0]
        assert np.all(lp[members] == members.min())
    cnt, _ = oracle.disconnected(g, lp)
    assert cnt == 0


@pytest.mark.parametrize("seed", range(10))
def test_disconnected_count_matches_library(seed):
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(2, 80))
    g, A = random_graph(rng, n, rng.uniform(0.01, 0.15))
    C = rng.integers(0, max(1, n // 5), size=n).astype(np.uint32)
    lab = scipy_split(A, C)
    expect = sum(1 for c in np.unique(C) if len(np.unique(lab[C == c])) > 1)
    cnt, D = oracle.disconnected(g, C)
    assert cnt == expect
    assert D.sum() == expect


def test_renumber_and_lookup_match_numpy():
    rng = np.random.default_rng(9)
    C = rng.integers(0, 50, size=200).astype(np.uint32)
    R, k = oracle.renumber(C)
    uniq, inv = np.unique(C, return_inverse=True)
    assert k == len(uniq)
    np.testing.assert_array_equal(R, inv)
    top = rng.integers(0, 200, size=500).astype(np.uint32)
    np.testing.assert_array_equal(oracle.lookup(top, R), R[top])


# --------------------------------------------------------- Algorithm 5 pins
@pytest.mark.parametrize("seed", range(8))
def test_aggregate_equals_indicator_product(seed):
    """Super-vertex weights = S^T A S (S the membership indicator), rows
    sorted, total weight kept, and Q(G'', singletons) = Q(G', C')."""
    rng = np.random.default_rng(600 + seed)
    n = int(rng.integers(2, 60))
    g, A = random_graph(rng, n, rng.uniform(0.05, 0.4))
    C = rng.integers(0, max(1, n // 3), size=n).astype(np.uint32)
    Cd, k = oracle.renumber(C)
    S = np.zeros((n, k))
    S[np.arange(n), Cd] = 1
    expect = S.T @ A @ S
    h = oracle.aggregate(g, Cd, k)
    got = np.zeros((k, k))
    for c in range(k):
        a, b = int(h.offsets[c]), int(h.offsets[c + 1])
        row = h.targets[a:b]
        assert np.all(np.diff(row.astype(np.int64)) > 0)
        got[c, row] = h.weights[a:b]
    np.testing.assert_array_equal(got, expect)
    assert h.weights.sum() == A.sum()
    assert oracle.modularity(h, np.arange(k, dtype=np.uint32)) == pytest.approx(
        oracle.modularity(g, Cd), abs=1e-12)


@pytest.mark.parametrize("seed", range(8))
def test_modularity_kept_by_aggregation_under_any_coarser_membership(seed):
    """Eq. 1 of a membership D of the super-vertices on the aggregated graph
    (Algorithm 5) equals Eq. 1 of the looked-up membership D[Cd] on the
    graph that was aggregated: aggregation keeps every weight, self-loops
    included.  (The library takes the final modularity of a run this way, on
    the last level's graph.)  Checked against the all-pairs brute force."""
    rng = np.random.default_rng(650 + seed)
    n = int(rng.integers(2, 60))
    g, A = random_graph(rng, n, rng.uniform(0.05, 0.4))
    C = rng.integers(0, max(1, n // 2), size=n).astype(np.uint32)
    Cd, k = oracle.renumber(C)
    h = oracle.aggregate(g, Cd, k)
    for D in (np.arange(k), rng.integers(0, max(1, k // 3), size=k), np.zeros(k, np.int64)):
        D = D.astype(np.uint32)
        full = oracle.lookup(Cd, D)
        q_full = brute_modularity(A, full)
        assert oracle.modularity(g, full) == pytest.approx(q_full, abs=1e-12)
        assert oracle.modularity(h, D) == pytest.approx(q_full, abs=1e-12)


# --------------------------------------------------------- Algorithm 1 pins
def brute_force_optimum(A):
    """Best Eq.1 value over all set partitions (restricted-growth strings)."""
    n = A.shape[0]
    best = -1.0
    C = [0] * n

    def rec(i, mx):
        nonlocal best
        if i == n:
            best = max(best, brute_modularity(A, np.array(C)))
            return
        for c in range(mx + 2):
            C[i] = c
            rec(i + 1, max(mx, c))

    C[0] = 0
    rec(1, 0)
    return best


@pytest.mark.parametrize("sync", [True, False])
def test_louvain_ring_of_cliques_exact(sync):
    A = ring_of_cliques(8, 5)
    g = dense_to_graph(A)
    C, st = oracle.louvain(g, oracle.LouvainOptions(sync=sync))
    np.testing.assert_array_equal(C, np.arange(40) // 5)
    m = 8 * 10 + 8
    closed = 8 * (20 / (2 * m) - (22 / (2 * m)) ** 2)
    assert st["modularity"] == pytest.approx(closed, abs=1e-14)


@pytest.mark.parametrize("seed", range(4))
def test_louvain_tiny_graphs_against_optimum(seed):
    rng = np.random.default_rng(700 + seed)
    n = 8
    g, A = random_graph(rng, n, 0.35, self_loops=False, weighted=False)
    if A.sum() == 0:
        return
    qopt = brute_force_optimum(A)
    for split in ["bfs", "lp", "none"]:
        C, st = oracle.louvain(g, oracle.LouvainOptions(split=split, tolerance=0.0))
        assert st["modularity"] <= qopt + 1e-12
        assert st["modularity"] == pytest.approx(brute_modularity(A, C.astype(np.int64)), abs=1e-12)


def test_louvain_two_cliques_bridge_reaches_optimum():
    A = np.zeros((8, 8))
    for blk in (range(0, 4), range(4, 8)):
        for a, b in itertools.combinations(blk, 2):
            A[a, b] = A[b, a] = 1
    A[3, 4] = A[4, 3] = 1
    g = dense_to_graph(A)
    C, st = oracle.louvain(g)
    assert st["modularity"] == pytest.approx(brute_force_optimum(A), abs=1e-12)


@pytest.mark.parametrize("split", ["bfs", "lp", "lpp"])
@pytest.mark.parametrize("split_last", [False, True])
def test_louvain_planted_partition(split, split_last):
    off, tgt, w = graphgen.planted(n=3000, k=24, mean_degree=16, p_intra=0.8, seed=11)
    g = oracle.Graph(off, tgt, w)
    truth = graphgen.planted_truth(3000, 24)
    q_truth = oracle.modularity(g, truth)
    C, st = oracle.louvain(g, oracle.LouvainOptions(split=split, split_last=split_last,
                                                    sync=False))
    assert st["modularity"] >= q_truth - 0.005
    assert oracle.disconnected(g, C)[0] == 0
    assert st["final_communities"] == len(np.unique(C))
    # numbering: community ids appear in order of their smallest vertex
    first = np.unique(C, return_index=True)[1]
    assert np.all(np.diff(first) > 0)


def test_louvain_planted_partition_frozen_state_sweeps():
    """Frozen-state sweeps (the parity mode) stay a valid Louvain: a partition
    with no disconnected community and modularity near the planted one."""
    off, tgt, w = graphgen.planted(n=3000, k=24, mean_degree=16, p_intra=0.8, seed=11)
    g = oracle.Graph(off, tgt, w)
    q_truth = oracle.modularity(g, graphgen.planted_truth(3000, 24))
    C, st = oracle.louvain(g, oracle.LouvainOptions(sync=True))
    assert st["modularity"] >= q_truth - 0.03
    assert oracle.disconnected(g, C)[0] == 0


def test_split_pass_removes_disconnection_that_gve_leaves():
    """The disconnection of Fig. 1 arises without a split step (GVE-Louvain);
    with the split pass no returned community is internally disconnected."""
    left = {False: 0, True: 0}
    for seed in range(12, 22):
        off, tgt, w = graphgen.rmat(10, 8, seed=seed)
        g = oracle.Graph(off, tgt, w)
        for sync in (False, True):
            Cn, _ = oracle.louvain(g, oracle.LouvainOptions(split="none", sync=sync))
            Cb, _ = oracle.louvain(g, oracle.LouvainOptions(split="bfs", sync=sync))
            assert oracle.disconnected(g, Cb)[0] == 0
            left[sync] += oracle.disconnected(g, Cn)[0]
    assert left[True] > 0 and left[False] > 0


def test_louvain_edgeless_and_single_vertex():
    g = oracle.Graph(np.zeros(6, dtype=np.uint64), np.zeros(0, np.uint32), np.zeros(0))
    C, st = oracle.louvain(g)
    np.testing.assert_array_equal(C, np.arange(5))
    assert st["modularity"] == 0.0
    g1 = oracle.Graph(np.array([0, 1], dtype=np.uint64), np.array([0], np.uint32), np.array([2.0]))
    C, st = oracle.louvain(g1)
    assert C.tolist() == [0]
