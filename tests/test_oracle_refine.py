"""Pins for the oracle's Leiden refinement (Section 3.5) and the GSP-Leiden
driver: a published generator test vector, brute force that recomputes every
quantity from scratch with exact rationals and takes the gains from Equation
1 (all ordered pairs), hand-built graphs whose outcome follows from the
well-connectedness conditions, the sampling law exp(gain / theta), and
invariants of the refined partition.  CPU only."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy.sparse.csgraph import connected_components
import scipy.sparse as sp

import oracle
from paper_2402_11454_gb300 import graphgen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
GAMMA = 0x9E3779B97F4A7C15


def dense_to_graph(A):
    n = A.shape[0]
    rows, cols = np.nonzero(A)
    off = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(np.bincount(rows, minlength=n), out=off[1:])
    return oracle.Graph(off, cols.astype(np.uint32), A[rows, cols])


def random_graph(rng, n, p, weighted=True):
    A = np.zeros((n, n))
    iu = np.triu_indices(n, 1)
    mask = rng.random(len(iu[0])) < p
    w = (rng.integers(1, 9, size=mask.sum()) / 4.0) if weighted else np.ones(mask.sum())
    A[iu[0][mask], iu[1][mask]] = w
    A = A + A.T
    d = rng.random(n) < 0.2
    A[np.arange(n)[d], np.arange(n)[d]] = rng.integers(1, 5, size=d.sum()) / 2.0
    return A


# ------------------------------------------------------------ generator
def test_splitmix64_published_sequence():
    vals = {}
    with open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = int(v)
    x = 1234567
    for i in range(5):
        assert oracle.splitmix64(x) == vals["out%d" % i]
        x = (x + GAMMA) % (1 << 64)


def test_refine_uniform_is_open_unit_interval_and_decorrelated():
    u = np.array([oracle.refine_uniform(7, p, v, c) for p in range(3) for v in range(40) for c in range(25)])
    assert np.all((u > 0) & (u < 1))
    assert len(np.unique(u)) == len(u)
    assert abs(u.mean() - 0.5) < 0.02 and abs(u.var() - 1 / 12) < 0.01
    # seeds and passes give different streams
    assert oracle.refine_uniform(7, 0, 3, 4) != oracle.refine_uniform(8, 0, 3, 4)
    assert oracle.refine_uniform(7, 0, 3, 4) != oracle.refine_uniform(7, 1, 3, 4)


# -------------------------------------------------- brute-force refinement
def _q_exact(A, K, two_m, labels):
    """Equation 1 over all ordered pairs, in exact rationals."""
    n = len(A)
    q = Fraction(0)
    for i in range(n):
        for j in range(n):
            if labels[i] == labels[j]:
                q += A[i][j] - K[i] * K[j] / two_m
    return q / two_m


def brute_refine(Aw, B, theta, seed, pass_index, waves, wave_hash):
    """The refinement recomputed from scratch at the start of every wave:
    E, S and the gains straight from the matrix (gains as m times the change
    of Equation 1), no incremental bookkeeping."""
    n = len(Aw)
    A = [[Fraction(x).limit_denominator(1 << 20) for x in row] for row in Aw]
    K = [sum(row) for row in A]
    two_m = sum(K)
    m = two_m / 2
    R = list(range(n))
    if two_m == 0:
        return R
    wave = [((int(oracle.wave_hash([i])[0]) if wave_hash else i) % waves) for i in range(n)]
    for wv in range(waves):
        members = [v for v in range(n) if wave[v] == wv]
        q0 = _q_exact(A, K, two_m, R)
        T = {}
        for v in members:
            T[v] = v
            if sum(1 for x in R if x == R[v]) != 1:
                continue
            b = B[v]
            Sb = sum(K[u] for u in range(n) if B[u] == b)
            Ev = sum(A[v][u] for u in range(n) if u != v and B[u] == b)
            if not Ev >= K[v] * (Sb - K[v]) / two_m:
                continue
            cands = sorted({R[u] for u in range(n) if u != v and B[u] == b and A[v][u] != 0})
            best, bc = None, v
            if theta > 0:
                best = -math.log(-math.log(oracle.refine_uniform(seed, pass_index, v, v)))
            for c in cands:
                mem = [u for u in range(n) if R[u] == c]
                Sc = sum(K[u] for u in mem)
                Ec = sum(A[x][u] for x in mem for u in range(n) if B[u] == b and R[u] != c)
                if not Ec >= Sc * (Sb - Sc) / two_m:
                    continue
                lab = list(R)
                lab[v] = c
                gain = m * (_q_exact(A, K, two_m, lab) - q0)
                if theta > 0:
                    if gain < 0:
                        continue
                    s = float(gain) / theta - math.log(-math.log(oracle.refine_uniform(seed, pass_index, v, c)))
                else:
                    if not gain > 0:
                        continue
                    s = gain
                if best is None or s > best or (s == best and c < bc):
                    best, bc = s, c
            T[v] = bc
        targeted = {T[v] for v in members if T[v] != v}
        for v in members:
            if T[v] != v and v not in targeted:
                R[v] = T[v]
    return R


def _bound(rng, A, k):
    """A bound membership: random labels, then each label split into its
    connected pieces (as the split step leaves it)."""
    n = len(A)
    lab = rng.integers(0, k, n)
    same = (lab[:, None] == lab[None, :]) & (A != 0)
    _, comp = connected_components(sp.csr_matrix(same.astype(float)), directed=False)
    return comp.astype(np.uint32)


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("theta", [0.0, 0.01, 0.7])
@pytest.mark.parametrize("waves,wave_hash", [(None, False), (1, False), (2, False), (3, False), (5, True)])
def test_refine_matches_brute_force(seed, theta, waves, wave_hash):
    """Sequential (one vertex per wave) and wave forms; bound communities
    from 2 or 3 random labels, so that a wave often has several joiners of
    one target that are adjacent to each other."""
    rng = np.random.default_rng(900 + seed)
    n = 22
    A = random_graph(rng, n, 0.25 + 0.15 * (seed % 3 == 0), weighted=(seed % 2 == 0))
    B = _bound(rng, A, 2 + seed % 2)
    W = n if waves is None else waves
    g = dense_to_graph(A)
    R, moves = oracle.refine(g, B, theta=theta, seed=seed, pass_index=seed % 3, waves=W, wave_hash=wave_hash)
    R_bf = brute_refine(A, B.tolist(), theta, seed, seed % 3, W, wave_hash)
    assert R.tolist() == R_bf
    assert moves == sum(1 for v in range(n) if R_bf[v] != v)


def test_refine_brute_force_sees_moves():
    """The cases above are not vacuous: refinement merges vertices."""
    moved = 0
    for seed in range(6):
        rng = np.random.default_rng(900 + seed)
        A = random_graph(rng, 22, 0.25, weighted=(seed % 2 == 0))
        B = _bound(rng, A, 3)
        moved += oracle.refine(dense_to_graph(A), B, theta=0.0, waves=22, wave_hash=False)[1]
    assert moved > 20


# ------------------------------------------------------ hand-built cases
def _graph(n, edges):
    A = np.zeros((n, n))
    for a, b, w in edges:
        A[a, b] = A[b, a] = w
    return A


def test_vertex_not_well_connected_stays_alone():
    """Vertex 0 has one unit edge into its bound community {0..6} (a clique on
    1..6) and two edges out of it.  E(0, b-0) = 1 < K_0 (S_b - K_0) / 2m =
    3 * 31 / 38, so it stays a singleton although joining {1} would gain
    1 - 3 * 6 / 38 > 0.  With w(0,1) = 6 the condition holds with equality
    (6 >= 8 * 36 / 48) and vertex 0 joins vertex 1."""
    def build(w01):
        edges = [(0, 1, w01), (0, 7, 1), (0, 8, 1), (7, 8, 1)]
        edges += [(a, b, 1) for a in range(1, 7) for b in range(a + 1, 7)]
        return _graph(9, edges)
    B = np.array([0] * 7 + [1] * 2, dtype=np.uint32)
    R, _ = oracle.refine(dense_to_graph(build(1)), B, theta=0.0, waves=9, wave_hash=False)
    assert R[0] == 0
    R, _ = oracle.refine(dense_to_graph(build(6)), B, theta=0.0, waves=9, wave_hash=False)
    assert R[0] == 1


def test_candidate_not_well_connected_is_skipped():
    """Vertex 1 puts 10 of its 13 units outside the bound community {0..4}:
    E({1}, b-{1}) = 3 < 13 * 11 / 36, so vertex 0 joins {2} (gain 1 - 4*3/36)
    instead of the larger-gain {1} (3 - 4*13/36)."""
    A = _graph(7, [(0, 1, 3), (0, 2, 1), (2, 3, 1), (3, 4, 1), (2, 4, 1), (1, 5, 10), (5, 6, 1)])
    B = np.array([0, 0, 0, 0, 0, 1, 1], dtype=np.uint32)
    R, _ = oracle.refine(dense_to_graph(A), B, theta=0.0, waves=7, wave_hash=False)
    assert R[0] == 2


def test_targeted_singletons_stay_within_a_wave():
    """Path 0-1-2 in one wave: 0 and 2 pick {1}, 1 picks {0} (tie to the lower
    id); 0 and 1 are targets of other movers and stay, 2 joins 1."""
    A = _graph(3, [(0, 1, 1), (1, 2, 1)])
    R, moves = oracle.refine(dense_to_graph(A), np.zeros(3, np.uint32), theta=0.0, waves=1, wave_hash=False)
    assert R.tolist() == [0, 1, 1] and moves == 1


def test_disjoint_cliques_refine_to_the_cliques():
    """Bound communities that are cliques (joined by single edges) refine to
    exactly those cliques, sequentially and in hashed waves of the default
    count: each joiner prefers the largest partial clique it touches."""
    k, s = 6, 7
    A = np.zeros((k * s, k * s))
    for c in range(k):
        idx = np.arange(c * s, (c + 1) * s)
        A[np.ix_(idx, idx)] = 1
        A[idx, idx] = 0
        a, b = c * s, ((c + 1) % k) * s + 1
        A[a, b] = A[b, a] = 1
    B = (np.arange(k * s) // s).astype(np.uint32)
    g = dense_to_graph(A)
    for W, h in ((k * s, False),):
        for theta in (0.0, 0.01):
            R, _ = oracle.refine(g, B, theta=theta, waves=W, wave_hash=h)
            assert len(np.unique(R)) == k
            assert np.all(B[R] == B)


def test_theta_sampling_law():
    """Vertex 0 (first in order) chooses among staying (gain 0) and joining
    {1}, {2}, {3} (gains 1 - 36/42, 2 - 42/42, 3 - 48/42) with probability
    proportional to exp(gain / theta); over 4000 seeds the frequencies agree
    within five standard deviations."""
    A = _graph(5, [(0, 1, 1), (0, 2, 2), (0, 3, 3), (1, 4, 5), (2, 4, 5), (3, 4, 5)])
    g = dense_to_graph(A)
    B = np.zeros(5, np.uint32)
    theta = 0.5
    gains = np.array([0.0, 1 - 36 / 42, 2 - 42 / 42, 3 - 48 / 42])
    p = np.exp(gains / theta)
    p /= p.sum()
    N = 4000
    counts = np.zeros(4)
    for s in range(N):
        R, _ = oracle.refine(g, B, theta=theta, seed=s, waves=5, wave_hash=False)
        counts[R[0]] += 1
    freq = counts / N
    sd = np.sqrt(p * (1 - p) / N)
    assert np.all(np.abs(freq - p) < 5 * sd), (freq, p)


# -------------------------------------------- invariants on larger graphs
@pytest.mark.parametrize("theta", [0.0, 0.01])
def test_refined_partition_is_connected_and_nested(theta):
    off, tgt, w = graphgen.rmat(12, 8, seed=3)
    g = oracle.Graph(off, tgt, w)
    K, m = oracle.vertex_weights(g)
    C, _, _, _ = oracle.move(g, np.arange(g.n), K, K.copy(), m, 1e-2, waves=17, wave_repeats=3, no_return_from=3)
    B = oracle.split_bfs(g, C)
    R, moves = oracle.refine(g, B, theta=theta, seed=5, waves=17)
    assert moves > 0
    assert np.all(B[R] == B)                        # refined communities nest in the bound ones
    assert np.all(R[R] == R)                        # every target kept its own member
    assert oracle.disconnected(g, R)[0] == 0        # joiners always touch their target
    assert len(np.unique(R)) < g.n


# ------------------------------------------------------ GSP-Leiden runs
def test_leiden_ring_of_cliques_exact():
    k, s = 8, 5
    A = np.zeros((k * s, k * s))
    for c in range(k):
        idx = np.arange(c * s, (c + 1) * s)
        A[np.ix_(idx, idx)] = 1
        A[idx, idx] = 0
        a, b = c * s, ((c + 1) % k) * s + 1
        A[a, b] = A[b, a] = 1
    C, st = oracle.louvain(dense_to_graph(A), oracle.LouvainOptions(refine=True))
    np.testing.assert_array_equal(C, np.arange(k * s) // s)


@pytest.mark.parametrize("theta", [0.0, 0.01])
def test_gsp_leiden_planted_partition(theta):
    off, tgt, w = graphgen.planted(n=3000, k=24, mean_degree=16, p_intra=0.8, seed=11)
    g = oracle.Graph(off, tgt, w)
    q_truth = oracle.modularity(g, graphgen.planted_truth(3000, 24))
    C, st = oracle.louvain(g, oracle.LouvainOptions(refine=True, refine_theta=theta))
    assert st["modularity"] >= q_truth - 0.03
    assert st["modularity"] == pytest.approx(oracle.modularity(g, C), abs=1e-12)
    assert oracle.disconnected(g, C)[0] == 0
    first = np.unique(C, return_index=True)[1]
    assert np.all(np.diff(first) > 0)


def test_gsp_leiden_on_rmat_keeps_quality_and_connectivity():
    """On R-MAT the refined run stays within 0.01 of the Louvain run's
    modularity, and with the split no community is disconnected."""
    off, tgt, w = graphgen.rmat(13, 8, seed=4)
    g = oracle.Graph(off, tgt, w)
    _, st0 = oracle.louvain(g)
    C, st1 = oracle.louvain(g, oracle.LouvainOptions(refine=True))
    assert st1["modularity"] >= st0["modularity"] - 0.01
    assert oracle.disconnected(g, C)[0] == 0


def test_leiden_edgeless_and_single_vertex():
    o = oracle.LouvainOptions(refine=True)
    g = oracle.Graph(np.zeros(6, dtype=np.uint64), np.zeros(0, np.uint32), np.zeros(0))
    C, st = oracle.louvain(g, o)
    np.testing.assert_array_equal(C, np.arange(5))
    g1 = oracle.Graph(np.array([0, 1], dtype=np.uint64), np.array([0], np.uint32), np.array([2.0]))
    assert oracle.louvain(g1, o)[0].tolist() == [0]
