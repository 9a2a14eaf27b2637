"""Host generators: structure of the synthetic inputs (symmetric, no
self-loops, no duplicate pairs) and their sizes.  CPU only."""
import numpy as np

from paper_2402_11454_gb300 import graphgen


def check_csr(off, tgt, w, n):
    assert len(off) == n + 1 and off[0] == 0 and off[-1] == len(tgt) == len(w)
    src = np.repeat(np.arange(n, dtype=np.uint64), np.diff(off).astype(np.int64))
    assert np.all(src != tgt)
    key = (src << np.uint64(32)) | tgt.astype(np.uint64)
    assert np.all(np.diff(key.astype(np.float64)) > 0) or np.all(key[1:] > key[:-1])
    rkey = (tgt.astype(np.uint64) << np.uint64(32)) | src
    assert np.array_equal(np.sort(key), np.sort(rkey))
    # weights symmetric
    order = np.argsort(rkey)
    assert np.array_equal(w[np.argsort(key)], w[order])
    assert np.all(w > 0)


def test_planted_config_size():
    off, tgt, w = graphgen.planted(n=10000, k=64, mean_degree=16, p_intra=0.8, seed=1)
    check_csr(off, tgt, w, 10000)
    assert 150_000 < len(tgt) <= 160_000
    truth = graphgen.planted_truth(10000, 64)
    src = np.repeat(np.arange(10000), np.diff(off).astype(np.int64))
    intra = np.mean(truth[src] == truth[tgt])
    assert 0.78 < intra < 0.83


def test_rmat_small():
    off, tgt, w = graphgen.rmat(10, 8, seed=3)
    check_csr(off, tgt, w, 1024)
    deg = np.diff(off)
    assert deg.max() > 10 * np.median(deg[deg > 0])


def test_grid_small():
    off, tgt, w = graphgen.grid(40, 50, seed=3)
    check_csr(off, tgt, w, 2000)
    assert np.all((w >= 1.0) & (w < 10.0))
    E = 40 * 49 + 39 * 50
    assert 0.9 * E < len(tgt) / 2 < 0.97 * E


def test_batch_small():
    voff, eoff, off, tgt, w = graphgen.batch(num_graphs=12, seed=4, nmax=2000)
    n = int(voff[-1])
    check_csr(off, tgt, w, n)
    src = np.repeat(np.arange(n), np.diff(off).astype(np.int64))
    g_src = np.searchsorted(voff, src, side="right") - 1
    g_tgt = np.searchsorted(voff, tgt, side="right") - 1
    assert np.all(g_src == g_tgt)


def test_rng_is_counter_based():
    key = graphgen.stream_key(5, 1)
    ctr = np.arange(10, dtype=np.uint64)
    a = graphgen.rand_u64(key, ctr)
    b = np.array([graphgen.mix64_int(key + (int(c) + 1) * graphgen.GAMMA) for c in range(10)],
                 dtype=np.uint64)
    assert np.array_equal(a, b)
