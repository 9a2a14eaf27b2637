"""The learned pruning predictor's kernels against the FP64 oracle
(oracle/mlp.py), its traces, and what the trained network gains over the
plain method.

Tolerances: the kernels round the weights to bfloat16 exactly as the oracle
does and then accumulate in float32, so P(move) differs from the oracle by
float32 rounding of ~40-term dot products (|dp| <= 1e-5); the gradient sums
per-row float32 terms over the batch (|dg| <= 1e-4 of the largest component,
on rows away from ReLU kinks, where float32 and float64 can take different
branches)."""
import numpy as np
import pytest
import torch

from oracle import mlp as omlp
from paper_2402_11454_gb300 import graphgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gsp():
    from paper_2402_11454_gb300 import build
    build.build()
    from paper_2402_11454_gb300 import gsp as g
    return g


def rows(rng, n):
    X = np.stack([rng.uniform(0, 1, n), rng.uniform(0, 1, n), rng.uniform(0, 1, n), rng.uniform(-1, 1, n),
                  rng.integers(0, 2, n), rng.integers(0, 20, n) / 20.0], axis=1).astype(np.float32)
    y = rng.integers(0, 2, n).astype(np.uint8)
    return X, y


def params(rng, scale=0.5):
    return (rng.standard_normal(omlp.N_PARAMS) * scale).astype(np.float32)


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n", [1, 31, 10007])
def test_forward_matches_oracle(gsp, n):
    rng = np.random.default_rng(n)
    P, (X, _) = params(rng), rows(rng, n)
    p = gsp.mlp_forward(cuda(P), cuda(X)).cpu().numpy()
    ref = omlp.forward(P, X.astype(np.float64))
    assert np.max(np.abs(p - ref)) <= 1e-5


def test_forward_zero_rows(gsp):
    rng = np.random.default_rng(0)
    p = gsp.mlp_forward(cuda(params(rng)), torch.zeros((0, 6), dtype=torch.float32, device="cuda"))
    assert p.numel() == 0


@pytest.mark.parametrize("n", [1, 100, 20011])
def test_backward_matches_oracle(gsp, n):
    rng = np.random.default_rng(100 + n)
    P = params(rng)
    X, y = rows(rng, 3 * n)
    # keep rows whose pre-activations are clear of the ReLU kinks
    _, a1, _, a2, _, _ = omlp._layers(P, X.astype(np.float64), True)
    ok = (np.abs(a1).min(axis=1) > 1e-3) & (np.abs(a2).min(axis=1) > 1e-3)
    X, y = X[ok][:n], y[ok][:n]
    assert len(y) == n
    g, loss = gsp.mlp_backward(cuda(P), cuda(X), cuda(y))
    L, gref = omlp.loss_and_grad(P, X.astype(np.float64), y)
    g = g.cpu().numpy()
    assert loss == pytest.approx(L, rel=1e-5, abs=1e-7)
    assert np.max(np.abs(g - gref)) <= 1e-4 * np.max(np.abs(gref)) + 1e-7


def test_adam_matches_oracle(gsp):
    rng = np.random.default_rng(7)
    P = params(rng)
    m = np.zeros_like(P)
    v = np.zeros_like(P)
    dP, dm, dv = cuda(P.copy()), cuda(m.copy()), cuda(v.copy())
    ref_p, ref_m, ref_v = P.astype(np.float64), m.astype(np.float64), v.astype(np.float64)
    for t in range(1, 6):
        G = (rng.standard_normal(omlp.N_PARAMS) * 0.1).astype(np.float32)
        gsp.mlp_adam(dP, cuda(G), dm, dv, 1e-2, t)
        # the C ABI takes float32 hyper-parameters: give the oracle the same values
        ref_p, ref_m, ref_v = omlp.adam_step(ref_p, G, ref_m, ref_v, float(np.float32(1e-2)), t,
                                             beta1=float(np.float32(0.9)), beta2=float(np.float32(0.999)),
                                             eps=float(np.float32(1e-8)))
    assert np.allclose(dP.cpu().numpy(), ref_p, rtol=1e-5, atol=1e-6)
    assert np.allclose(dm.cpu().numpy(), ref_m, rtol=1e-5, atol=1e-9)
    assert np.allclose(dv.cpu().numpy(), ref_v, rtol=1e-5, atol=1e-12)


def test_sgd_step(gsp):
    rng = np.random.default_rng(8)
    P, G = params(rng), params(rng)
    d = cuda(P.copy())
    gsp.mlp_sgd(d, cuda(G), 0.125)
    ref = P.astype(np.float64) - 0.125 * G.astype(np.float64)
    assert np.allclose(d.cpu().numpy(), ref, rtol=2 ** -23, atol=1e-30)


def test_trace_rows(gsp):
    off, tgt, w = graphgen.planted(n=10000, k=64, mean_degree=16, p_intra=0.8, seed=1)
    d = (cuda(off.astype(np.int64)), cuda(tgt.astype(np.int32)), cuda(w))
    # each wave runs once: the first sweep of a pass then visits each vertex once
    x, y = gsp.louvain_trace(*d, capacity=1 << 16, sample_every=2, wave_repeats=1)
    x, y = x.cpu().numpy(), y.cpu().numpy()
    assert 1000 < len(y) <= 1 << 16
    assert set(np.unique(y)) == {0, 1}
    deg = np.diff(off.astype(np.int64))
    assert np.all(x[:, 0] >= 0) and np.all(x[:, 0] <= np.log1p(8 * deg.sum()) / 16 + 1e-6)
    assert np.all((x[:, 1] >= 0) & (x[:, 1] <= 1 + 1e-6))
    assert np.all((x[:, 2] >= 0) & (x[:, 2] <= 1 + 1e-6))
    assert np.all((x[:, 3] >= -1) & (x[:, 3] <= 1))
    assert set(np.unique(x[:, 4])) <= {0.0, 1.0}
    assert np.allclose(x[:, 5] * 20, np.round(x[:, 5] * 20), atol=1e-5)
    first = x[:, 5] == 0  # first sweep of a pass: nothing visited yet
    assert first.any()
    assert np.all(x[first, 2] == 0) and np.all(x[first, 3] == 1) and np.all(x[first, 4] == 1)


@pytest.mark.parametrize("name", ["rmat12", "planted", "grid"])
def test_trace_features_match_oracle(gsp, name):
    """Every visit the GPU records (every visit, frozen-state FP64 mode) has
    the predictor inputs that oracle.mlp.features computes from the oracle's
    own run state at that visit (degree, K_i, the kept fraction, scaled gain
    and move of the vertex's previous visit in the pass, the iteration), and
    the same move label.  Rows are matched by (pass, iteration, repeat,
    vertex)."""
    import oracle
    if name == "rmat12":
        off, tgt, w = graphgen.rmat(12, 16, seed=2)
    elif name == "planted":
        off, tgt, w = graphgen.planted(n=3000, k=24, mean_degree=12, p_intra=0.8, seed=1)
    else:
        off, tgt, w = graphgen.grid(40, 50, seed=3)
    d = (cuda(off.astype(np.int64)), cuda(tgt.astype(np.int32)), cuda(w))
    x, y, keys = gsp.louvain_trace(*d, capacity=1 << 20, sample_every=1, with_keys=True, precision="fp64")
    x, y, keys = x.cpu().numpy(), y.cpu().numpy(), keys.cpu().numpy().astype(np.uint64)
    g = oracle.Graph(off, tgt, w.astype(np.float64))
    _, _, r = oracle.louvain_trace(g, oracle.LouvainOptions(sync=True, split="lpp"), capacity=1 << 20)
    keep = r["degree"] > 0  # isolated vertices have no candidate and no kernel visit
    okeys = ((r["pass"].astype(np.uint64) << np.uint64(56)) | (r["iteration"].astype(np.uint64) << np.uint64(48))
             | (r["repeat"].astype(np.uint64) << np.uint64(40)) | r["vertex"].astype(np.uint64))[keep]
    assert len(np.unique(keys)) == len(keys)
    assert len(keys) == len(okeys) and np.array_equal(np.sort(keys), np.sort(okeys))
    ox = np.zeros((int(keep.sum()), 6))
    rk = {k: v[keep] for k, v in r.items()}
    for p in np.unique(rk["pass"]):  # one largest K per pass's graph
        sel = rk["pass"] == p
        ox[sel] = omlp.features(rk["degree"][sel], rk["K"][sel], rk["kept"][sel], rk["gain"][sel],
                                rk["moved_last"][sel], rk["max_K"][sel][0], rk["iteration"][sel], 20)
    gi, oi = np.argsort(keys), np.argsort(okeys)
    np.testing.assert_allclose(x[gi], ox[oi], rtol=1e-5, atol=1e-6)
    assert np.array_equal(y[gi], r["moved"][keep][oi].astype(np.uint8))
    assert y.sum() > 0 and (x[:, 4] == 0).sum() > 0


def test_learned_pruning_gain(gsp):
    """Trained on traces of one R-MAT graph, the predictor ranks the visits of
    another graph better than the same network untrained (more visits skipped
    at the same recall of the moving ones); a learned run on that graph does
    less local-moving work than the plain method (fewer edge visits), leaves
    no internally disconnected community and stays within 0.002 of the plain
    run's modularity."""
    from paper_2402_11454_gb300 import pruner
    off, tgt, w = gsp.gen_rmat(15, 16, seed=2)
    x, y = pruner.collect_traces(off, tgt, w, capacity=1 << 21, sample_every=1)
    xb, yb = pruner.balance(x, y, seed=0)
    P, rep = pruner.train(xb, yb, steps=600, batch=16384, seed=0)
    assert rep["holdout_loss"] < 0.69  # better than chance (ln 2)
    off2, tgt2, w2 = gsp.gen_rmat(17, 16, seed=3)
    x2, y2 = pruner.collect_traces(off2, tgt2, w2, capacity=1 << 22, sample_every=1)
    P0 = pruner.init_params(seed=0)
    ev_trained = pruner.evaluate(P, x2, y2, pruner.threshold_for_recall(P, x2, y2, recall=0.95))
    ev_untrained = pruner.evaluate(P0, x2, y2, pruner.threshold_for_recall(P0, x2, y2, recall=0.95))
    assert ev_trained["recall"] >= 0.94
    assert ev_trained["skip_rate"] > ev_untrained["skip_rate"] + 0.05
    thr = pruner.threshold_for_recall(P, x, y, recall=0.95)
    C0, q0, st0 = gsp.louvain(off2, tgt2, w2)
    C1, q1, st1 = gsp.louvain(off2, tgt2, w2, prune="learned", mlp_params=P, prune_threshold=thr)
    assert sum(st1["vertices_skipped"]) > 0
    assert sum(st1["edges_scanned"]) < sum(st0["edges_scanned"]), (st1["edges_scanned"], st0["edges_scanned"])
    assert gsp.count_disconnected(off2, tgt2, C1)[0] == 0
    assert q1 >= q0 - 0.002
    assert q1 == pytest.approx(gsp.modularity(off2, tgt2, w2, C1), rel=1e-9)


def test_learned_pruning_never_skipping_is_plain(gsp):
    """Threshold 0 skips nothing: the run equals the plain method's."""
    off, tgt, w = gsp.gen_rmat(14, 16, seed=2)
    P = torch.zeros(gsp.mlp_param_count(), dtype=torch.float32, device="cuda")
    C0, q0, _ = gsp.louvain(off, tgt, w, precision="fp64")
    C1, q1, st1 = gsp.louvain(off, tgt, w, precision="fp64", prune="learned", mlp_params=P, prune_threshold=0.0)
    assert sum(st1["vertices_skipped"]) == 0
    assert torch.equal(C0, C1) and q0 == q1


def test_learned_pruning_skipping_everything_still_converges(gsp):
    """A predictor that skips every vertex leaves the work to the periodic
    plain sweeps; the result keeps the method's guarantees."""
    off, tgt, w = gsp.gen_rmat(14, 16, seed=2)
    P = torch.zeros(gsp.mlp_param_count(), dtype=torch.float32, device="cuda")
    P[-1] = -30.0  # b3: P(move) ~ 1e-13 everywhere
    C0, q0, _ = gsp.louvain(off, tgt, w)
    C1, q1, st1 = gsp.louvain(off, tgt, w, prune="learned", mlp_params=P, prune_threshold=0.5)
    assert sum(st1["vertices_skipped"]) > 0
    assert gsp.count_disconnected(off, tgt, C1)[0] == 0
    assert q1 >= q0 - 0.01
