"""Training of the learned vertex-pruning predictor.

The predictor (a 6 -> 32 -> 32 -> 1 MLP, see gsp_mlp_forward) estimates from a
vertex's state at its last visit whether its next visit of local moving
(Algorithm 4) will move it; with ``prune="learned"`` a sweep skips the active
vertices it scores below a threshold, and every ``full_sweep_every``-th
sweep is a plain sweep that catches what the skipped visits missed.

Training data are move/no-move traces of the plain method (gsp_louvain_trace).
All arithmetic of training and inference runs in the library's kernels
(forward, binary cross-entropy backward, Adam); this module only draws the
initial weights, shuffles and slices the rows, and picks the threshold.
"""
import numpy as np
import torch

from . import gsp

N_IN, N_H = 6, 32


def init_params(seed=0, device="cuda"):
    """He-normal initial weights (fan-in scaling for the ReLU layers), zero
    biases, packed W1, b1, W2, b2, W3, b3."""
    rng = np.random.default_rng(seed)
    parts = [rng.standard_normal(N_H * N_IN) * np.sqrt(2.0 / N_IN), np.zeros(N_H),
             rng.standard_normal(N_H * N_H) * np.sqrt(2.0 / N_H), np.zeros(N_H),
             rng.standard_normal(N_H) * np.sqrt(1.0 / N_H), np.zeros(1)]
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == gsp.mlp_param_count()
    return torch.from_numpy(p).to(device)


def collect_traces(offsets, targets, weights, capacity=1 << 24, sample_every=8, **kw):
    """Move/no-move rows of one plain run: (features [rows, 6], labels [rows])."""
    return gsp.louvain_trace(offsets, targets, weights, capacity, sample_every, **kw)


def balance(x, y, seed=0):
    """Rows with equal numbers of moved and not-moved labels (the larger class
    subsampled), shuffled."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    pos = torch.nonzero(y == 1).flatten().cpu()
    neg = torch.nonzero(y == 0).flatten().cpu()
    k = min(len(pos), len(neg))
    if k == 0:
        raise ValueError("traces hold a single class")
    pos = pos[torch.randperm(len(pos), generator=g)[:k]]
    neg = neg[torch.randperm(len(neg), generator=g)[:k]]
    idx = torch.cat([pos, neg])[torch.randperm(2 * k, generator=g)].to(x.device)
    return x[idx].contiguous(), y[idx].contiguous()


def train(x, y, steps=1500, batch=65536, lr=3e-3, seed=0, holdout=0.1):
    """Adam on the mean binary cross-entropy over minibatches of the rows.
    Returns (params, report) with the loss on the held-out rows."""
    n = x.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    perm = torch.randperm(n, generator=g).to(x.device)
    x, y = x[perm].contiguous(), y[perm].contiguous()
    n_hold = max(1, int(n * holdout))
    xh, yh = x[:n_hold], y[:n_hold]
    xt, yt = x[n_hold:], y[n_hold:]
    params = init_params(seed, x.device)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    nt = xt.shape[0]
    batch = min(batch, nt)
    nb = max(1, nt // batch)
    losses = []
    for t in range(1, steps + 1):
        b = (t - 1) % nb
        grad, loss = gsp.mlp_backward(params, xt[b * batch:(b + 1) * batch], yt[b * batch:(b + 1) * batch])
        gsp.mlp_adam(params, grad, m, v, lr, t)
        if t % 100 == 0 or t == steps:
            losses.append(loss)
    _, hold_loss = gsp.mlp_backward(params, xh, yh)
    return params, {"train_rows": nt, "holdout_rows": n_hold, "steps": steps, "batch": batch,
                    "train_loss": losses[-1], "holdout_loss": hold_loss, "loss_curve": losses}


def threshold_for_recall(params, x, y, recall=0.9):
    """The largest threshold that still keeps `recall` of the moving rows
    (P(move) >= threshold for that fraction of them)."""
    p = gsp.mlp_forward(params, x)
    pos = p[y == 1].double().cpu().numpy()
    if pos.size == 0:
        return 0.0
    return float(np.quantile(pos, 1.0 - recall, method="lower"))


def evaluate(params, x, y, threshold):
    """Recall of moving rows and skip rate of all rows at a threshold."""
    p = gsp.mlp_forward(params, x)
    keep = p >= threshold
    pos = y == 1
    npos = int(pos.sum())
    return {"recall": float((keep & pos).sum()) / max(1, npos),
            "skip_rate": 1.0 - float(keep.float().mean()),
            "moved_fraction": npos / max(1, y.numel())}
