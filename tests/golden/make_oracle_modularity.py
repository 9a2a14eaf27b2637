"""Write oracle_modularity.json: the sequential oracle's modularity on the
synthetic workloads that the benchmark times.

Each value is the oracle's run of Algorithm 1 with the one-thread in-place
loop of Algorithm 4 (vertices in id order), the LPP split every pass and the
default parameters (10 passes, 20 iterations, tau 1e-2, drop 10, tau_agg
0.8).  The graphs come from the seeded host generators; nothing here calls
the CUDA library.  The R-MAT scale-26 graph (2.1 B entries) is left out: its
oracle run needs more host memory than this machine has.

    python tests/golden/make_oracle_modularity.py [--jobs 8] [--skip-batch]
"""
import argparse
import json
import os
import sys
import time
from multiprocessing import get_context

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
OUT = os.path.join(HERE, "oracle_modularity.json")


def _oracle_q(off, tgt, w):
    import numpy as np
    import oracle
    g = oracle.Graph(off, tgt, np.asarray(w, dtype=np.float64))
    t0 = time.perf_counter()
    _, st = oracle.louvain(g, oracle.LouvainOptions(sync=False, split="lpp"))
    return {"modularity": st["modularity"], "communities": int(st["final_communities"]),
            "passes": int(st["passes"]), "iterations": [int(x) for x in st["iterations"]],
            "vertices": int(g.n), "edges": int(g.nnz), "seconds": round(time.perf_counter() - t0, 2)}


def single(name):
    from paper_2402_11454_gb300 import graphgen
    if name == "planted":
        off, tgt, w = graphgen.planted(n=10000, k=64, mean_degree=16, p_intra=0.8, seed=1)
    elif name.startswith("rmat"):
        scale, seed = {"rmat20": (20, 2), "rmat22": (22, 2)}[name]
        off, tgt, w = graphgen.rmat(scale, 16, seed=seed)
    elif name == "grid4096":
        off, tgt, w = graphgen.grid(4096, 4096, seed=3)
    else:
        raise ValueError(name)
    r = _oracle_q(off, tgt, w)
    print(name, r, flush=True)
    return name, r


def batch_graph(g):
    """Graph g of the 4096-graph batch, drawn alone (the batch is the
    concatenation of these graphs, so its per-graph results are these)."""
    from paper_2402_11454_gb300 import graphgen
    n, k, e, p = graphgen.batch_params(4096, seed=4)
    u, v = graphgen.planted_edges(int(n[g]), int(k[g]), int(e[g]), float(p[g]), graphgen.batch_graph_seed(4, g))
    off, tgt, w = graphgen.edges_to_csr(int(n[g]), u, v)
    return g, _oracle_q(off, tgt, w)["modularity"]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=os.cpu_count() or 4)
    ap.add_argument("--skip-batch", action="store_true")
    ap.add_argument("--only", default=None, help="comma-separated subset of planted,rmat20,rmat22,grid4096")
    args = ap.parse_args()
    import oracle
    oracle.build_oracle()
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    data["_about"] = ("Sequential oracle (Algorithm 1, one-thread in-place Algorithm 4, LPP split, default "
                      "parameters) on the seeded synthetic workloads; written by make_oracle_modularity.py")
    names = ["planted", "rmat20", "rmat22", "grid4096"]
    if args.only:
        names = [x for x in args.only.split(",") if x]
    ctx = get_context("spawn")
    with ctx.Pool(min(args.jobs, len(names))) as pool:
        for name, r in pool.imap_unordered(single, names):
            data[name] = r
    if not args.skip_batch:
        t0 = time.perf_counter()
        with ctx.Pool(args.jobs) as pool:
            qs = dict(pool.imap_unordered(batch_graph, range(4096), chunksize=16))
        data["batch4096"] = {"graphs": 4096, "seconds": round(time.perf_counter() - t0, 1),
                             "modularity": [round(qs[g], 9) for g in range(4096)]}
    with open(OUT, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
