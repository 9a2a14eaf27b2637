"""Split ablation on the synthetic stand-ins of the paper's graphs: the split
technique (none = GVE-Louvain, label propagation, label propagation with
pruning, BFS, and hooking/shortcutting (SV), which is not in the paper) and
its placement (after every pass, or once at the end), as in the paper's
comparison of split variants (Section 4.1) and of GSP-Louvain against the
method without a split (Section 5); and the Leiden refinement (Section 3.5)
with and without the split (GSP-Leiden).

For every configuration it reports the device time of one gsp_louvain call,
the modularity, the number of communities and the number of internally
disconnected communities (Algorithm 6, counted on the GPU).

    python -m paper_2402_11454_gb300.ablation [--workloads planted,rmat22,grid] [--steps 3]

Prints one JSON object per line.
"""
import argparse
import json
import sys

# (split technique, placement, Leiden refinement)
VARIANTS = [
    ("none", "pass", False),   # GVE-Louvain: no split
    ("lp", "pass", False),
    ("lpp", "pass", False),
    ("bfs", "pass", False),
    ("sv", "pass", False),
    ("lp", "last", False),
    ("lpp", "last", False),
    ("bfs", "last", False),
    ("sv", "last", False),
    ("none", "pass", True),    # refinement (Section 3.5) without a split
    ("lpp", "pass", True),     # GSP-Leiden
]


def workload(gsp, name):
    if name == "planted":
        return gsp.gen_planted(n=10000, k=64, mean_degree=16, p_intra=0.8, seed=1)
    if name == "grid":
        return gsp.gen_grid(4096, 4096, seed=3)
    if name.startswith("rmat") and name[4:].isdigit():
        return gsp.gen_rmat(int(name[4:]), 16, seed=2)
    raise SystemExit("unknown workload %s" % name)


def main(argv=None):
    import torch
    from . import build
    build.build()
    from . import gsp
    ap = argparse.ArgumentParser()
    ap.add_argument("--workloads", default="planted,rmat22,grid")
    ap.add_argument("--steps", type=int, default=3)
    args = ap.parse_args(argv)
    for name in args.workloads.split(","):
        off, tgt, w = workload(gsp, name)
        gsp.autotune(off, tgt, w)
        for split, when, refine in VARIANTS:
            kw = dict(split=split, split_when=when, refine=refine)
            gsp.louvain(off, tgt, w, **kw)  # warm-up
            times = []
            for _ in range(args.steps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                C, q, st = gsp.louvain(off, tgt, w, **kw)
                e1.record()
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
            dis, _ = gsp.count_disconnected(off, tgt, C)
            print(json.dumps({"workload": name, "edges": int(tgt.numel()), "split": split, "split_when": when,
                              "refine": refine,
                              "ms": round(min(times), 3), "modularity": q,
                              "communities": st["final_communities"], "disconnected": dis,
                              "passes": st["passes"], "split_ms": round(sum(st["ms_split"]), 3)}), flush=True)
        del off, tgt, w
        torch.cuda.empty_cache()
    return 0


if __name__ == "__main__":
    sys.exit(main())
