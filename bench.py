"""GSP-Louvain benchmark: edges/s of the whole method on one GB300.

Default workload: R-MAT scale 26 (67.1 M vertices, edge factor 16,
a/b/c/d = 0.57/0.19/0.19/0.05, symmetrised, deduplicated, self-loops dropped,
unit float32 weights, seed 5), the plain method (flag pruning), float32
delta-Q with float64 m / Sigma_tot / modularity.  A step is one full
gsp_louvain call (all passes: local moving, split, aggregation, final
modularity) on the graph already resident in HBM.  edges/s = directed CSR
entries / step time.

Beside the timed line the same JSON carries:
  learned  the learned-pruning form on the same graph, its predictor trained
           (untimed) on move traces of the R-MAT scale-22 graph (seed 2);
  e2e      the same metric through gsp_louvain_host (pinned host buffers,
           copies inside the timing);
  configs  the other workloads (planted 10 K, R-MAT 22, grid 4096^2, batch
           of 4096 planted graphs), fewer steps each: edges/s, modularity,
           its error against the float64 run, against the sequential oracle
           (stored values) and the local-moving roofline fraction;
  gsp_leiden  the GSP-Leiden variant (Leiden refinement after each pass's
           split) on R-MAT 22: the same figures, and its modularity and time
           against the GSP-Louvain run of that graph.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload rmat26|rmat22|planted|grid|batch|rmatNN]
                  [--configs all|none|name,name] [--learned auto|on|off]

Under torchrun (N > 1) every rank runs its own replica (the method does not
shard a single graph); value = edges of all ranks / max time over ranks.
--impl reference times the sequential CPU oracle on a bounded R-MAT sample.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GSP-Louvain edges/s on 1 GB300"
UNIT = "edges/s"
GOLDEN = os.path.join(ROOT, "tests", "golden", "oracle_modularity.json")


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def log(msg):
    print("[bench %s] %s" % (time.strftime("%H:%M:%S"), msg), file=sys.stderr, flush=True)


def load_golden():
    """Sequential-oracle modularity of the workloads (stored by
    tests/golden/make_oracle_modularity.py), or {}."""
    if os.path.exists(GOLDEN):
        with open(GOLDEN) as f:
            return json.load(f)
    return {}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region.  The log
    goes to `path` (default: a temporary file)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, path=None):
        self.idx = gpu_index
        self.proc = None
        self.path = path

    def start(self):
        try:
            if self.path:
                os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
                self.f = open(self.path, "w")
            else:
                fd, self.path = tempfile.mkstemp(prefix="gsp_clocks_", suffix=".csv")
                self.f = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        with open(self.path) as f:
            return parse_clock_log(f)


def parse_clock_log(lines):
    """Median SM clock, maximum SM clock and the throttle reasons seen in
    nvidia-smi samples (ClockSampler.FIELDS, csv, no header, no units)."""
    sm, mx, reasons = [], 0.0, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            mx = max(mx, float(parts[2]))
        except ValueError:
            continue
        for nm, val in zip(names, parts[5:9]):
            if val.lower() == "active":
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x, dist, device):
    """The largest x over the ranks of the process group (x itself without
    one): the job takes as long as its slowest rank."""
    if not dist:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, steps, world_size, seconds):
    """Whole-job rate: every rank processes units_per_rank per step (one
    replica each), all ranks together in `seconds` (the max over ranks)."""
    return units_per_rank * steps * world_size / seconds


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


RMAT_ABCD = [0.57, 0.19, 0.19, 0.05]


def make_workload(gsp, graphgen, name):
    """Generate the workload on the device; returns (off, tgt, w, config, gvo),
    gvo = per-graph vertex offsets of a batch (None for one graph)."""
    gvo = None
    if name in ("rmat26", "rmat22"):
        scale, seed = (26, 5) if name == "rmat26" else (22, 2)
        off, tgt, w = gsp.gen_rmat(scale, 16, seed=seed)
        cfg = {"workload": name, "scale": scale, "edge_factor": 16, "abcd": RMAT_ABCD, "seed": seed}
    elif name.startswith("rmat") and name[4:].isdigit():  # other R-MAT scales, for profiling
        sc = int(name[4:])
        off, tgt, w = gsp.gen_rmat(sc, 16, seed=2)
        cfg = {"workload": name, "scale": sc, "edge_factor": 16, "abcd": RMAT_ABCD, "seed": 2}
    elif name == "planted":
        off, tgt, w = gsp.gen_planted(n=10000, k=64, mean_degree=16, p_intra=0.8, seed=1)
        cfg = {"workload": "planted", "vertices": 10000, "communities": 64, "mean_degree": 16,
               "p_intra": 0.8, "seed": 1}
    elif name == "grid":
        off, tgt, w = gsp.gen_grid(4096, 4096, seed=3)
        cfg = {"workload": "grid4096", "rows": 4096, "cols": 4096, "p_remove": 0.05, "p_long": 0.001,
               "weights": [1.0, 10.0], "seed": 3}
    elif name == "batch":
        import numpy as np
        G = 4096
        n, k, e, p = graphgen.batch_params(G, seed=4)
        seeds = [graphgen.batch_graph_seed(4, g) for g in range(G)]
        off, tgt, w = gsp.gen_planted_batch(n, k, e, p, seeds)
        gvo = np.zeros(G + 1, dtype=np.uint64)
        np.cumsum(n, out=gvo[1:])
        cfg = {"workload": "batch4096", "graphs": G, "vertices_per_graph": "log-uniform [64, 65536]",
               "communities": "uniform {4..64}", "mean_degree": "uniform [4, 64]",
               "p_intra": "uniform [0.7, 0.9]", "seed": 4}
    else:
        raise SystemExit("unknown workload %s" % name)
    cfg["vertices"] = int(off.numel() - 1)
    cfg["edges"] = int(tgt.numel())
    return off, tgt, w, cfg, gvo


# DRAM bytes (ncu dram__bytes_read.sum + dram__bytes_write.sum) of all
# local-moving launches of one call divided by that call's algorithmic bytes,
# per workload whose capture exists (profiles/dram_local_moving_rmat26.md,
# profiles/dram_local_moving_rmat20.md).  Above L2 the gathers of C_j and
# Sigma_c go to DRAM in 32-byte sectors, so the ratio grows with the graph:
# the R-MAT 20 figure stands in for the smaller workloads (scaled, and said
# so in the line).
MOVE_TRAFFIC_RATIO = {"rmat26": (3.737, "measured: an ncu capture of every local-moving launch of one R-MAT 26 "
                                        "call, 872.7 GB over 233.5 GB of algorithmic bytes")}
MOVE_TRAFFIC_FALLBACK = (2.153, "scaled: the ratio of an ncu capture of every local-moving launch of one R-MAT 20 "
                                "call, times the algorithmic bytes of this workload")


def roofline_from(stats_list, peak_gbs, peak_kind, workload=None):
    byt = sum(sum(s["move_bytes"]) for s in stats_list)
    ms = sum(sum(s["ms_move_kernels"]) for s in stats_list)
    if ms <= 0:
        return None
    achieved = byt / (ms * 1e-3) / 1e9
    per_step = byt / max(1, len(stats_list))
    r = {"bound": "hbm", "kernel": "local-moving sweep (all k_move_*/k_hub_*/k_apply_moves launches of a sweep)",
         "achieved": round(achieved, 1), "peak": peak_gbs, "peak_kind": peak_kind + " (burst copy)",
         "unit": "GB/s", "frac": round(achieved / peak_gbs, 4), "traffic": None,
         "algorithmic_bytes_per_step": per_step}
    ratio, basis = MOVE_TRAFFIC_RATIO.get(workload, MOVE_TRAFFIC_FALLBACK)
    r["traffic"] = round(per_step * ratio)
    r["traffic_basis"] = "DRAM bytes per step, %.3f x the algorithmic bytes; %s" % (ratio, basis)
    # DRAM throughput those bytes mean over the kernels' device time
    r["dram_gbs"] = round(r["traffic"] / (ms / max(1, len(stats_list)) * 1e-3) / 1e9, 1)
    r["dram_frac"] = round(r["dram_gbs"] / peak_gbs, 4)
    return r


def phase_rooflines(st, peak_gbs, input_wbytes=4):
    """Algorithmic bytes and GB/s of each phase of one step (lower bounds:
    one pass over what the phase must read and write).
      split: per edge target 4 + C_j 4 + label_j 4, per vertex C_i 4 +
             label 4 + offsets 16;
      aggregation: per input edge target 4 + weight (4 or 8) + Cd_j 4, per
             vertex Cd 4 + offsets 16 + member list 8, per output super-edge
             target 4 + weight 8, per super-vertex offset 8."""
    P = min(st["passes"], len(st["edges"]))
    E, V = st["edges"], st["vertices"]
    split_b = sum(12.0 * E[p] + 24.0 * V[p] for p in range(P))
    agg_b = 0.0
    for p in range(P):
        if st["ms_aggregate"][p] <= 0 or p + 1 >= P:
            continue
        wb = input_wbytes if p == 0 else 8
        agg_b += (8.0 + wb) * E[p] + 28.0 * V[p] + 12.0 * E[p + 1] + 8.0 * V[p + 1]
    # refinement (GSP-Leiden): per edge target 4 + weight (4 or 8) + B_u 4 +
    # R_u 4, per vertex B, R, T 4 each, K, S_R, E(c, b-c), E(v, T) 8 each,
    # size 4 (the passes that refined)
    ref_b = 0.0
    for p in range(P):
        if st.get("ms_refine") and st["ms_refine"][p] > 0:
            wb = input_wbytes if p == 0 else 8
            ref_b += (12.0 + wb) * E[p] + 48.0 * V[p]
    out = {}
    for name, b, ms in (("split", split_b, sum(st["ms_split"])), ("aggregate", agg_b, sum(st["ms_aggregate"])),
                        ("move", sum(st["move_bytes"]), sum(st["ms_move_kernels"])),
                        ("refine", ref_b, sum(st.get("ms_refine") or [0.0]))):
        if ms > 0 and b > 0:
            gbs = b / (ms * 1e-3) / 1e9
            out[name] = {"bytes": b, "ms": round(ms, 3), "achieved_gbs": round(gbs, 1),
                         "frac": round(gbs / peak_gbs, 4)}
    return out


def timed_steps(step, steps, flush, stream):
    """Device time of `steps` calls (CUDA events on the launching stream, a
    256 MB L2 flush before each); returns (ms list, stats list, last result)."""
    import torch
    times, stats, res = [], [], None
    for _ in range(steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        stats.append(res[2])
    return times, stats, res


def oracle_reference(golden, cfg):
    """Sequential-oracle modularity stored for this workload (None when the
    workload has no stored value)."""
    name = cfg["workload"]
    d = golden.get(name)
    if not d:
        return None
    return d["modularity"]


def quality(gsp, off, tgt, w, gvo, kw, q, golden, cfg):
    """Untimed runs for the per-result error: the float64 run's modularity
    (error of the mixed-precision result), the disconnected-community count,
    and the distance to the sequential oracle's stored modularity."""
    import numpy as np
    out = {}
    if gvo is None:
        _, q64, st64 = gsp.louvain(off, tgt, w, **dict(kw, precision="fp64"))
        _, _, stc = gsp.louvain(off, tgt, w, count_disconnected=True, **kw)
        out["modularity_fp64"] = q64
        out["dQ_mixed_vs_fp64"] = q - q64
        out["disconnected_communities"] = stc["disconnected"]
        ref = oracle_reference(golden, cfg)
        if ref is not None:
            out["oracle_modularity"] = ref
            out["dQ_vs_oracle"] = q - ref
        else:
            out["oracle_modularity"] = None
            out["oracle_note"] = "not run: the sequential oracle on this graph needs more host memory than the " \
                                 "machine that stores the oracle's values has" if cfg["workload"] == "rmat26" \
                else "no stored value"
    else:
        _, qg64, _ = gsp.louvain_batched(gvo, off, tgt, w, **dict(kw, precision="fp64"))
        _, qg, stc = gsp.louvain_batched(gvo, off, tgt, w, count_disconnected=True, **kw)
        qg, qg64 = qg.cpu().numpy(), qg64.cpu().numpy()
        out["modularity_fp64_mean"] = float(qg64.mean())
        out["dQ_mixed_vs_fp64"] = {"mean": float((qg - qg64).mean()), "min": float((qg - qg64).min()),
                                   "max": float((qg - qg64).max())}
        out["disconnected_communities"] = stc["disconnected"]
        ref = golden.get("batch4096", {}).get("modularity")
        if ref is not None and len(ref) == len(qg):
            d = qg - np.asarray(ref)
            out["dQ_vs_oracle"] = {"mean": float(d.mean()), "min": float(d.min()),
                                   "graphs_below_0.002": int((d < -0.002).sum())}
    return out


def run_workload(gsp, graphgen, name, kw, steps, warmup, flush, stream, peak, kind, golden, autotune=True):
    """One workload: generate, autotune (untimed), warm up, time `steps`
    calls; returns a summary dict (and the device graph for further use)."""
    off, tgt, w, cfg, gvo = make_workload(gsp, graphgen, name)

    def step():
        if gvo is None:
            return gsp.louvain(off, tgt, w, **kw)
        C, qg, st = gsp.louvain_batched(gvo, off, tgt, w, **kw)
        return C, st["modularity"], st

    tuning = {"caps": gsp.get_tuning(), "autotuned": False}
    if autotune:
        caps, ms0, ms1 = gsp.autotune(off, tgt, w, graph_vertex_offsets=gvo, **kw)
        tuning = {"caps": caps, "autotuned": True, "tuning_run_ms_default": round(ms0, 3),
                  "tuning_run_ms_tuned": round(ms1, 3)}
    for _ in range(max(warmup, 0)):
        step()
    times, stats, (C, q, st) = timed_steps(step, steps, flush, stream)
    ms = sum(times) / len(times)
    cfg = dict(cfg, wave_repeats=kw.get("wave_repeats", 3))
    summary = {"config": cfg, "edges_per_s": cfg["edges"] / (ms * 1e-3), "ms_per_step": ms, "steps": steps,
               "modularity": q, "communities": st["final_communities"], "passes": st["passes"],
               "iterations": st["iterations"], "roofline_move": roofline_from(stats, peak, kind, name),
               "phase_roofline": phase_rooflines(st, peak), "tuning": tuning}
    summary.update(quality(gsp, off, tgt, w, gvo, kw, q, golden, cfg))
    return summary, (off, tgt, w, cfg, gvo, times, stats, st, q, tuning)


def learned_compare(gsp, args, off, tgt, w, kw, flush, stream, plain_ms, plain_q, plain_stats, edges, timed_name):
    """Learned pruning against the plain method on the same graph: the
    predictor is trained (untimed) on move traces of the R-MAT scale-22 graph
    (seed 2) with the library's kernels, its threshold set to keep `recall`
    of the moving visits; then timed like the plain run."""
    import torch
    from paper_2402_11454_gb300 import pruner
    t0 = time.perf_counter()
    o2, t2, w2 = gsp.gen_rmat(22, 16, seed=2)
    x, y = pruner.collect_traces(o2, t2, w2, capacity=1 << 23, sample_every=8, **kw)
    xb, yb = pruner.balance(x, y, seed=0)
    P, rep = pruner.train(xb, yb, steps=1500, batch=65536, seed=0)
    thr = pruner.threshold_for_recall(P, x, y, recall=args.recall)
    ev = pruner.evaluate(P, x, y, thr)
    del o2, t2, w2, x, y, xb, yb
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    train_s = time.perf_counter() - t0
    lkw = dict(kw, prune="learned", mlp_params=P, prune_threshold=thr)
    for _ in range(max(args.warmup, 0)):
        gsp.louvain(off, tgt, w, **lkw)
    times, _, (C, q, st) = timed_steps(lambda: gsp.louvain(off, tgt, w, **lkw), args.learned_steps, flush, stream)
    ms = sum(times) / len(times)
    dis = gsp.count_disconnected(off, tgt, C)[0]
    return {"value": edges / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": args.learned_steps,
            "modularity": q, "dQ_vs_plain": q - plain_q, "speedup_vs_plain": plain_ms / ms,
            "disconnected_communities": dis,
            "vertices_skipped": sum(st["vertices_skipped"]),
            "visits_ratio_vs_plain": sum(st["vertices_processed"]) / max(1, sum(plain_stats["vertices_processed"])),
            "edges_scanned_ratio_vs_plain": sum(st["edges_scanned"]) / max(1, sum(plain_stats["edges_scanned"])),
            "iterations": st["iterations"], "full_sweep_every": 4, "threshold": thr,
            "recall_target": args.recall, "trace_recall": ev["recall"], "trace_skip_rate": ev["skip_rate"],
            "trained_on": "R-MAT scale 22, seed 2 (1 in 8 visits sampled)",
            "timed_graph": timed_name, "trained_on_timed_graph": timed_name == "rmat22",
            "train": {k: v for k, v in rep.items() if k != "loss_curve"}, "train_seconds": round(train_s, 2)}


def cpu_baseline(sample_scale=20, seed=2):
    import oracle
    from paper_2402_11454_gb300 import graphgen
    off, tgt, w = graphgen.rmat(sample_scale, 16, seed=seed)
    g = oracle.Graph(off, tgt, w.astype("float64"))
    t0 = time.perf_counter()
    _, st = oracle.louvain(g, oracle.LouvainOptions(sync=False, split="lpp"))
    dt = time.perf_counter() - t0
    return {"value": len(tgt) / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "R-MAT scale %d (edge factor 16, same a/b/c/d), %d directed edges, one sequential "
                      "oracle run (%.1f s, Q=%.4f)" % (sample_scale, len(tgt), dt, st["modularity"]),
            "cpu": cpu_model()}


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    import oracle
    from paper_2402_11454_gb300 import graphgen
    scale = args.ref_scale
    off, tgt, w = graphgen.rmat(scale, 16, seed=2)
    g = oracle.Graph(off, tgt, w.astype("float64"))
    for _ in range(args.warmup):
        oracle.louvain(g, oracle.LouvainOptions(sync=False, split="lpp"))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.louvain(g, oracle.LouvainOptions(sync=False, split="lpp"))
    dt = time.perf_counter() - t0
    val = len(tgt) * args.steps / dt
    cfg = {"workload": args.workload, "sample": "R-MAT scale %d" % scale, "edges": int(len(tgt))}
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "R-MAT scale %d, sequential oracle, %d steps" % (scale, args.steps)},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


EXTRA_CONFIGS = ("planted", "rmat22", "grid", "batch")

# Repeats of each wave in a pass's first iteration, per workload: the
# library's default (3) everywhere but the batch of small planted graphs,
# where one repeat measured both faster (450 against 510 ms per call) and
# closer to the sequential oracle (436 against 533 of the 4096 graphs more
# than 0.002 below it; worst -0.042 against -0.079).  On R-MAT the repeats
# raise the modularity at every scale tested (14-22).
WAVE_REPEATS = {"batch": 1}


def wave_repeats_for(name, args):
    return args.wave_repeats if args.wave_repeats is not None else WAVE_REPEATS.get(name, 3)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat26")
    ap.add_argument("--precision", default="mixed")
    ap.add_argument("--split", default="lpp")
    ap.add_argument("--move", default="sync")
    ap.add_argument("--waves", type=int, default=0, help="waves per iteration (0: 17 frozen-state, 64 in-place)")
    ap.add_argument("--wave-repeats", type=int, default=None,
                    help="repeats of each wave in a pass's first iteration (default: the workload's, "
                         "see WAVE_REPEATS)")
    ap.add_argument("--ref-scale", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--learned", default="auto", choices=["auto", "on", "off"],
                    help="also time learned pruning against the plain run (auto: R-MAT workloads)")
    ap.add_argument("--learned-steps", type=int, default=None, help="timed steps of the learned form (default: --steps)")
    ap.add_argument("--recall", type=float, default=0.9)
    ap.add_argument("--leiden", default="rmat22",
                    help="workload of the GSP-Leiden line (rmat22, planted, grid, ...), or none")
    ap.add_argument("--configs", default="all",
                    help="other workloads reported under 'configs': all, none, or a comma list of %s"
                         % ",".join(EXTRA_CONFIGS))
    ap.add_argument("--config-steps", type=int, default=3)
    ap.add_argument("--no-quality", action="store_true",
                    help="skip the untimed float64 and disconnected-count runs (for profiling)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default grid caps instead of tuning them on the workload (untimed)")
    ap.add_argument("--caps", default=None,
                    help="fixed grid caps 'groups,w512,block,hub' (blocks per SM) instead of autotuning")
    ap.add_argument("--clock-log", default=os.environ.get("GSP_BENCH_CLOCK_LOG"),
                    help="file for the nvidia-smi clock samples (default: a temporary file)")
    args = ap.parse_args()
    if args.learned_steps is None:
        args.learned_steps = args.steps
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, ws, rank)

    import torch
    from paper_2402_11454_gb300 import build as gbuild
    gbuild.build()
    from paper_2402_11454_gb300 import graphgen, gsp

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    kw = dict(precision=args.precision, split=args.split, move=args.move, waves=args.waves,
              wave_repeats=wave_repeats_for(args.workload, args))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # 256 MB > 129 MB L2
    stream = torch.cuda.current_stream()
    peak, kind = load_peaks()
    golden = load_golden()

    if args.caps:
        g4, w5, bl, hb = (int(x) for x in args.caps.split(","))
        gsp.set_tuning(groups_blocks_per_sm=g4, w512_blocks_per_sm=w5, block_blocks_per_sm=bl, hub_blocks_per_sm=hb)
    off, tgt, w, cfg, gvo = make_workload(gsp, graphgen, args.workload)
    log("generated %s: %d vertices, %d edges" % (cfg["workload"], cfg["vertices"], cfg["edges"]))

    def step():
        if gvo is None:
            return gsp.louvain(off, tgt, w, **kw)
        C, qg, st = gsp.louvain_batched(gvo, off, tgt, w, **kw)
        return C, st["modularity"], st

    tuning = {"caps": gsp.get_tuning(), "autotuned": False}
    if not args.no_autotune and not args.caps:  # untimed: picks the local-moving grid caps for this input
        caps, ms0, ms1 = gsp.autotune(off, tgt, w, graph_vertex_offsets=gvo, **kw)
        tuning = {"caps": caps, "autotuned": True, "tuning_run_ms_default": round(ms0, 3),
                  "tuning_run_ms_tuned": round(ms1, 3)}

    for _ in range(max(args.warmup, 0)):
        C, q, st = step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local, args.clock_log)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    l0 = gsp.kernel_launches()
    times, stats, (C, q, st) = timed_steps(step, args.steps, flush, stream)
    launches = gsp.kernel_launches() - l0
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    total_ms = max_over_ranks(sum(times), dist, "cuda")
    edges = cfg["edges"]
    value = job_throughput(edges, args.steps, ws, total_ms * 1e-3)

    # end to end: host (pinned) buffers through the C ABI, copies inside the timing
    e2e = None
    if not args.no_e2e:
        h_off = off.cpu().pin_memory()
        h_tgt = tgt.cpu().pin_memory()
        h_w = w.cpu().pin_memory()
        h_C = torch.empty(off.numel() - 1, dtype=torch.int32, pin_memory=True)

        def e2e_step():
            if gvo is None:
                gsp.louvain_host(h_off, h_tgt, h_w, h_C, **kw)
                return
            # batches: pinned host -> device, the batched call, membership back
            d_off = h_off.to("cuda", non_blocking=True)
            d_tgt = h_tgt.to("cuda", non_blocking=True)
            d_w = h_w.to("cuda", non_blocking=True)
            C2, _, _ = gsp.louvain_batched(gvo, d_off, d_tgt, d_w, **kw)
            h_C.copy_(C2)

        e2e_step()
        et = []
        for _ in range(args.steps):
            flush.fill_(1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e2e_step()
            torch.cuda.synchronize()
            et.append(time.perf_counter() - t0)
        e2e_s = max_over_ranks(sum(et), dist, "cuda")
        e2e = {"value": job_throughput(edges, args.steps, ws, e2e_s), "unit": UNIT,
               "h2d_bytes_per_step": int(h_off.numel() * 8 + h_tgt.numel() * 4 + h_w.numel() * 4),
               "d2h_bytes_per_step": int(h_C.numel() * 4)}
        del h_off, h_tgt, h_w, h_C
    workspace = {"peak_bytes_per_call": st.get("workspace_bytes"), "reserved_bytes": gsp.workspace_reserved()}
    gsp.release_workspace()  # the untimed runs below regrow what they need

    log("timed %d steps: %.1f ms/step; e2e %s" % (args.steps, total_ms / args.steps, e2e and e2e["value"]))
    learned = None
    if args.learned == "on" or (args.learned == "auto" and args.workload.startswith("rmat") and gvo is None):
        learned = learned_compare(gsp, args, off, tgt, w, kw, flush, stream, total_ms / args.steps, q, st, edges,
                                  cfg["workload"])
    gsp.release_workspace()
    main_quality = None if args.no_quality else quality(gsp, off, tgt, w, gvo, kw, q, golden, cfg)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if args.precision == "mixed" else "f64",
            "data": "synthetic (device-generated R-MAT / planted / grid, seeded)",
            "config": dict(cfg, precision=args.precision, split=args.split, move=args.move,
                           waves=args.waves or (17 if args.move == "sync" else 64),
                           wave_repeats=kw["wave_repeats"], parallelism="replicas" if ws > 1 else "single",
                           l2="inputs larger than L2 plus a 256 MB flush between steps"),
            "modularity": q, "communities": st["final_communities"], "passes": st["passes"],
            "quality": main_quality,
            "pass_stats": {k: st[k] for k in ("iterations", "vertices", "communities", "edges", "ms_move",
                                                "ms_split", "ms_aggregate", "ms_other")},
            "phase_ms": {"move": sum(st["ms_move"]), "split": sum(st["ms_split"]),
                         "aggregate": sum(st["ms_aggregate"]), "other": sum(st["ms_other"]),
                         "total": st["ms_total"]},
            "roofline": roofline_from(stats, peak, kind, args.workload), "gpu_launches": launches, "workspace": workspace,
            "phase_roofline": phase_rooflines(st, peak), "learned": learned, "tuning": tuning,
            "clocks": clocks, "e2e": e2e}

    # the other workloads: fewer steps each, untimed quality runs beside them
    names = [] if args.configs == "none" else (list(EXTRA_CONFIGS) if args.configs == "all"
                                                else [x for x in args.configs.split(",") if x])
    names = [x for x in names if x != args.workload]
    if names and ws == 1:  # replicas (N > 1) time the main workload only
        del off, tgt, w, C
        log("main workload done: %.1f ms/step, Q %.5f" % (total_ms / args.steps, q))
        configs = {}
        for name in names:
            gsp.release_workspace()
            torch.cuda.empty_cache()
            ckw = dict(kw, wave_repeats=wave_repeats_for(name, args))
            summ, _ = run_workload(gsp, graphgen, name, ckw, args.config_steps, 2, flush, stream, peak, kind, golden,
                                   autotune=not args.no_autotune and not args.caps)
            configs[summ["config"]["workload"]] = summ
            log("%s: %.2f ms/step, Q %.5f" % (name, summ["ms_per_step"], summ["modularity"]))
            torch.cuda.empty_cache()
        line["configs"] = configs
    if args.leiden != "none" and ws == 1:
        # the GSP-Leiden variant (refinement of Section 3.5) on one workload,
        # beside the GSP-Louvain run of the same graph
        gsp.release_workspace()
        torch.cuda.empty_cache()
        lkw = dict(kw, refine=True, refine_theta=0.01, seed=0)
        summ, extra = run_workload(gsp, graphgen, args.leiden, lkw, args.config_steps, 2, flush, stream, peak, kind,
                                   golden, autotune=not args.no_autotune and not args.caps)
        st_l = extra[7]
        summ["variant"] = "GSP-Leiden: refinement (Section 3.5, theta 0.01, seed 0) after each pass's split"
        summ["refined_communities"] = st_l["refined"]
        summ["ms_refine"] = round(sum(st_l["ms_refine"]), 3)
        if "oracle_modularity" in summ:
            summ["oracle_gsp_louvain_modularity"] = summ.pop("oracle_modularity")
            if "dQ_vs_oracle" in summ:
                summ["dQ_vs_oracle_gsp_louvain"] = summ.pop("dQ_vs_oracle")
        plain = (line.get("configs") or {}).get(summ["config"]["workload"])
        if plain is None and summ["config"]["workload"] == line["config"]["workload"]:
            plain = {"modularity": q, "ms_per_step": line["ms_per_step"]}
        if plain:
            summ["gsp_louvain_modularity"] = plain["modularity"]
            summ["dQ_vs_gsp_louvain"] = summ["modularity"] - plain["modularity"]
            summ["time_vs_gsp_louvain"] = summ["ms_per_step"] / plain["ms_per_step"]
        line["gsp_leiden"] = summ
        log("gsp_leiden %s: %.2f ms/step, Q %.5f" % (args.leiden, summ["ms_per_step"], summ["modularity"]))
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
