"""Benchmark: Brandes samples/s and GTEPS on undirected R-MAT scale 20.

Workload (one step): on the resident R-MAT scale-20 graph (edge factor 16,
a=0.57 b=0.19 c=0.19, seed 2; int32 CSR, symmetrised and deduplicated):
  * Bader's adaptive source sampling, c = 5, 512 uniform targets, cap n/20
    draws (Sec. 4), and
  * a uniform 4096-source all-vertex estimate,
each with its own draw stream (a fresh qid per step, so nothing is reused).
A sample is one per-source Brandes step (forward BFS with sigma + backward
dependency accumulation). samples = (largest k over the Bader targets) + 4096;
draws computed past the last target's stop inside the final batch are not
counted. GTEPS counts, per sample, the undirected edges of the source's
connected component.

Timing: CUDA events on the stream the library launches on, after W warm-up
steps, K timed steps bracketed by (barrier +) synchronize; max over ranks.
Inputs exceed L2 (CSR 134 MB, per-batch lane state 0.6 GB), so no L2 flush.
`e2e` repeats the step through the C ABI with host buffers: the CSR upload,
both queries and their result downloads are inside the timed region.

--impl reference times the CPU oracle (single-threaded C) on a bounded
sample of the same workload (the first Bader draws), same metric and unit.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SCALE, EF, A, B, C, SEED = 20, 16, 0.57, 0.19, 0.19, 2
T_TARGETS, C_BADER, K_UNIFORM = 512, 5.0, 4096
WORKLOAD = "rmat_s20_ef16_bader_c5_T512_capn20_plus_uniform_k4096"
METRIC = "Brandes samples/s (R-MAT s20, batched 64-wide)"


def rank_qids(rank: int, steps: int, warmup: int):
    """Query ids of one rank: (warm-up qids, timed qids). Each step uses two
    streams (Bader, uniform); ranks never share a stream, so N ranks do N times
    the work of one (weak scaling) with no data exchanged between them."""
    base = 1_000_000 * (rank + 1)
    warm = [base + 2 * i for i in range(warmup)]
    timed = [base + 2 * (warmup + i) for i in range(steps)]
    return warm, timed


def reduce_over_ranks(dist, device, ms: float, samples: float, edges: float):
    """Max of the timed region over ranks; sums of samples and edges."""
    if dist is None:
        return ms, samples, edges
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([samples, edges], dtype=torch.float64, device=device)
    dist.all_reduce(u)
    return float(t[0]), float(u[0]), float(u[1])


def recorded_traffic():
    """DRAM bytes per algorithmic byte of the backward kernels, from the committed
    ncu summary (a capture of every backward launch of a reduced-cap run on the
    same graph, divided by that run's own algorithmic bytes), or None when the
    kernel source has changed since the counters were taken."""
    import hashlib
    try:
        txt = open(os.path.join(ROOT, "profiles", "bwd_traffic_rmat_s20.md")).read()
        val = float(txt.split("traffic_per_algorithmic_byte:")[1].split()[0])
        sha = txt.split("sha256/16 = ")[1].split()[0]
        cur = hashlib.sha256(open(os.path.join(ROOT, "paper_1608_04472_gb300", "csrc", "bc_batch.cu"),
                                  "rb").read()).hexdigest()[:16]
        return val if cur == sha else None
    except Exception:
        return None


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def build_graph():
    import graphgen as gg
    return gg.rmat(SCALE, EF, A, B, C, SEED)


def component_edges(g):
    """Undirected edges of each vertex's connected component (for TEPS)."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    adj = sp.csr_matrix((np.ones(g.nnz, np.int8), g.col, g.row_ptr), shape=(g.n, g.n))
    ncomp, labels = connected_components(adj, directed=False)
    comp_nnz = np.bincount(labels, weights=g.degrees(), minlength=ncomp)
    return (comp_nnz / 2.0)[labels]


def run_reference(args):
    """CPU oracle on a bounded sample of the same workload."""
    import graphgen as gg
    import oracle
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    g = build_graph()
    targets = gg.uniform_targets(g.n, T_TARGETS, SEED)
    per_step = 4  # oracle per-sample Brandes steps per bench step
    ce = component_edges(g)
    n = g.n
    for w in range(args.warmup):
        oracle.adaptive_sources(g, targets, C_BADER, 1, SEED, 1000 + w)
    t0 = time.perf_counter()
    edges = 0.0
    for st in range(args.steps):
        qid = 2000 + st
        oracle.adaptive_sources(g, targets, C_BADER, per_step, SEED, qid)
        for i in range(per_step):
            edges += ce[oracle.draw_source(SEED, qid, i, n)]
    dt = time.perf_counter() - t0
    samples = per_step * args.steps
    value = samples / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "samples/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "graph": f"rmat s{SCALE} ef{EF} seed {SEED}",
                   "reference": "CPU oracle (oracle/bc_oracle.c), single thread",
                   "sample": f"{per_step} Bader draws per step (full per-sample Brandes step each)"},
        "gteps": edges / dt / 1e9,
        "cpu_baseline": {"value": value, "unit": "samples/s", "cores": 1, "kind": "oracle",
                         "sample": f"first {per_step} draws of the Bader stream per step, {args.steps} steps"},
        "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def cpu_baseline(g, targets, budget_s=12.0):
    """The oracle timed on a bounded sample: Bader draws until ~budget_s."""
    import oracle
    n = g.n
    oracle.dependencies(g, 0)  # warm the library
    t0 = time.perf_counter()
    k = 0
    while time.perf_counter() - t0 < budget_s and k < 64:
        oracle.dependencies(g, oracle.draw_source(SEED, 999, k, n))
        k += 1
    dt = time.perf_counter() - t0
    return {"value": k / dt, "unit": "samples/s", "cores": 1, "kind": "oracle",
            "sample": f"{k} per-sample Brandes steps (Bader draws of R-MAT s20), single-threaded C"}


def cpu_multicore(g, budget_s=10.0):
    """The same oracle routine on every host core at once (one sample per
    thread; the C call releases the interpreter lock), reported beside the
    single-core oracle figure."""
    import concurrent.futures as cf
    import oracle
    n = g.n
    cores = os.cpu_count() or 1
    oracle.dependencies(g, 0)
    t0 = time.perf_counter()
    done = 0
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        i = 0
        while time.perf_counter() - t0 < budget_s and i < 16 * cores:
            futs = [ex.submit(oracle.dependencies, g, oracle.draw_source(SEED, 998, i + j, n)) for j in range(cores)]
            for f in futs:
                f.result()
            i += cores
            done += cores
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "samples/s", "cores": cores, "kind": "oracle, all host cores",
            "sample": f"{done} per-sample Brandes steps (source draws of R-MAT s20), one per thread"}


def cpu_small_configs(budget_s=3.0):
    """The single-threaded oracle on the two small workloads it also runs in
    full in the tests: per-sample Brandes steps on ER n=2000 (average degree 8,
    seed 1) and Algorithm 1 pair draws on BA n=20,000 (4 edges per new vertex,
    seed 3; one BFS from s per draw and target)."""
    import graphgen as gg
    import oracle
    out = {}
    er = gg.erdos_renyi(2000, 8, 1)
    oracle.dependencies(er, 0)
    t0, k = time.perf_counter(), 0
    while time.perf_counter() - t0 < budget_s and k < 20000:
        oracle.dependencies(er, oracle.draw_source(SEED, 997, k, er.n))
        k += 1
    out["er2000_samples_per_s"] = k / (time.perf_counter() - t0)
    ba = gg.barabasi_albert(20000, 4, 3)
    t = int(gg.degree_targets(ba, 1, 3)[0])
    t0, k = time.perf_counter(), 0
    while time.perf_counter() - t0 < budget_s and k < 20000:
        oracle.pair_sequence(ba, t, SEED, 996, k, 16)
        k += 16
    out["ba20k_pair_draws_per_s"] = k / (time.perf_counter() - t0)
    out["cores"] = 1
    return out


def oracle_pair_rate(g, targets, draws=4):
    """The oracle's marginal cost of a pair draw of Algorithm 1 (one BFS from s)
    on one host core: a run of `draws` draws minus a run of one, same stream."""
    import oracle
    t0 = time.perf_counter()
    oracle.adaptive_pairs(g, targets[:1], 1.0, 1, 3, 2)
    t1 = time.perf_counter()
    oracle.adaptive_pairs(g, targets[:1], 1.0, draws, 3, 2)
    t2 = time.perf_counter()
    return (draws - 1) / max(1e-9, (t2 - t1) - (t1 - t0))


def measure_pairs(pkg, torch, local, stream, caps=(2048, 16384), T=256, n=2_000_000):
    """Algorithm 1 on BA n=2,000,000 (4 edges per new vertex, seed 3) with 256
    degree-proportional targets and the paper's threshold c*n (c=1): every
    target runs to the cap, so a run is `cap` pair draws plus one BFS per
    target. Timed at two caps, so that the marginal cost of a pair draw is
    separated from the targets' BFS, for the bidirectional pair search (the
    default: one pair per CTA), the same search one pair per warp with large
    balls handed to the CTA form (BCG_PAIR_ENGINE=2) and the one-sided BFS
    truncated at t's level (BCG_PAIR_ENGINE=1).
    Returns pair draws per second."""
    import graphgen as gg
    g = gg.barabasi_albert(n, 4, 3)
    targets = gg.degree_targets(g, T, 3)
    out = {"workload": f"BA n={n} m=4 seed 3, {T} degree-proportional targets, c=1 (threshold c*n), "
                       f"caps {caps[0]} and {caps[1]}"}
    prev = os.environ.get("BCG_PAIR_ENGINE")
    try:
        for engine, name in (("0", "bidirectional"), ("2", "bidirectional_warp"), ("1", "one_sided")):
            os.environ["BCG_PAIR_ENGINE"] = engine  # read when the context is made
            ctx = pkg.Context(local, batch_width=64, stream=stream.cuda_stream)
            h = ctx.load_graph(g.row_ptr, g.col)
            ctx.adaptive_pairs(h, targets[:8], 1.0, 64, 3, 1)  # warm-up
            ms = []
            for cap in caps:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                res = ctx.adaptive_pairs(h, targets, 1.0, cap, 3, 2)
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
                assert int((res["status"] == 1).sum()) == T  # every target ran to the cap
            # per-family device time of the longer run (profiling on: not a timed number)
            ctx.set_profiling(True)
            ctx.reset_stats()
            ctx.adaptive_pairs(h, targets, 1.0, caps[1], 3, 2)
            st = ctx.stats()
            # vertices in the two balls per pair: the counter also takes the
            # target's BFS, so a one-draw run is subtracted
            ctx.reset_stats()
            ctx.adaptive_pairs(h, targets[:1], 1.0, 1, 3, 2)
            r1 = ctx.stats()["reached"]
            ctx.reset_stats()
            ctx.adaptive_pairs(h, targets[:1], 1.0, caps[1], 3, 2)
            rk = ctx.stats()["reached"]
            ctx.set_profiling(False)
            ctx.close()
            out[name] = {"ms": ms, "pair_draws_per_s_with_targets": caps[0] / (ms[0] / 1e3),
                         "pair_draws_per_s_marginal": (caps[1] - caps[0]) / ((ms[1] - ms[0]) / 1e3),
                         "profile_cap": caps[1],
                         "family_ms": {k: round(v["ms"], 2) for k, v in st["kernels"].items() if v["launches"]},
                         "family_launches": {k: v["launches"] for k, v in st["kernels"].items() if v["launches"]}}
            if engine != "1":
                out[name]["ball_vertices_per_pair"] = (rk - r1) / (caps[1] - 1)
                out[name]["pairs_to_cta_search"] = st["pair_fallbacks"]
    finally:
        if prev is None:
            os.environ.pop("BCG_PAIR_ENGINE", None)
        else:
            os.environ["BCG_PAIR_ENGINE"] = prev
    out["oracle_1core_pair_draws_per_s"] = oracle_pair_rate(g, targets)
    out["pair_draws_per_s"] = out["bidirectional"]["pair_draws_per_s_with_targets"]
    out["marginal_speedup"] = (out["bidirectional"]["pair_draws_per_s_marginal"]
                               / out["one_sided"]["pair_draws_per_s_marginal"])
    out["note"] = "with_targets includes one BFS per target (256) before the pair draws"
    return out


def measure_variants(pkg, torch, local, stream, k=512, scale=SCALE):
    """The uniform k-source estimate (the per-sample step of Sec. 3 summed over
    k draws) on R-MAT s20 with edge lengths 1-100 (weighted engine: near-far
    distances, Kahn rounds over the shortest-path DAG) and on R-MAT s20 read
    as a directed graph (lane-major engine, counts pulled over the
    in-neighbour CSR), each beside the same graph's unit-length/undirected
    figure and the oracle on one host core for a few draws of the same
    stream."""
    import graphgen as gg
    import oracle
    g = gg.rmat(scale, EF, A, B, C, SEED)
    w = gg.edge_lengths(g, 1, 100, 9)
    gd = gg.directed_rmat(scale, EF, A, B, C, SEED)
    out = {"k": k, "scale": scale}

    def timed(ctx, h):
        ctx.uniform_sources(h, 64, 1, 1)  # warm-up (scratch sized once)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.uniform_sources(h, k, 3, 4)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    def oracle_rate(fn, n_draws=3):
        t0 = time.perf_counter()
        for i in range(n_draws):
            fn(oracle.draw_source(3, 4, i, g.n))
        return n_draws / (time.perf_counter() - t0)

    ctx = pkg.Context(local, batch_width=64, stream=stream.cuda_stream)
    hw = ctx.load_graph(g.row_ptr, g.col, lengths=w)
    ms_w = timed(ctx, hw)
    ctx.free_graph(hw)
    h1 = ctx.load_graph(g.row_ptr, g.col, lengths=np.ones(g.col.shape[0], np.uint32))
    ms_1 = timed(ctx, h1)
    ctx.free_graph(h1)
    hd = ctx.load_graph(gd.row_ptr, gd.col, directed=True)
    ms_d = timed(ctx, hd)
    ctx.close()
    out["weighted"] = {
        "workload": f"R-MAT s{scale} (seed {SEED}), lengths uniform 1-100 (graphgen.edge_lengths seed 9), "
                    f"uniform k={k}",
        "samples_per_s": k / (ms_w / 1e3), "ms": ms_w,
        "unit_lengths_samples_per_s": k / (ms_1 / 1e3),
        "oracle_1core_samples_per_s": oracle_rate(lambda s: oracle.dependencies_w(g, w, s))}
    out["directed"] = {
        "workload": f"R-MAT s{scale} edges read row -> column (seed {SEED}, {gd.col.shape[0]} arcs), uniform k={k}",
        "samples_per_s": k / (ms_d / 1e3), "ms": ms_d,
        "oracle_1core_samples_per_s": oracle_rate(lambda s: oracle.dependencies(gd, s))}
    return out


def measure_uneven(pkg, torch, local, stream, k=1024, reps=2, count=256, n_hi=200000):
    """Uniform 1024-draw estimates for 256 graphs of uneven size and depth
    (log-uniform 2k-200k vertices; ER, R-MAT ef 8 or 2D grid, from base seed 6)
    in one bc_uniform_sources_multi call: deep graphs on the persistent kernel,
    shallow ones beside it on the batched engine. Compared with one
    bc_uniform_sources call per graph on every 4th graph (the same graphs
    through both paths)."""
    import graphgen as gg
    S = gg.uneven_set(count=count, n_hi=n_hi)
    G = len(S)
    seeds = [6000 + i for i in range(G)]
    qids = list(range(G))
    ctx = pkg.Context(local, batch_width=64, stream=stream.cuda_stream)
    hs = [ctx.load_graph(g.row_ptr, g.col) for _, g in S]

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3, r

    ctx.uniform_sources_multi(hs, [k] * G, seeds, qids)  # warm-up: hub distances, plan, captured graph
    best = min(timed(lambda: ctx.uniform_sources_multi(hs, [k] * G, seeds, qids))[0] for _ in range(reps))
    sub = list(range(0, G, 4))
    hsub = [hs[i] for i in sub]
    ssub = [seeds[i] for i in sub]
    qsub = [qids[i] for i in sub]
    ctx.uniform_sources_multi(hsub, [k] * len(sub), ssub, qsub)
    t_multi, out_m = timed(lambda: ctx.uniform_sources_multi(hsub, [k] * len(sub), ssub, qsub))
    t_per, out_p = timed(lambda: [ctx.uniform_sources(h, k, s_, q) for h, s_, q in zip(hsub, ssub, qsub)])
    same = all(np.array_equal(a, b) for a, b in zip(out_m, out_p))
    fam = {f: sum(1 for x, _ in S if x == f) for f in ("er", "rmat", "grid")}
    # algorithmic bytes per sample, lane-major: per directed edge and pass
    # (discovery, count pull, dependency pull) a 4 B column and a 4 B distance;
    # per vertex an 8 B count, an 8 B coefficient and an 8 B partial sum
    alg = sum(k * (3 * 8 * g.nnz + 24 * g.n) for _, g in S)
    ctx.close()
    return {"workload": f"{G} graphs (ER {fam['er']}, R-MAT {fam['rmat']}, grid {fam['grid']}), "
                        f"{sum(g.n for _, g in S)} vertices, {k} draws each",
            "samples_per_s": G * k / best, "seconds": best,
            "algorithmic_gb_per_s": alg / best / 1e9,
            "per_graph_subset": {"graphs": len(sub), "one_call_s": t_multi, "per_graph_calls_s": t_per,
                                 "speedup": t_per / t_multi, "identical_estimates": bool(same)}}


def measure_serving(pkg, g, h_ctx, rng_seed=7, nq=48, cap=1024, graphs=None, label=None):
    """Continuous batching on resident graphs: a mix of Bader queries (75 %) and
    pair queries (25 %), each on a graph chosen uniformly (default: the one
    graph g), 1-64 uniform targets, c in {2, 5, 10}, cap draws each. Saturation
    rate from submitting all at once, then Poisson arrivals at 0.5 and 0.8 of
    it; latency = submit -> result written."""
    import graphgen as gg
    ctx, h = h_ctx
    graphs = graphs or [(g, h)]
    rng = np.random.default_rng(rng_seed)
    specs = []
    for i in range(nq):
        T = int(rng.integers(1, 65))
        gi = int(rng.integers(0, len(graphs)))
        gq, hq = graphs[gi]
        specs.append(dict(h=hq, kind=pkg.BC_QUERY_PAIRS if rng.random() < 0.25 else pkg.BC_QUERY_SOURCES,
                          targets=gg.uniform_targets(gq.n, T, 1000 + i), c=float(rng.choice([2.0, 5.0, 10.0])),
                          cap=cap, seed=SEED, qid=5_000_000 + i))

    def run(rate, subset=None):
        tks = []
        t0 = time.perf_counter()
        for i, sp in enumerate(specs[:subset] if subset else specs):
            if rate:
                time.sleep(float(rng.exponential(1.0 / rate)))
            kw = dict(sp)
            kw["qid"] = sp["qid"] + int(rate * 1000)
            hq = kw.pop("h")
            tks.append(ctx.submit(hq, kw.pop("kind"), **kw))
        for tk in tks:
            ctx.poll(tk, -1)
        wall = time.perf_counter() - t0
        lat = np.array([tk.stats.queue_ms + tk.stats.run_ms for tk in tks])
        samples = sum(int(tk.stats.samples) for tk in tks)
        return wall, lat, samples

    run(0, subset=min(nq, 48))  # warm-up (per-query state allocation paths)
    wall, lat, samples = run(0)
    lam = nq / wall
    out = {"workload": f"{label or 'R-MAT s20'} resident; {nq} queries, 75% Bader / 25% pairs, 1-64 targets, "
                       f"c in {{2,5,10}}, cap {cap}",
           "saturation_queries_per_s": lam, "saturation_samples_per_s": samples / wall,
           "saturation_p50_ms": float(np.percentile(lat, 50)), "saturation_p99_ms": float(np.percentile(lat, 99))}
    for frac in (0.5, 0.8):
        wall, lat, samples = run(frac * lam)
        out[f"load_{frac}"] = {"offered_queries_per_s": frac * lam, "p50_ms": float(np.percentile(lat, 50)),
                               "p99_ms": float(np.percentile(lat, 99)), "samples_per_s": samples / wall}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the pair-sampling (BA 2M), serving-latency and uneven multi-graph measurements")
    ap.add_argument("--cap", type=int, default=0,
                    help="override the Bader cap (default n/20); for short profiling runs only")
    ap.add_argument("--uniform-k", type=int, default=K_UNIFORM,
                    help="override the uniform sample count; for short profiling runs only")
    ap.add_argument("--serving-full", action="store_true",
                    help="run only the serving measurement on resident R-MAT s21 and s22 (about a minute "
                         "of graph generation first) and print its JSON object")
    ap.add_argument("--serving-queries", type=int, default=48, help="queries in the --serving-full stream")
    ap.add_argument("--serving-grid", type=int, default=0,
                    help="also serve a 2D grid of this side in --serving-full (0: none)")
    ap.add_argument("--uneven-only", action="store_true",
                    help="run only the uneven multi-graph measurement and print its JSON object")
    ap.add_argument("--variants-only", action="store_true",
                    help="run only the weighted / directed R-MAT s20 measurements and print them")
    ap.add_argument("--variants-scale", type=int, default=SCALE,
                    help="R-MAT scale of --variants-only (smaller for profiling captures)")
    ap.add_argument("--pairs-only", action="store_true",
                    help="run only the pair-sampling measurement (BA 2M, both pair engines) and print it")
    ap.add_argument("--pairs-n", type=int, default=2_000_000,
                    help="BA size of --pairs-only (smaller for profiling captures)")
    ap.add_argument("--pairs-targets", type=int, default=256, help="targets of --pairs-only")
    ap.add_argument("--uneven-count", type=int, default=256, help="graphs in the uneven workload")
    ap.add_argument("--uneven-nmax", type=int, default=200000, help="largest graph size in the uneven workload")
    ap.add_argument("--sharded", action="store_true",
                    help="share each step's two queries among the ranks (blocks of draws dealt round-robin, "
                         "blocks allgathered, the same stop scan on every rank; strong scaling) instead of "
                         "running independent queries per rank")
    ap.add_argument("--shard-block", type=int, default=1024, help="draws per block with --sharded")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the library's per-graph tuning (bc_autotune) before the warm-up")
    ap.add_argument("--tune-k", type=int, default=512, help="draws per tuning trial")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.serving_full:
        import torch
        import graphgen as gg
        import paper_1608_04472_gb300 as pkg
        torch.cuda.set_device(0)
        t0 = time.perf_counter()
        gs = [gg.rmat(21, EF, 0.57, 0.19, 0.19, 4), gg.rmat(22, EF, 0.57, 0.19, 0.19, 5)]
        if args.serving_grid:
            gs.append(gg.grid(args.serving_grid))
        gen_s = time.perf_counter() - t0
        ctx = pkg.Context(0, batch_width=64, stream=torch.cuda.current_stream().cuda_stream)
        hs = [ctx.load_graph(x.row_ptr, x.col) for x in gs]
        r = measure_serving(pkg, gs[0], (ctx, hs[0]), nq=args.serving_queries, graphs=list(zip(gs, hs)),
                            label="R-MAT s21 (seed 4) + R-MAT s22 (seed 5)"
                                  + (f" + {args.serving_grid}x{args.serving_grid} grid" if args.serving_grid else ""))
        r["graph_generation_s"] = gen_s
        ctx.close()
        print(json.dumps(r))
        return 0
    if args.variants_only:
        import torch
        import paper_1608_04472_gb300 as pkg
        torch.cuda.set_device(0)
        print(json.dumps(measure_variants(pkg, torch, 0, torch.cuda.current_stream(), scale=args.variants_scale)))
        return 0
    if args.pairs_only:
        import torch
        import paper_1608_04472_gb300 as pkg
        torch.cuda.set_device(0)
        print(json.dumps(measure_pairs(pkg, torch, 0, torch.cuda.current_stream(), T=args.pairs_targets,
                                       n=args.pairs_n)))
        return 0
    if args.uneven_only:
        import torch
        import paper_1608_04472_gb300 as pkg
        torch.cuda.set_device(0)
        r = measure_uneven(pkg, torch, 0, torch.cuda.current_stream(), count=args.uneven_count,
                           n_hi=args.uneven_nmax)
        print(json.dumps(r))
        return 0

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.gpus != world:
        print(f"bench.py: --gpus {args.gpus} but WORLD_SIZE={world}; launch N > 1 ranks with "
              f"python -m torch.distributed.run --nproc-per-node {args.gpus} bench.py --gpus {args.gpus}",
              file=sys.stderr)
        return 2
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)

    import graphgen as gg
    import paper_1608_04472_gb300 as pkg

    g = build_graph()
    n = g.n
    cap = args.cap if args.cap > 0 else n // 20
    kuni = args.uniform_k
    targets = gg.uniform_targets(n, T_TARGETS, SEED)
    ce = component_edges(g)

    stream = torch.cuda.current_stream()
    ctx = pkg.Context(local, batch_width=64, stream=stream.cuda_stream)
    h = ctx.load_graph(g.row_ptr, g.col)
    # per-graph launch settings picked by the library's tuner (timed trials of
    # a uniform estimate, results checked bit-identical), outside the timed region
    tuning = ctx.get_tuning(h) if args.no_tune else ctx.autotune(h, args.tune_k, 0xBE7C)

    if args.sharded:
        from paper_1608_04472_gb300 import sharded
        ag, ar = sharded.torch_collectives(dist, "cuda") if dist else (lambda a: [a], lambda a: a)

        def step(qid_base):
            rb = sharded.adaptive_sources_sharded(ctx, h, targets, C_BADER, cap, SEED, qid_base, rank, world, ag,
                                                  B=args.shard_block)
            est = sharded.uniform_sources_sharded(ctx, h, kuni, SEED, qid_base + 1, rank, world, ar,
                                                  B=args.shard_block)
            return rb, est
    else:
        def step(qid_base):
            rb = ctx.adaptive_sources(h, targets, C_BADER, cap, SEED, qid_base)
            est = ctx.uniform_sources(h, kuni, SEED, qid_base + 1)
            return rb, est

    # sharded: every rank works on the same queries (rank 0's streams)
    warm_qids, timed_qids = rank_qids(0 if args.sharded else rank, args.steps, args.warmup)
    for q in warm_qids:
        step(q)
    ctx.reset_stats()
    ctx.set_profiling(True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    kmax, qids = [], []
    for q in timed_qids:
        rb, _ = step(q)
        kmax.append(int(rb["k"].max()))
        qids.append(q)
    qid = timed_qids[-1] + 2 if timed_qids else 0
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    stats = ctx.stats()
    ctx.set_profiling(False)
    samples_local = sum(kmax) + kuni * args.steps
    edges_local = 0.0
    for q, km in zip(qids, kmax):
        edges_local += float(ce[ctx.draw_sources(SEED, q, 0, km, n)].sum())
        edges_local += float(ce[ctx.draw_sources(SEED, q + 1, 0, kuni, n)].sum())
    if args.sharded and rank != 0:  # one shared query: its samples are counted once
        samples_local, edges_local = 0, 0.0
    ms, samples_total, edges_total = reduce_over_ranks(dist, "cuda", ms, float(samples_local), edges_local)
    value = samples_total / (ms / 1e3)

    # roofline of the dominant kernel family (measured live over the timed region)
    peaks, peak_kind = load_peaks()
    kern = stats["kernels"]
    dom = max(("fwd", "bwd"), key=lambda k: kern[k]["ms"])
    lanes_processed = stats["samples"]
    bytes_fwd = 8.0 * stats["dag_edges"] + 8.0 * stats["reached"]
    bytes_bwd = 8.0 * stats["dag_edges"] + 16.0 * stats["reached"]
    alg_bytes = bytes_bwd if dom == "bwd" else bytes_fwd
    dom_ms = kern[dom]["ms"]
    achieved = alg_bytes / (dom_ms / 1e3) / 1e9 if dom_ms > 0 else 0.0
    kern_names = {"bwd": "backward pass: k_bwd_light_fx + k_bwd_heavy_seg_fx + k_bwd_heavy_fin_fx per level",
                  "fwd": "forward pass: k_fwd_light + the heavy-vertex kernels + k_fwd_heavy_fin per level"}
    ratio = recorded_traffic() if dom == "bwd" else None
    alg_per_launch = alg_bytes / max(kern[dom]["launches"], 1)
    roofline = {"bound": "hbm", "kernel": kern_names[dom], "achieved": achieved,
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                # ncu DRAM bytes per algorithmic byte (reduced-cap capture, same graph and
                # kernels) times this run's algorithmic bytes per launch
                "traffic": ratio * alg_per_launch if ratio is not None else None,
                "traffic_per_algorithmic_byte": ratio, "peak_kind": peak_kind,
                "launches": kern[dom]["launches"], "avg_launch_ms": dom_ms / max(kern[dom]["launches"], 1),
                "alg_bytes_per_launch": alg_bytes / max(kern[dom]["launches"], 1),
                "dag_edges_per_sample": stats["dag_edges"] / max(lanes_processed, 1),
                "reached_per_sample": stats["reached"] / max(lanes_processed, 1)}
    gpu_launches = int(stats["launches"])

    out = {
        "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "strong" if args.sharded else "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "graph": f"R-MAT s{SCALE} ef{EF} a{A} b{B} c{C} seed {SEED}",
                   "n": n, "nnz": g.nnz, "targets": T_TARGETS, "c": C_BADER, "cap": cap,
                   "uniform_k": kuni, "batch_width": int(tuning["batch_width"]),
                   "tuning": {k: v for k, v in tuning.items() if k != "trial_ms"},
                   "tuned": not args.no_tune,
                   "parallelism": (f"one query sharded x{world} (blocks of {args.shard_block} draws)"
                                   if args.sharded else f"replicas x{world}"),
                   "l2": "inputs larger than L2 (CSR 134 MB + 0.6 GB lane state); no flush"},
        "gteps": edges_total / (ms / 1e3) / 1e9,
        "samples_per_step": samples_total / args.steps,
        "lane_samples_computed": lanes_processed,
        "kernel_ms": {k: round(v["ms"], 3) for k, v in kern.items() if v["launches"]},
        "roofline": roofline,
        "gpu_launches": gpu_launches,
        "clocks": clk,
    }

    if rank == 0 and not args.no_plain:
        # plain (one source per launch sequence) vs batched on the same uniform query
        kq = 256
        # the graph's tuning overrides the context's width: width 1 goes through it
        tun = ctx.get_tuning(h)
        ctx.set_tuning(h, dict(tun, batch_width=1))
        ctx.uniform_sources(h, 8, SEED, 7)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        est_plain = ctx.uniform_sources(h, kq, SEED, 77)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_plain = e0.elapsed_time(e1)
        ctx.set_tuning(h, tun)
        e0.record(stream)
        est_b = ctx.uniform_sources(h, kq, SEED, 77)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_b = e0.elapsed_time(e1)
        out["plain"] = {"workload": f"uniform k={kq} on the same graph",
                        "plain_samples_per_s": kq / (ms_plain / 1e3),
                        "batched_samples_per_s": kq / (ms_b / 1e3),
                        "speedup": ms_plain / ms_b,
                        "identical_estimates": bool(np.array_equal(est_plain, est_b))}

    if rank == 0 and world == 1 and not args.no_extra:
        out["serving"] = measure_serving(pkg, g, (ctx, h))
        out["pairs"] = measure_pairs(pkg, torch, local, stream)
        out["uneven"] = measure_uneven(pkg, torch, local, stream)

    if not args.no_e2e:
        e2e_steps = max(1, min(2, args.steps))
        h2d = g.row_ptr.nbytes + g.col.nbytes + targets.nbytes
        d2h = T_TARGETS * (8 + 8 + 8 + 4) + n * 8
        ctx.free_graph(h)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        samp = 0
        for _ in range(e2e_steps):
            h2 = ctx.load_graph(g.row_ptr, g.col)
            ctx.set_tuning(h2, tuning)  # the choice made once for this graph (a user caches it likewise)
            if args.sharded:
                rb = sharded.adaptive_sources_sharded(ctx, h2, targets, C_BADER, cap, SEED, qid, rank, world, ag,
                                                      B=args.shard_block)
                sharded.uniform_sources_sharded(ctx, h2, kuni, SEED, qid + 1, rank, world, ar, B=args.shard_block)
            else:
                rb = ctx.adaptive_sources(h2, targets, C_BADER, cap, SEED, qid)
                ctx.uniform_sources(h2, kuni, SEED, qid + 1)
            samp += int(rb["k"].max()) + kuni
            ctx.free_graph(h2)
            qid += 2
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e_val = samp / dt
        if dist:
            t = torch.tensor([dt], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            # replicas: every rank ran its own queries; sharded: one query per step
            e2e_val = samp * (1 if args.sharded else world) / float(t.item())
        out["e2e"] = {"value": e2e_val, "unit": "samples/s", "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(d2h), "steps": e2e_steps}
    else:
        ctx.free_graph(h)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(g, targets)
        out["cpu_multicore"] = cpu_multicore(g)
        out["cpu_small_configs"] = cpu_small_configs()
    ctx.close()
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
