"""Benchmark of the temporal 3-path sampling estimator on one GB300.

A step is one pass of the whole hot path over the resident graph: path
weights and their exact prefix sum with the sampling index (Claim 1, Alg. 1),
then k sampled 3-paths with CheckMotif / ListCount and the reduction of the
estimate (Alg. 2-5).  The workload is the 20M-edge Chung-Lu graph (n = 1M,
power-law exponent 2.1, maximum degree ~1e5, 30% multi-edges, bursty times
over 1e8 s) with the path+chord motif a->b, b->c, c->d, a->d (in that time
order), delta = 3600 s and k = 1e8 samples per step.

Printed: one JSON line with samples/s (device, graph resident), the same
metric end to end through tc_estimate_from_host with pinned host buffers, the
roofline of the dominant kernel (the sampler), the oracle's CPU rate and the
SM clocks seen during the timed region.

``--impl reference`` times the CPU oracle instead (the reference arm).
Under torchrun each rank runs the full path on its own GPU over its own
sample-id range (weak scaling); the integer sums merge exactly afterwards.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "temporal-path samples/sec"
MOTIFS = {  # name -> edges in time-rank order
    "c4": [(0, 1), (1, 2), (2, 3), (3, 0)],             # directed 4-cycle (M4-0)
    "path_chord": [(0, 1), (1, 2), (2, 3), (0, 3)],     # a->b, b->c, c->d, then a->d
    "ff_triangle": [(0, 1), (0, 2), (1, 2)],            # 3-vertex: a->b, a->c, b->c (wedge anchor <+,>>)
    "cyclic_triangle": [(0, 1), (1, 2), (2, 0)],        # 3-vertex: a->b, b->c, c->a
}
MOTIF_NAMES = {str(v): k for k, v in MOTIFS.items()}
# DRAM bytes (read + write) per sample of the sampler kernel, from one ncu
# capture of the benchmark's own launch (dram__bytes_read.sum +
# dram__bytes_write.sum over two 1e8-sample launches); valid while the kernel
# is unchanged, null for workloads that were not captured
SAMPLER_TRAFFIC_PER_SAMPLE = {("mid", "path_chord"): 79.3}
UNIT = "samples/s"
SECTOR = 32


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--samples", type=int, default=None, help="samples per step (default: the config's k)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--exact-max-paths", type=float, default=2e11,
                    help="run the exhaustive exact count when W is at most this")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-proposal comparison")
    ap.add_argument("--train-samples", type=int, default=10_000_000)
    ap.add_argument("--stats-samples", type=int, default=None,
                    help="plain samples behind the sample-statistics features (default: --train-samples)")
    ap.add_argument("--eps", type=float, default=0.05, help="the learned proposal's mixture weight: q ~ w (eps + g)")
    ap.add_argument("--objective", default="both", choices=["closure", "variance", "both"],
                    help="training objective of the learned proposal (both: one comparison each, "
                         "the closure loss under 'learned', the variance objective under 'learned_variance')")
    ap.add_argument("--motif", default=None, choices=sorted(MOTIFS),
                    help="another motif on the workload's graph (default: the workload's own)")
    ap.add_argument("--workload", default="mid", choices=["mid", "learned", "large", "batch", "small", "batch_small"],
                    help="mid: the 20M-edge graph (default); learned: n=2e7, m=1e8; large: n=1e8, m=3e8")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def workload(name="mid"):
    from paper_2409_08975_gb300 import synth
    return synth.CONFIGS[name]()


WORKLOADS = {
    "mid": "mid: Chung-Lu-weighted bursty graph n=1M m=20M gamma=2.1 max_deg~1e5 30% multi-edges over 1e8 s; "
           "motif a->b,b->c,c->d,a->d (path+chord), delta=3600, k=1e8 samples per step",
    "learned": "learned: the mid generator at n=20M m=100M; path+chord, delta=3600, k=1e8 samples per step; "
               "learned proposal trained on 1e7 plain samples",
    "large": "large: n=100M m=300M, top degree ~1e6, pair multiplicities Zipf(1.8), daily periodicity over 1e8 s; "
             "directed 4-cycle (M4-0), delta=3600, k=1e9 samples per step",
    "small": "small (profiling case): the mid generator at n=5e5 m=1e7; path+chord, delta=3600, k=1e7",
    "batch_small": "batch_small (profiling case): as batch with a 1e7-edge big graph, 8 small graphs and 1e5-1e7 "
                   "samples per query",
    "batch": "batch: 136 queries in one persistent launch replayed from a CUDA graph; a 50M-edge graph of the mid "
             "generator (n=2.5M) with all 24 time-rank orders of the directed 4-cycle x delta in {600, 3600, 86400}, "
             "plus 64 graphs of 1e4-2e6 edges (log-uniform) with one query each; 1e6-1e8 samples per query "
             "(log-uniform), ~2.5e9 samples per step",
}


def cpu_baseline(cfg, k_total, sample_k=300_000):
    """The oracle as it stands on the host cores: weights and prefix over the
    whole graph timed in full, the sampler timed on sample_k samples and
    scaled to k_total samples per step."""
    import oracle
    og = oracle.build_csr(cfg["n"], cfg["src"], cfg["dst"], cfg["t"], sort="lexsort")
    plan = oracle.compile_motif(cfg["motif"])
    t0 = time.perf_counter()
    w = oracle.path_weights(og, plan, cfg["delta"])["w"]
    pre = oracle.prefix_sum(w)
    t_prep = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.sample_run(og, plan, cfg["delta"], pre, sample_k, 0, 0)
    t_samp = time.perf_counter() - t0
    per = t_samp / sample_k
    value = k_total / (t_prep + per * k_total)
    return {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "serial C oracle: weights+prefix over all %d edges timed in full (%.2f s); sampler timed "
                      "on %d samples (%.2f s) and scaled to k=%d per step" % (og.m, t_prep, sample_k, t_samp,
                                                                               k_total)}, og, plan, pre


def run_reference(args, rank, world):
    if rank != 0:
        return
    cfg = workload(args.workload)
    k = args.samples or cfg["k"]
    if args.workload in ("batch", "batch_small"):  # the oracle on the big graph's first query, scaled
        gi, edges, delta = cfg["queries"][0][:3]
        cfg = dict(cfg["graphs"][gi], name=args.workload, motif=edges, delta=delta)
    elif args.motif:
        cfg["motif"], cfg["motif_override"] = MOTIFS[args.motif], args.motif
    import oracle
    og = oracle.build_csr(cfg["n"], cfg["src"], cfg["dst"], cfg["t"], sort="lexsort")
    plan = oracle.compile_motif(cfg["motif"])
    t0 = time.perf_counter()
    pre = oracle.prefix_sum(oracle.path_weights(og, plan, cfg["delta"])["w"])
    t_prep = time.perf_counter() - t0
    step_k = 100_000
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.sample_run(og, plan, cfg["delta"], pre, step_k, 0, s * step_k)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    per = sum(times) / (len(times) * step_k)
    step_s = t_prep + per * k
    value = k / step_s
    sample = ("serial C oracle on the host: weights+prefix over all %d edges once (%.2f s), each step %d samples "
              "(%.3f s mean), scaled to k=%d samples per step" % (og.m, t_prep, step_k, per * step_k, k))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": config_dict(cfg, k, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


BUDGET_SEEDS = (1, 2, 3, 4, 5)


def run_errors(tc, g, mot, delta, wts, C, k, prop=None):
    """|C_hat - C| / C of independent runs of k samples, one per seed of
    BUDGET_SEEDS, with the plain proposal or the learned one (prop)."""
    errs = []
    for s in BUDGET_SEEDS:
        r = (tc.tc_sample_estimate(g, mot, delta, wts, k, seed=s) if prop is None
             else tc.tc_sample_estimate_q(g, mot, delta, wts, prop, k, seed=s))
        errs.append(abs(r["estimate"] - C) / C)
    return errs


def learned_comparison(tc, g, mot, delta, wts, k, plain, plain_sampler_ms, weights_ms, n_train, stream,
                       objective="closure", exact_C=None, plain_errors=None, n_stats=None, eps=0.05):
    """Learned proposal q ~ w (eps + g) against the plain q ~ w on the same
    graph: features, training on n_train plain samples and the proposal are
    timed once; then k samples with the proposal.  Relative error at a fixed
    GPU time follows from the per-sample variance (k SE^2) and the GPU time
    per sample of each sampler; with the exact count C, also as the mean
    relative error of five seeds' runs at the GPU time of k plain samples."""
    import torch

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        out = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return out, a.elapsed_time(b)

    feat, feat_ms = timed(lambda: tc.tc_edge_features(g, mot, delta, wts))
    # sample statistics from n_stats plain samples (default n_train) of another seed than the training paths
    n_stats = n_stats or n_train
    _, sfeat_ms = timed(lambda: tc.tc_sample_features(g, mot, delta, wts, feat, n_stats, seed=777))
    mlp = tc.MLP(seed=1)
    losses, train_ms = timed(lambda: tc.tc_mlp_train(mlp, g, mot, delta, wts, feat, n_train, seed=12345,
                                                     batch=16384, lr=3e-3, objective=objective, eps=eps))
    prop, prop_ms = timed(lambda: tc.tc_proposal_weights(mlp, g, mot, delta, wts, feat, eps=eps))
    runs = []
    for i in range(4):
        r, ms = timed(lambda: tc.tc_sample_estimate_q(g, mot, delta, wts, prop, k, seed=0, offset=(50 + i) * k))
        runs.append((r, ms))
    q_ms = statistics.median(ms for _, ms in runs[1:])
    rq = runs[-1][0]
    var_plain = plain["std_err"] ** 2 * k
    var_learned = rq["std_err"] ** 2 * k
    c = rq["estimate"]

    def t_1pct(var, ms_per_sample):  # sampling time for a 1% relative standard error
        return var / (0.01 * c) ** 2 * ms_per_sample

    tp = t_1pct(var_plain, plain_sampler_ms / k)
    tl = t_1pct(var_learned, q_ms / k)
    budget = None
    if exact_C and plain_errors:
        # the paper's metric: mean relative error over seeds at one GPU-time
        # budget, that of k plain samples; the learned sampler gets as many
        # samples as fit in it
        k_l = max(2, int(k * plain_sampler_ms / q_ms))
        errs = run_errors(tc, g, mot, delta, wts, exact_C, k_l, prop)
        budget = {"budget_ms": plain_sampler_ms, "seeds": list(BUDGET_SEEDS), "k_plain": k, "k_learned": k_l,
                  "rel_error_plain": statistics.mean(plain_errors), "rel_error_learned": statistics.mean(errs),
                  "rel_error_ratio_learned_over_plain": statistics.mean(errs) / max(statistics.mean(plain_errors),
                                                                                    1e-300)}
    mlp.destroy()
    return {"objective": objective, "eps": eps, "train_samples": n_train, "stats_samples": n_stats,
            "train_ms": train_ms, "features_ms": feat_ms, "sample_features_ms": sfeat_ms, "proposal_ms": prop_ms,
            "loss_first_batch": losses[0], "loss_last_batch": losses[1],
            "sampler_ms": q_ms, "samples_per_s": k / (q_ms / 1e3), "estimate": c, "std_err": rq["std_err"],
            "plain_estimate": plain["estimate"], "plain_std_err": plain["std_err"],
            "variance_ratio_learned_over_plain": var_learned / var_plain,
            "time_to_1pct_ms_plain": tp, "time_to_1pct_ms_learned": tl, "time_ratio_learned_over_plain": tl / tp,
            "time_ratio_with_setup": (tl + feat_ms + sfeat_ms + train_ms + prop_ms) / (tp + weights_ms),
            "fixed_budget": budget}


def config_dict(cfg, k, world):
    if cfg["name"] in ("batch", "batch_small"):
        return {"workload": WORKLOADS[cfg["name"]], "k": int(k), "seed": 0,
                "parallelism": "dp%d (sample-id ranges)" % world,
                "reference_sample": "oracle on the 50M-edge graph, first query (4-cycle, delta=600)"}
    wl = WORKLOADS[cfg["name"]]
    if cfg.get("motif_override"):
        wl += "; motif replaced by %s" % cfg["motif_override"]
    return {"workload": wl,
            "n": int(cfg["n"]), "m": int(len(cfg["src"])),
            "motif": MOTIF_NAMES.get(str([tuple(e) for e in cfg["motif"]]), str(cfg["motif"])),
            "delta": int(cfg["delta"]),
            "k": int(k), "seed": 0, "parallelism": "dp%d (sample-id ranges)" % world,
            "l2": "inputs larger than L2 (graph + index ~2.4 GB resident)"}


def run_batch(args, rank, world, local):
    """The batched-query workload: every step is one tc_batch_run (weights
    per distinct key, key sorts, one persistent sampling launch)."""
    import torch
    from paper_2409_08975_gb300 import tc
    cfg = workload(args.workload)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dev = [(torch.from_numpy(g["src"]).cuda(), torch.from_numpy(g["dst"]).cuda(), torch.from_numpy(g["t"]).cuda())
           for g in cfg["graphs"]]
    torch.cuda.synchronize()
    ev0.record(stream)
    graphs = [tc.tc_build_temporal_csr(g["n"], *d) for g, d in zip(cfg["graphs"], dev)]
    ev1.record(stream)
    torch.cuda.synchronize()
    csr_ms = ev0.elapsed_time(ev1)
    del dev
    # rank r answers every query over its own sample-id range
    queries = [(graphs[gi], edges, delta, k, seed, rank * k) for gi, edges, delta, k, seed, _ in cfg["queries"]]
    k_total = sum(q[3] for q in queries)
    t0 = time.perf_counter()
    b = tc.Batch(queries)
    create_s = time.perf_counter() - t0
    info = b.info()
    for _ in range(args.warmup):
        b.run()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    launches0 = tc.tc_kernel_launches()
    samp = []
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    for _ in range(args.steps):
        res = b.run()
        samp.append(b.timing()[1])
    end.record(stream)
    torch.cuda.synchronize()
    launches = tc.tc_kernel_launches() - launches0
    clk = clocks.stop()
    total_ms = start.elapsed_time(end)
    merged = None
    if world > 1:
        tt = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(tt.item())
        from paper_2409_08975_gb300 import dist as tcdist  # the one exchange: exact per-query sums
        merged = tcdist.merge_batch(res, device="cuda")
    ms_per_step = total_ms / args.steps
    value = world * k_total / (ms_per_step / 1e3)
    sampler_ms = statistics.median(samp)
    checked = sum(r["checked"] for r in res)
    bytes_per_sample = SECTOR * (5 + 4 * checked / k_total)
    peak, peak_kind = load_peaks()
    achieved = bytes_per_sample * k_total / (sampler_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "kernel": "k_sample_batch (persistent sampler over all queries, Alg. 2-4)",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                "peak_kind": peak_kind, "bytes_per_sample": bytes_per_sample, "sampler_ms": sampler_ms}
    b.destroy()
    # end to end: host edge arrays -> device, graph builds, batch creation with
    # the tuned shape (no CUDA graph), one run, results to the host
    pinned = [(torch.from_numpy(g["src"]).pin_memory(), torch.from_numpy(g["dst"]).pin_memory(),
               torch.from_numpy(g["t"]).pin_memory()) for g in cfg["graphs"]]
    m_total = sum(len(g["src"]) for g in cfg["graphs"])
    e2e_times = []
    for i in range(1 + args.e2e_steps if args.e2e_steps > 0 else 0):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gs = []
        for g, (s_h, d_h, t_h) in zip(cfg["graphs"], pinned):
            d = (s_h.to("cuda", non_blocking=True), d_h.to("cuda", non_blocking=True),
                 t_h.to("cuda", non_blocking=True))
            gs.append(tc.tc_build_temporal_csr(g["n"], *d))
        qs = [(gs[gi], edges, delta, k, seed, rank * k) for gi, edges, delta, k, seed, _ in cfg["queries"]]
        bb = tc.Batch(qs, block_size=info["block_size"], tile=info["tile"], use_graph=False)
        bb.run()
        bb.destroy()
        for g in gs:
            g.destroy()
        dt = time.perf_counter() - t0
        if i > 0:
            e2e_times.append(dt)
    e2e = None
    if e2e_times:
        e2e_s = statistics.mean(e2e_times)
        # device->host per graph build 24 B; per query the sums (56 B); per
        # weights key W (8 B) and its error word (4 B)
        d2h = 24 * len(cfg["graphs"]) + 56 * len(queries) + 12 * info["weight_slots"]
        e2e = {"value": world * k_total / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 16 * m_total,
               "d2h_bytes_per_step": d2h, "ms_per_step": e2e_s * 1e3}
    if world > 1:
        torch.distributed.barrier()
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "queries": len(queries), "graphs": len(graphs),
                       "m_total": int(m_total), "k": int(k_total), "seed": 0,
                       "parallelism": "dp%d (sample-id ranges)" % world,
                       "l2": "inputs larger than L2 (the big graph and its weight indexes)"},
            "clocks": clk, "e2e": e2e, "gpu_launches": int(launches), "roofline": roofline, "cpu_baseline": None,
            "csr_build_ms": csr_ms, "batch": dict(info, create_s=create_s, sampling_ms_median=sampler_ms),
            "estimates": [{"W": r["W"], "k": r["k"], "estimate": r["estimate"], "std_err": r["std_err"]}
                          for r in (merged or res)[:8]],
            "merged_over_ranks": merged is not None,
        }))
    for g in graphs:
        g.destroy()


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2409_08975_gb300 import _build, tc
    if rank == 0:
        _build.build()
    if world > 1:
        torch.distributed.barrier()
    tc.lib()
    if args.workload in ("batch", "batch_small"):
        run_batch(args, rank, world, local)
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    cfg = workload(args.workload)
    if args.motif:
        cfg["motif"], cfg["motif_override"] = MOTIFS[args.motif], args.motif
    k = args.samples or cfg["k"]
    n, m, delta = cfg["n"], len(cfg["src"]), cfg["delta"]
    stream = torch.cuda.current_stream()
    mot = tc.make_motif(cfg["motif"])

    src_d = torch.from_numpy(cfg["src"]).cuda()
    dst_d = torch.from_numpy(cfg["dst"]).cuda()
    t_d = torch.from_numpy(cfg["t"]).cuda()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    g = tc.tc_build_temporal_csr(n, src_d, dst_d, t_d)
    ev1.record(stream)
    torch.cuda.synchronize()
    csr_ms = ev0.elapsed_time(ev1)
    del src_d, dst_d, t_d

    wts = tc.alloc_weights(g)

    kernel_ms = []

    def step(i, sample_events=None):
        # step i of rank r draws sample ids [(i * world + r) * k, + k)
        tc.tc_path_weights(g, mot, delta, out=wts, want_W=False)
        if sample_events is not None:
            sample_events[0].record(stream)
        r = tc.tc_sample_estimate(g, mot, delta, wts, k, seed=0, offset=(i * world + rank) * k)
        if sample_events is not None:
            sample_events[1].record(stream)
            kernel_ms.append(tc.tc_last_sampler_ms())
        return r

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    pairs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = tc.tc_kernel_launches()
    tc.tc_set_timing(True)  # events around the sampling launch inside each call
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    results = []
    for i in range(args.steps):
        results.append(step(args.warmup + i, pairs[i]))
    end.record(stream)
    torch.cuda.synchronize()
    tc.tc_set_timing(False)
    launches = tc.tc_kernel_launches() - launches0
    clk = clocks.stop()
    total_ms = start.elapsed_time(end)
    if world > 1:
        tt = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(tt.item())
    ms_per_step = total_ms / args.steps
    value = world * k / (ms_per_step / 1e3)
    sampler_ms = statistics.mean(a.elapsed_time(b) for a, b in pairs)

    # weights-only timing (the HBM-bound kernels), after the timed region
    wev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
    for a, b in wev:
        a.record(stream)
        tc.tc_path_weights(g, mot, delta, out=wts, want_W=False)
        b.record(stream)
    torch.cuda.synchronize()
    weights_ms = statistics.median(a.elapsed_time(b) for a, b in wev)

    r0 = results[-1]
    # exact count by the exhaustive path sum (all W paths), for the relative error
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    exact = None
    if r0["W"] <= args.exact_max_paths:
        ev[0].record(stream)
        ex = tc.tc_exact_count(g, mot, delta, wts)
        ev[1].record(stream)
        torch.cuda.synchronize()
        ex_ms = ev[0].elapsed_time(ev[1])
        exact = {"C": ex["sum_x"], "paths": ex["k"], "ms": ex_ms,
                 "paths_per_s": ex["k"] / (ex_ms / 1e3) if ex_ms > 0 else None,
                 "rel_error_plain": abs(r0["estimate"] - ex["sum_x"]) / max(ex["sum_x"], 1)}
    merged = None
    if world > 1:  # the one exchange: exact integer sums of the last step over ranks
        from paper_2409_08975_gb300 import dist as tcdist
        merged = tcdist.merge_runs(r0, r0["W"], device="cuda")
    checked_frac = r0["checked"] / max(r0["k"], 1)
    # sampler bytes per sample: guide entry, prefix entry, edge record and the
    # end-edge entries (two for a 3-path anchor, one for a wedge): 5 or 4
    # sectors; a checked path adds the pair list lookup (4 sectors)
    ends = sum(1 for a in tc.tc_motif_plan(mot)[1][:2] if a != 0)
    bytes_per_sample = SECTOR * (3 + ends + 4 * checked_frac)
    peak, peak_kind = load_peaks()
    k_sample_ms = statistics.mean(kernel_ms)  # the sampling launch alone, key-order sort excluded
    achieved = bytes_per_sample * k / (k_sample_ms / 1e3) / 1e9
    tps = SAMPLER_TRAFFIC_PER_SAMPLE.get((cfg["name"], MOTIF_NAMES.get(str([tuple(e) for e in cfg["motif"]]))))
    roofline = {"bound": "hbm", "kernel": "k_sample (sampler, Alg. 2-4)", "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "traffic": tps * k if tps else None, "peak_kind": peak_kind,
                "bytes_per_sample": bytes_per_sample, "kernel_ms": k_sample_ms, "sampler_call_ms": sampler_ms}
    # algorithmic bytes of the weights step, per the kernels: the v-window pass
    # 44 B/edge (absent for a wedge whose window is at u); the u-window pass
    # 16 B edge + 8 B parked v window + 16 B of the searched list (absent for
    # a wedge at v) + 32 B record + 8 B w; the exact scan 24 B/edge; the
    # guide 8 B/edge plus 4 B per bucket
    alpha1, alpha3 = tc.tc_motif_plan(mot)[1][:2]
    per_edge = (44 if alpha3 else 0) + 16 + (8 if alpha3 else 0) + (16 if alpha1 else 0) + 40 + 24 + 8
    weights_bytes = per_edge * m + 4 * (2 ** max(1, (m - 1).bit_length()))
    weights = {"ms": weights_ms, "bytes": weights_bytes, "bytes_per_edge": per_edge,
               "achieved_gbs": weights_bytes / (weights_ms / 1e3) / 1e9,
               "frac": weights_bytes / (weights_ms / 1e3) / 1e9 / peak}

    # end to end through the host entry point, pinned host buffers
    src_h = torch.from_numpy(cfg["src"]).pin_memory()
    dst_h = torch.from_numpy(cfg["dst"]).pin_memory()
    t_h = torch.from_numpy(cfg["t"]).pin_memory()
    e2e_times = []
    for i in range(1 + args.e2e_steps if args.e2e_steps > 0 else 0):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tc.tc_estimate_from_host(n, src_h, dst_h, t_h, mot, delta, k, seed=0)
        dt = time.perf_counter() - t0
        if i > 0:
            e2e_times.append(dt)
    e2e = None
    if e2e_times:
        e2e_s = statistics.mean(e2e_times)
        # host->device: the three edge arrays; device->host: the id/time check
        # (4 + 16 B), the pair count (4 B), W and the error word (12 B), the sums (56 B)
        e2e = {"value": world * k / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 16 * m, "d2h_bytes_per_step": 92,
               "ms_per_step": e2e_s * 1e3}

    comparisons = {}
    plain_errors = None
    if exact and exact["C"] and not args.no_learned and rank == 0:
        plain_errors = run_errors(tc, g, mot, delta, wts, exact["C"], k)
    if not args.no_learned and rank == 0:
        objectives = ["closure", "variance"] if args.objective == "both" else [args.objective]
        for obj in objectives:
            comparisons[obj] = learned_comparison(tc, g, mot, delta, wts, k, r0, sampler_ms, weights_ms,
                                                  args.train_samples, stream, obj,
                                                  exact["C"] if exact else None, plain_errors, args.stats_samples,
                                                  args.eps)
            if exact:
                comparisons[obj]["rel_error"] = abs(comparisons[obj]["estimate"] - exact["C"]) / max(exact["C"], 1)
    learned = comparisons.get("closure", comparisons.get("variance"))
    learned_variance = comparisons.get("variance") if len(comparisons) == 2 else None

    base = None
    if rank == 0 and not args.no_cpu_baseline and args.workload == "mid":
        base = cpu_baseline(cfg, k)[0]

    if world > 1:
        torch.distributed.barrier()
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic", "config": config_dict(cfg, k, world),
            "clocks": clk, "e2e": e2e, "gpu_launches": int(launches), "roofline": roofline,
            "cpu_baseline": base, "csr_build_ms": csr_ms, "weights": weights, "learned": learned,
            "learned_variance": learned_variance,
            "estimate": {"W": r0["W"], "estimate": r0["estimate"], "std_err": r0["std_err"], "hits": r0["hits"],
                         "checked": r0["checked"]},
            "merged_over_ranks": merged, "exact": exact,
        }))
    g.destroy()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
