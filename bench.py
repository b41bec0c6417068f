"""Benchmark of the temporal 3-path sampling estimator on one GB300.

A step is one pass of the whole hot path over the resident graph: path
weights and their exact prefix sum with the sampling index (Claim 1, Alg. 1),
then k sampled 3-paths with CheckMotif / ListCount and the reduction of the
estimate (Alg. 2-5).  The default workload is the large transaction-like
graph: n = 1e8 vertices, m = 3e8 edges, top in/out degree about 1e6, pair
multiplicities Zipf(1.8), times over 1e8 s with daily periodicity, the
directed 4-cycle (M4-0) with delta = 3600 s and k = 1e9 samples per step.

Printed: one JSON line with samples/s (device, graph resident); the same
metric end to end through tc_estimate_from_host with pinned host buffers;
the roofline of the dominant kernel (the sampler) and of the weights and
prefix (the paper's algorithmic bytes per edge), each from CUDA events the
library records around its launches; the oracle's rate on all host cores (a
bounded sample: a 1% time slice of the graph); the exact count of that slice
by the oracle's enumerator beside the GPU's; the relative error of the
estimate against the GPU's exact count of the whole graph; the learned
proposals against the plain one at a fixed GPU-time budget; and the SM
clocks seen during the timed region.

``--impl reference`` times the CPU oracle instead (the reference arm).
Under torchrun each rank runs the full path on its own GPU over its own
sample-id range (weak scaling); the integer sums merge exactly afterwards.
"""
import argparse
import json
import os
import platform
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
# DRAM bytes (read + write) per unit of a kernel, from one ncu capture of the
# benchmark's own launches (dram__bytes_read.sum + dram__bytes_write.sum, one
# pass over the default workload's list build and five steps: the launch list
# summarised in profiles/launch_list_large_bench.md); valid while the kernel
# is unchanged, null for workloads not captured
SAMPLER_TRAFFIC_PER_SAMPLE = {("large", "c4"): 76.3}   # k_sample
WEIGHTS_TRAFFIC_PER_EDGE = {("large", "c4"): 89.9}     # k_weights_rw 74.1 + the scan of w 15.8
UNIT = "samples/s"
SECTOR = 32
LEARNED_VARIANTS = ("closure", "variance", "as_written")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--samples", type=int, default=None, help="samples per step (default: the config's k)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--exact-max-paths", type=float, default=1e12,
                    help="run the exhaustive exact count when W is at most this")
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the oracle's timing on the host cores and the slice check that uses it")
    ap.add_argument("--cpu-samples", type=int, default=2_000_000,
                    help="samples of the oracle's timed sampler run (all host cores)")
    ap.add_argument("--learned", default=",".join(LEARNED_VARIANTS),
                    help="learned proposals to compare with the plain one (comma list of %s; '' for none): "
                         "closure = 16 inputs (12 edge counts and 4 sample statistics) trained on the closure "
                         "count; variance = the same inputs trained on the estimator's variance; as_written = "
                         "the 12 edge counts alone trained by binary cross-entropy on the closure outcome "
                         "1[X > 0]" % ", ".join(LEARNED_VARIANTS))
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-proposal comparison")
    ap.add_argument("--train-samples", type=int, default=10_000_000)
    ap.add_argument("--stats-samples", type=int, default=None,
                    help="plain samples behind the sample-statistics features (default: --train-samples)")
    ap.add_argument("--eps", type=float, default=0.05, help="the learned proposal's mixture weight: q ~ w (eps + g)")
    ap.add_argument("--motif", default=None, choices=sorted(MOTIFS),
                    help="another motif on the workload's graph (default: the workload's own)")
    ap.add_argument("--workload", default="large",
                    choices=["large", "mid", "learned", "batch", "small", "large_small", "batch_small"],
                    help="large: n=1e8, m=3e8 (default); mid: the 20M-edge graph; learned: n=2e7, m=1e8")
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


def load_bf16_peak():
    """Dense bf16 tensor throughput (TFLOP/s) of MEASURED_PEAKS.json (burst), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        return 1900.0


def workload(name="large"):
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
    "large_small": "large_small (profiling case): the large generator at n=1e7 m=3e7, top degree ~1e5, pair "
                   "multiplicities Zipf(1.8), daily periodicity; directed 4-cycle (M4-0), delta=3600, k=3e7",
    "batch_small": "batch_small (profiling case): as batch with a 1e7-edge big graph, 8 small graphs and 1e5-1e7 "
                   "samples per query",
    "batch": "batch: 136 queries in one persistent launch replayed from a CUDA graph; a 50M-edge graph of the mid "
             "generator (n=2.5M) with all 24 time-rank orders of the directed 4-cycle x delta in {600, 3600, 86400}, "
             "plus 64 graphs of 1e4-2e6 edges (log-uniform) with one query each; 1e6-1e8 samples per query "
             "(log-uniform), ~2.5e9 samples per step",
}
SLICE_PARTS = 100  # the oracle's bounded sample of a graph above SLICE_MIN_EDGES: one 1% time slice
SLICE_MIN_EDGES = 50_000_000


def host_info():
    """Host cores and CPU model (lscpu), for the CPU baseline."""
    model = platform.processor() or platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"cores": os.cpu_count() or 1, "model": model, "arch": platform.machine()}


def oracle_sample(cfg):
    """The graph the oracle runs on: the whole graph, or for graphs above
    SLICE_MIN_EDGES its first 1% time slice (a contiguous bounded sample of
    the same workload: same generator, same delta windows)."""
    from paper_2409_08975_gb300 import synth
    m = len(cfg["src"])
    if m <= SLICE_MIN_EDGES:
        return dict(cfg, t_lo=None, t_hi=None, m_parent=m), 1.0
    s = synth.time_slice(cfg, 0, SLICE_PARTS)
    return s, m / len(s["src"])


def cpu_baseline(cfg, k_total, sample_k, exact=True):
    """The oracle as it stands, on all host cores (OpenMP; the sums are
    integers, so the results equal the serial ones), on a bounded sample of
    the workload: weights and prefix over the sample graph timed in full and
    scaled to the whole graph's edge count; the sampler timed on sample_k
    samples and scaled to k_total samples per step; and, timed apart, the
    exact count of the sample graph by the oracle's enumerator (chronological
    backtracking over the motif's edges, Def. 2)."""
    import oracle
    info = host_info()
    sg, scale = oracle_sample(cfg)
    threads = oracle.set_threads(info["cores"])
    try:
        og = oracle.build_csr(sg["n"], sg["src"], sg["dst"], sg["t"], sort="lexsort")
        plan = oracle.compile_motif(cfg["motif"])
        t0 = time.perf_counter()
        w = oracle.path_weights(og, plan, cfg["delta"])["w"]
        pre = oracle.prefix_sum(w)
        t_prep = time.perf_counter() - t0
        t0 = time.perf_counter()
        oracle.sample_run(og, plan, cfg["delta"], pre, sample_k, 0, 0)
        t_samp = time.perf_counter() - t0
        ex = None
        if exact:
            t0 = time.perf_counter()
            C = oracle.exact_count(og, cfg["motif"], cfg["delta"])
            ex = {"C": int(C), "W": int(pre[-1]), "edges": int(og.m), "n": int(og.n), "t_lo": sg["t_lo"],
                  "t_hi": sg["t_hi"], "s": time.perf_counter() - t0, "threads": threads}
    finally:
        oracle.set_threads(1)
    per = t_samp / sample_k
    step_s = t_prep * scale + per * k_total
    where = ("the whole graph (%d edges)" % og.m if scale == 1.0 else
             "its first 1%% time slice (%d of %d edges, t in [%d, %d))" % (og.m, len(cfg["src"]), sg["t_lo"],
                                                                           sg["t_hi"]))
    base = {"value": k_total / step_s, "unit": UNIT, "cores": threads, "kind": "oracle",
            "host": info,
            "sample": "C oracle, %d OpenMP threads, on %s: weights+prefix %.3f s, scaled x%.1f to all edges; sampler "
                      "%d samples in %.3f s, scaled to k=%d per step; extrapolated step %.1f s" % (
                          threads, where, t_prep, scale, sample_k, t_samp, k_total, step_s),
            "weights_s_sample": t_prep, "edge_scale": scale, "sampler_s": t_samp, "sampler_samples": sample_k,
            "step_s_extrapolated": step_s}
    return base, ex, sg


def run_reference(args, rank, world):
    """The reference arm: the oracle on all host cores (rank 0 only), each
    step a bounded sample of sampler work on the oracle's sample graph (the
    whole graph, or its first 1% time slice for the large graph)."""
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
    info = host_info()
    sg, scale = oracle_sample(cfg)
    threads = oracle.set_threads(info["cores"])
    og = oracle.build_csr(sg["n"], sg["src"], sg["dst"], sg["t"], sort="lexsort")
    plan = oracle.compile_motif(cfg["motif"])
    t0 = time.perf_counter()
    pre = oracle.prefix_sum(oracle.path_weights(og, plan, cfg["delta"])["w"])
    t_prep = time.perf_counter() - t0
    step_k = 200_000
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.sample_run(og, plan, cfg["delta"], pre, step_k, 0, s * step_k)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    oracle.set_threads(1)
    per = sum(times) / (len(times) * step_k)
    step_s = t_prep * scale + per * k
    value = k / step_s
    where = "the whole graph" if scale == 1.0 else "its first 1%% time slice (%d edges)" % og.m
    sample = ("C oracle, %d OpenMP threads, on %s: weights+prefix %.3f s scaled x%.1f to all edges; each measured "
              "step %d samples (%.3f s mean), scaled to k=%d samples per step" % (threads, where, t_prep, scale,
                                                                                 step_k, per * step_k, k))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_s * 1e3, "ms_per_step_extrapolated": True,
        "measured_step_ms": statistics.mean(times) * 1e3, "measured_step_samples": step_k,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": config_dict(cfg, k, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
                         "host": info},
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


def learned_comparison(tc, g, mot, delta, wts, k, plain, plain_ms, weights_ms, n_train, stream, variant="closure",
                       exact_C=None, plain_errors=None, n_stats=None, eps=0.05):
    """A learned proposal q ~ w (eps + g) against the plain q ~ w on the same
    graph.  Setup, once per (graph, motif, delta): the edge features, the
    sample statistics (not for as_written) and training on n_train plain
    samples.  Per query: the inference, h, q and q-prefix with its guide
    (tc_proposal_weights), then the proposal's sampling.  The learned GPU time
    is inference + q-scan + sampling (a second figure adds the features and
    sample statistics, a third all of the setup), the plain one its sampling
    (key-order sort and sampling launches: plain_ms per k samples).  Relative error at a
    fixed GPU time follows from the per-sample variance (k SE^2) and the time
    per sample of each sampler; with the exact count C, it is also measured
    as the mean relative error of five seeds' runs at the GPU time of k plain
    samples, the learned sampler taking what the budget leaves after its
    inference."""
    import torch

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        out = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return out, a.elapsed_time(b)

    objective = {"closure": "closure", "variance": "variance", "as_written": "bce"}[variant]
    fbuf = tc.alloc_features(g)  # the 32 B per edge buffer is allocated outside the timed call
    torch.cuda.synchronize()
    feat, feat_ms = timed(lambda: tc.tc_edge_features(g, mot, delta, wts, out=fbuf))
    n_stats = 0 if variant == "as_written" else (n_stats or n_train)
    sfeat_ms = 0.0
    if n_stats:  # sample statistics from plain samples of another seed than the training paths
        _, sfeat_ms = timed(lambda: tc.tc_sample_features(g, mot, delta, wts, feat, n_stats, seed=777))
    mlp = tc.MLP(seed=1)
    losses, train_ms = timed(lambda: tc.tc_mlp_train(mlp, g, mot, delta, wts, feat, n_train, seed=12345,
                                                     batch=16384, lr=3e-3, objective=objective, eps=eps))
    props, net_ms, guide_ms = [], [], []
    tc.tc_set_timing(True)
    for _ in range(3):
        props.append(timed(lambda: tc.tc_proposal_weights(mlp, g, mot, delta, wts, feat, eps=eps)))
        net_ms.append(tc.tc_last_phase_ms("proposal"))
        guide_ms.append(tc.tc_last_phase_ms("index"))
    tc.tc_set_timing(False)
    prop = props[-1][0]
    prop_call_ms = statistics.median(ms for _, ms in props)
    # GPU time of the inference: its kernels (network, h, q and q-prefix; the
    # guide of the q index), as the plain side counts its sampling kernels
    prop_ms = statistics.median(a + b for a, b in zip(net_ms, guide_ms))
    # the network on the tensor cores: 2 (16 x 64 + 64 x 64 + 64) FLOP per edge
    # with w > 0 (the proposal runs only those; counted here from the prefix)
    live = int(torch.count_nonzero(wts.prefix[1:g.m + 1] != wts.prefix[:g.m]).item())
    flops = 2 * (16 * 64 + 64 * 64 + 64) * live
    tflops_peak = load_bf16_peak()
    net = statistics.median(net_ms)
    # the inference's HBM bytes: per edge the prefix entry read (8), h and q
    # written (2 + 8), the q-prefix scan (16); per live edge its feature row (32)
    hbm_bytes = (8 + 2 + 8 + 16) * g.m + 32 * live
    inference_phases = {"network_h_q_prefix_ms": net, "guide_ms": statistics.median(guide_ms),
                        "live_edges": live, "hbm_gbs": hbm_bytes / (net / 1e3) / 1e9 if net > 0 else None,
                        "frac_of_hbm": hbm_bytes / (net / 1e3) / 1e9 / load_peaks()[0] if net > 0 else None,
                        "tensor_tflops": flops / (net / 1e3) / 1e12 if net > 0 else None,
                        "bf16_peak_tflops": tflops_peak,
                        "frac_of_bf16_peak": flops / (net / 1e3) / 1e12 / tflops_peak if net > 0 else None,
                        "path": ("tcgen05.mma kind::f16 M128 N64 (TMEM accumulators, one issuing thread)"
                                 if tc.tc_mlp_kernel() == "tcgen05" else
                                 "mma.sync m16n8k16 bf16 (warp-level tensor-core MMA)")}
    runs, q_phase = [], []
    tc.tc_set_timing(True)
    for i in range(4):
        r, ms = timed(lambda: tc.tc_sample_estimate_q(g, mot, delta, wts, prop, k, seed=0, offset=(50 + i) * k))
        runs.append((r, ms))
        q_phase.append(tc.tc_last_phase_ms("order") + tc.tc_last_phase_ms("sample"))
    tc.tc_set_timing(False)
    q_call_ms = statistics.median(ms for _, ms in runs[1:])
    q_ms = statistics.median(q_phase[1:])  # the key-order sort and sampling kernels, as plain_ms
    rq = runs[-1][0]
    var_plain = plain["std_err"] ** 2 * k
    var_learned = rq["std_err"] ** 2 * k
    c = rq["estimate"]
    # GPU time to a 1% relative standard error
    tp = var_plain / (0.01 * c) ** 2 * plain_ms / k
    tl_sampling = var_learned / (0.01 * c) ** 2 * q_ms / k
    setup_ms = feat_ms + sfeat_ms + train_ms
    # time to the plain sampler's error at k samples: the learned sampler needs
    # k var_learned / var_plain samples after its inference and q-scan
    k_equal = k * var_learned / var_plain
    t_equal = prop_ms + k_equal * q_ms / k
    budget = None
    if exact_C and plain_errors:
        k_l = int(k * (plain_ms - prop_ms) / q_ms)
        if k_l >= 2:
            errs = run_errors(tc, g, mot, delta, wts, exact_C, k_l, prop)
            budget = {"budget_ms": plain_ms, "inference_ms": prop_ms, "seeds": list(BUDGET_SEEDS), "k_plain": k,
                      "k_learned": k_l, "rel_error_plain": statistics.mean(plain_errors),
                      "rel_error_learned": statistics.mean(errs),
                      "rel_error_ratio_learned_over_plain": statistics.mean(errs) / max(statistics.mean(plain_errors),
                                                                                        1e-300)}
        else:
            budget = {"budget_ms": plain_ms, "inference_ms": prop_ms, "k_learned": 0,
                      "note": "the inference and q-scan alone exceed the budget"}
    mlp.destroy()
    del feat, fbuf
    return {"variant": variant, "objective": objective, "inputs": 12 if variant == "as_written" else 16, "eps": eps,
            "train_samples": n_train, "stats_samples": n_stats,
            "setup_ms": {"features": feat_ms, "sample_statistics": sfeat_ms, "training": train_ms},
            "inference_ms": prop_ms, "inference_call_ms": prop_call_ms, "inference_phases": inference_phases,
            "sampler_ms": q_ms, "sampler_call_ms": q_call_ms,
            "samples_per_s": k / (q_ms / 1e3),
            "loss_first_batch": losses[0], "loss_last_batch": losses[1],
            "estimate": c, "std_err": rq["std_err"], "plain_estimate": plain["estimate"],
            "plain_std_err": plain["std_err"],
            "variance_ratio_learned_over_plain": var_learned / var_plain,
            "sampling_time_ratio": tl_sampling / tp,
            "time_to_plain_error_ms": {"plain": plain_ms, "learned": t_equal,
                                       "ratio": t_equal / plain_ms,
                                       "ratio_with_features": (t_equal + feat_ms + sfeat_ms) / plain_ms,
                                       "ratio_with_setup": (t_equal + setup_ms) / plain_ms,
                                       "ratio_with_weights_both": (t_equal + weights_ms) / (plain_ms + weights_ms)},
            "fixed_budget": budget}


def config_dict(cfg, k, world):
    if cfg["name"] in ("batch", "batch_small"):
        return {"workload": WORKLOADS[cfg["name"]], "k": int(k), "seed": 0,
                "parallelism": "dp%d (sample-id ranges)" % world,
                "reference_sample": "oracle on the 50M-edge graph, first query (4-cycle, delta=600)"}
    wl = WORKLOADS.get(cfg["name"], cfg["name"])
    if cfg.get("motif_override"):
        wl += "; motif replaced by %s" % cfg["motif_override"]
    m = int(len(cfg["src"]))
    return {"workload": wl,
            "n": int(cfg["n"]), "m": m,
            "motif": MOTIF_NAMES.get(str([tuple(e) for e in cfg["motif"]]), str(cfg["motif"])),
            "delta": int(cfg["delta"]),
            "k": int(k), "seed": 0, "parallelism": "dp%d (sample-id ranges)" % world,
            "l2": "inputs larger than L2: resident graph lists ~%.1f GB, sampling index %.1f GB, prefix %.1f GB "
                  "(L2 129 MB); no flush between steps" % (110e-9 * m, 23e-9 * m, 8e-9 * m)}


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
    (alpha1, alpha3, _, _) = tc.tc_motif_plan(mot)[1]

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
    compact_times = (g.t_max - g.t_min) < (1 << 32)

    wts = tc.alloc_weights(g)
    phases = {"weights": [], "index": [], "order": [], "sample": []}

    def step(i, record=False):
        # step i of rank r draws sample ids [(i * world + r) * k, + k)
        tc.tc_path_weights(g, mot, delta, out=wts, want_W=False)
        if record:
            phases["weights"].append(tc.tc_last_phase_ms("weights"))
            phases["index"].append(tc.tc_last_phase_ms("index"))
        r = tc.tc_sample_estimate(g, mot, delta, wts, k, seed=0, offset=(i * world + rank) * k)
        if record:
            phases["order"].append(tc.tc_last_phase_ms("order"))
            phases["sample"].append(tc.tc_last_phase_ms("sample"))
        return r

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    launches0 = tc.tc_kernel_launches()
    tc.tc_set_timing(True)  # events around each phase's launches inside each call
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    results = []
    for i in range(args.steps):
        results.append(step(args.warmup + i, record=True))
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
    ph = {p: statistics.mean(v) for p, v in phases.items()}
    sampler_call_ms = ph["order"] + ph["sample"]  # the plain sampler's GPU time per k samples

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
                 "rel_error_plain": abs(r0["estimate"] - ex["sum_x"]) / max(ex["sum_x"], 1),
                 "method": "tc_exact_count: CheckMotif summed over all W paths (Claim 2's proof); pinned against "
                           "the oracle's backtracking count on 1% time slices (slice_check, tests)"}
    merged = None
    if world > 1:  # the one exchange: exact integer sums of the last step over ranks
        from paper_2409_08975_gb300 import dist as tcdist
        merged = tcdist.merge_runs(r0, r0["W"], device="cuda")

    peak, peak_kind = load_peaks()
    checked_frac = r0["checked"] / max(r0["k"], 1)
    # sampler algorithmic bytes per sample (sector model): guide entry, prefix
    # entry, edge record and the end-edge entries (two for a 3-path anchor,
    # one for a wedge): 5 or 4 sectors; a checked path adds the pair-list
    # lookup (hash slot and pair-list times: 4 sectors)
    ends = sum(1 for a in (alpha1, alpha3) if a != 0)
    bytes_per_sample = SECTOR * (3 + ends + 4 * checked_frac)
    achieved = bytes_per_sample * k / (ph["sample"] / 1e3) / 1e9
    key = (cfg["name"], MOTIF_NAMES.get(str([tuple(e) for e in cfg["motif"]])))
    tps = SAMPLER_TRAFFIC_PER_SAMPLE.get(key)
    roofline = {"bound": "hbm", "kernel": "k_sample (sampler with CheckMotif / ListCount, Alg. 2-4)",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": tps * k if tps else None, "peak_kind": peak_kind,
                "limiter": "latency of dependent random loads (long-scoreboard stalls in ncu)",
                "bytes_per_sample": bytes_per_sample, "kernel_ms": ph["sample"],
                "dram_bytes_per_sample": tps,
                "dram_frac": (tps * k / (ph["sample"] / 1e3) / 1e9 / peak) if tps else None}
    # the paper's algorithmic bytes of a1 (Claim 1, Alg. 1): the edge's time,
    # the searched list's times, its dst / in->out entry and the w write --
    # 20 B per edge with 32-bit time offsets (28 with int64 times); a2: 16 B
    # per edge (read w, write prefix); the implementation's DRAM bytes beside
    a1 = 20 if compact_times else 28
    a12 = (a1 + 16) * m
    wtr = WEIGHTS_TRAFFIC_PER_EDGE.get(key)
    weights = {"ms": ph["weights"], "alg_bytes_per_edge": {"a1": a1, "a2": 16}, "alg_bytes": a12,
               "achieved_gbs": a12 / (ph["weights"] / 1e3) / 1e9,
               "frac": a12 / (ph["weights"] / 1e3) / 1e9 / peak, "peak": peak, "peak_kind": peak_kind,
               "dram_bytes_per_edge": wtr, "kernel": "k_weights_rw, then the scan of w (k_tile_scan)",
               "index_ms": ph["index"], "order_ms": ph["order"], "sample_ms": ph["sample"]}

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
    del src_h, dst_h, t_h
    e2e = None
    if e2e_times:
        e2e_s = statistics.mean(e2e_times)
        # host->device: the three edge arrays; device->host: the id/time check
        # (4 + 16 B), the pair count (4 B), W and the error word (12 B), the sums (56 B)
        e2e = {"value": world * k / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 16 * m, "d2h_bytes_per_step": 92,
               "ms_per_step": e2e_s * 1e3}

    comparisons = {}
    plain_errors = None
    variants = [] if args.no_learned else [v for v in args.learned.split(",") if v]
    if exact and exact["C"] and variants and rank == 0:
        plain_errors = run_errors(tc, g, mot, delta, wts, exact["C"], k)
    if rank == 0:
        for var in variants:
            try:
                comparisons[var] = learned_comparison(tc, g, mot, delta, wts, k, r0, sampler_call_ms, ph["weights"],
                                                      args.train_samples, stream, var,
                                                      exact["C"] if exact else None, plain_errors,
                                                      args.stats_samples, args.eps)
                if exact:
                    comparisons[var]["rel_error"] = abs(comparisons[var]["estimate"] - exact["C"]) / max(exact["C"],
                                                                                                         1)
            except Exception as exc:  # keep the line: report the failure instead
                comparisons[var] = {"variant": var, "error": "%s: %s" % (type(exc).__name__, exc)}

    base, slice_check = None, None
    if rank == 0 and not args.no_cpu_baseline:
        try:
            base, slice_check = cpu_leg(args, cfg, k, tc, mot, delta, stream, ev)
        except Exception as exc:  # keep the line: report the failure instead
            slice_check = {"error": "%s: %s" % (type(exc).__name__, exc)}

    if world > 1:
        torch.distributed.barrier()
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic", "config": config_dict(cfg, k, world),
            "clocks": clk, "e2e": e2e, "gpu_launches": int(launches), "roofline": roofline,
            "cpu_baseline": base, "csr_build_ms": csr_ms, "weights": weights,
            "learned": comparisons.get("closure"), "learned_variance": comparisons.get("variance"),
            "learned_as_written": comparisons.get("as_written"),
            "estimate": {"W": r0["W"], "estimate": r0["estimate"], "std_err": r0["std_err"], "hits": r0["hits"],
                         "checked": r0["checked"]},
            "merged_over_ranks": merged, "exact": exact, "slice_check": slice_check,
        }))
    g.destroy()
    if world > 1:
        torch.distributed.destroy_process_group()


def cpu_leg(args, cfg, k, tc, mot, delta, stream, ev):
    """The oracle's CPU baseline, and the GPU's exact count of the oracle's
    sample graph beside the oracle's."""
    import torch
    base, ex_or, sg = cpu_baseline(cfg, k, args.cpu_samples)
    # the GPU's exact count of the oracle's sample graph, against the oracle's
    dev = lambda a, dt: torch.from_numpy(a).to(device="cuda", dtype=dt)
    gs = tc.tc_build_temporal_csr(sg["n"], dev(sg["src"], torch.int32), dev(sg["dst"], torch.int32),
                                  dev(sg["t"], torch.int64))
    ws = tc.tc_path_weights(gs, mot, delta)
    ev[0].record(stream)
    exs = tc.tc_exact_count(gs, mot, delta, ws)
    ev[1].record(stream)
    torch.cuda.synchronize()
    slice_check = dict(ex_or, C_gpu=exs["sum_x"], W_gpu=ws.W, gpu_ms=ev[0].elapsed_time(ev[1]),
                       equal=(exs["sum_x"] == ex_or["C"] and ws.W == ex_or["W"]),
                       what="exact count of the oracle's sample graph (1%% time slice of a graph above %d edges, "
                            "else the whole graph): oracle backtracking (Def. 2, all host cores) vs "
                            "tc_exact_count" % SLICE_MIN_EDGES)
    gs.destroy()
    return base, slice_check


if __name__ == "__main__":
    main()
