"""Seeded synthetic temporal multigraphs shaped like the paper's workloads.

Input generation only: nothing in this module computes any part of the
estimator.  The paper's datasets (Table II: WT, SO, BI, RE) are not
available, so these generators stand in for them:

  * ``tiny``       n=2,000, m=20,000, uniform pairs, ~10% of pairs repeated
                   2-5 times, times uniform in [0, 1e6)
  * ``dense_tiny`` few vertices and the same edge count, so that delta windows
                   hold many edges and the exact count is large
  * ``chung_lu``   directed power-law (Chung-Lu weighted) multigraph whose
                   edges arrive in bursts: Poisson burst starts over the
                   span, Pareto(alpha = 1.5, x_m = 1 s) gaps inside a burst,
                   and a share of repeated pairs (multi-edges)
"""
import numpy as np

C4 = [(0, 1), (1, 2), (2, 3), (3, 0)]         # M4-0, directed temporal 4-cycle
PATH_CHORD = [(0, 1), (1, 2), (2, 3), (0, 3)]  # a->b, b->c, c->d, then a->d last


def _pairs_with_multiplicity(rng, n, m, repeat_prob, rep_lo=2, rep_hi=5):
    """Unique ordered pairs (src != dst) drawn uniformly; each pair gets
    multiplicity 1 or U{rep_lo..rep_hi} with probability repeat_prob; stop at
    m edges, trimming the last pair's multiplicity."""
    src_l, dst_l, total = [], [], 0
    seen = set()
    while total < m:
        need = max(1024, int((m - total) * 0.8))
        a = rng.integers(0, n, need)
        b = rng.integers(0, n, need)
        mult = np.where(rng.random(need) < repeat_prob, rng.integers(rep_lo, rep_hi + 1, need), 1)
        for x, y, k in zip(a.tolist(), b.tolist(), mult.tolist()):
            if x == y or (x, y) in seen:
                continue
            seen.add((x, y))
            k = min(k, m - total)
            src_l.extend([x] * k)
            dst_l.extend([y] * k)
            total += k
            if total >= m:
                break
    return np.array(src_l, np.int32), np.array(dst_l, np.int32)


def tiny(seed=1001):
    rng = np.random.default_rng(seed)
    src, dst = _pairs_with_multiplicity(rng, 2000, 20000, 0.10)
    t = rng.integers(0, 1_000_000, len(src)).astype(np.int64)
    return {"name": "tiny", "n": 2000, "src": src, "dst": dst, "t": t, "motif": C4, "delta": 10_000,
            "k": 100_000}


def dense_tiny(seed=1011, n=24, m=20000, span=1_000_000, bursty=False):
    """Companion graphs whose exact count is large (the tiny config's is ~0)."""
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n, 2 * m)
    dst = rng.integers(0, n, 2 * m)
    keep = src != dst
    src, dst = src[keep][:m], dst[keep][:m]
    rep = rng.random(m) < 0.10
    idx = np.flatnonzero(rep)
    if len(idx) > 1:  # repeat some earlier pairs
        j = rng.integers(0, len(src), len(idx))
        src[idx], dst[idx] = src[j], dst[j]
    if bursty:
        starts = rng.integers(0, span, m)
        gaps = np.floor(rng.pareto(1.5, m) + 1.0) * 60
        t = np.minimum(starts + gaps.astype(np.int64), span - 1)
    else:
        t = rng.integers(0, span, m)
    return {"name": "dense_tiny_n%d%s" % (n, "_bursty" if bursty else ""), "n": n,
            "src": src.astype(np.int32), "dst": dst.astype(np.int32), "t": t.astype(np.int64), "motif": C4,
            "delta": 10_000, "k": 100_000}


ZIPF_CAP = 1000


def _power_weights(n, gamma, i0):
    return (np.arange(n, dtype=np.float64) + i0) ** (-1.0 / (gamma - 1.0))


def _solve_i0(n, pairs, gamma, max_deg):
    lo, hi = 1e-3, float(n)
    for _ in range(80):
        mid = np.sqrt(lo * hi)
        w = _power_weights(n, gamma, mid)
        top = pairs * w[0] / w.sum()
        if top > max_deg:
            lo = mid
        else:
            hi = mid
    return hi


def chung_lu(n, m, gamma=2.1, max_deg=1e5, multi_frac=0.30, span=100_000_000, pareto_alpha=1.5, seed=1002,
             mean_burst_edges=200, burst_degree=(1.5, 24.0), daily=False, zipf_repeats=None):
    """Directed power-law multigraph whose edges arrive in bursts.

    Bursts start at uniform times over the span (a Poisson process
    conditioned on its count); a burst of B ~ Geometric(mean_burst_edges)
    edges draws max(4, B / d) vertex slots with Chung-Lu weights
    w_i ~ (i + i0)^(-1/(gamma-1)) (i0 set so the top vertex's expected
    out-degree is max_deg) and joins uniform slot pairs (no self-loops); its
    edges follow one another after Pareto(alpha, x_m = 1 s) gaps.  The edges
    per vertex slot d of a burst is burst_degree, or log-uniform in
    burst_degree = (lo, hi) per burst, so that dense and sparse bursts mix.
    A vertex's degree is then proportional to its weight, and edges close in
    time share vertices, as in transaction and communication networks.  A share
    multi_frac of all edges repeat an earlier edge's pair a Pareto gap later.
    ``daily`` modulates burst starts by 1 + 0.5 sin(2 pi t / 86400).
    ``zipf_repeats = s`` replaces the uniform repeats: every pair of the
    burst edges gets a total multiplicity drawn from Zipf(s) (truncated at
    ZIPF_CAP), the repeats following the pair's first edge after Pareto gaps,
    and the base edge count and top degree are scaled by the mean
    multiplicity so that the total is m and the top degree about max_deg."""
    rng = np.random.default_rng(seed)
    base_m = int(round(m * (1.0 - multi_frac)))
    base_max_deg = max_deg
    if zipf_repeats:
        j = np.arange(1, ZIPF_CAP + 1, dtype=np.float64)
        p = j ** (-float(zipf_repeats))
        mean_mult = float((j * p).sum() / p.sum())
        base_m = int(m / mean_mult)
        base_max_deg = max_deg / mean_mult  # the repeats multiply degrees
    sizes = rng.geometric(1.0 / mean_burst_edges, int(base_m / mean_burst_edges * 1.2) + 100)
    cs = np.cumsum(sizes)
    S = int(np.searchsorted(cs, base_m)) + 1
    sizes = sizes[:S].copy()
    sizes[-1] -= cs[S - 1] - base_m
    if np.isscalar(burst_degree):
        deg = np.full(S, float(burst_degree))
    else:
        lo, hi = burst_degree
        deg = np.exp(rng.uniform(np.log(lo), np.log(hi), S))
    nv = np.maximum(4, np.round(sizes / deg)).astype(np.int64)
    slots_total = int(nv.sum())
    i0 = _solve_i0(n, base_m, gamma, base_max_deg)
    w = _power_weights(n, gamma, i0)
    cdf = np.cumsum(w / w.sum())
    cdf[-1] = 1.0
    perm = rng.permutation(n)
    slots = perm[np.searchsorted(cdf, rng.random(slots_total), side="right").clip(0, n - 1)]
    soff = np.concatenate([[0], np.cumsum(nv)])
    burst = np.repeat(np.arange(S), sizes)
    src = slots[soff[burst] + rng.integers(0, nv[burst])]
    dst = slots[soff[burst] + rng.integers(0, nv[burst])]
    bad = src == dst
    while bad.any():
        idx = np.flatnonzero(bad)
        src[idx] = slots[soff[burst[idx]] + rng.integers(0, nv[burst[idx]])]
        dst[idx] = slots[soff[burst[idx]] + rng.integers(0, nv[burst[idx]])]
        bad = src == dst
    start = rng.integers(0, span, S)
    if daily:  # accept a start with probability (1 + 0.5 sin(2 pi t / 86400)) / 1.5
        bad = np.ones(S, bool)
        while bad.any():
            idx = np.flatnonzero(bad)
            c = rng.integers(0, span, len(idx))
            acc = rng.random(len(idx)) * 1.5 < 1.0 + 0.5 * np.sin(2 * np.pi * c / 86400.0)
            start[idx[acc]] = c[acc]
            bad[idx[acc]] = False
    gaps = np.floor(rng.pareto(pareto_alpha, base_m) + 1.0).astype(np.int64)
    first = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    gaps[first] = 0
    cum = np.cumsum(gaps)
    cum = cum - cum[first][burst]
    t = np.minimum(start[burst] + cum, span - 1)
    extra = m - base_m
    if zipf_repeats:  # copies of pair i: Zipf(s) - 1 more, then trimmed to m in total
        mult = np.minimum(rng.zipf(float(zipf_repeats), base_m), ZIPF_CAP) - 1
        cum = np.cumsum(mult)
        if cum[-1] < extra:  # top up uniformly (rare)
            mult[rng.integers(0, base_m, extra - int(cum[-1]))] += 1
            cum = np.cumsum(mult)
        cut = int(np.searchsorted(cum, extra))
        mult[cut] -= int(cum[cut] - extra)
        mult[cut + 1:] = 0
        pick = np.repeat(np.arange(base_m), mult)  # grouped by pair
        gsum = np.cumsum(np.floor(rng.pareto(pareto_alpha, len(pick)) + 1.0).astype(np.int64))
        first = np.repeat(np.cumsum(mult) - mult, mult)  # index of the pair's first repeat
        offset = gsum - np.concatenate([[0], gsum])[first]  # Pareto gaps summed since the first edge
        rt = np.minimum(t[pick] + offset, span - 1)
    else:
        pick = rng.integers(0, base_m, extra)
        rt = np.minimum(t[pick] + np.floor(rng.pareto(pareto_alpha, extra) + 1.0).astype(np.int64), span - 1)
    src = np.concatenate([src, src[pick]]).astype(np.int32)
    dst = np.concatenate([dst, dst[pick]]).astype(np.int32)
    t = np.concatenate([t, rt]).astype(np.int64)
    shuffle = rng.permutation(m)
    return {"n": n, "src": src[shuffle], "dst": dst[shuffle], "t": t[shuffle]}


def mid(seed=1002):
    g = chung_lu(1_000_000, 20_000_000, gamma=2.1, max_deg=1e5, multi_frac=0.30, seed=seed)
    g.update({"name": "mid", "motif": PATH_CHORD, "delta": 3600, "k": 100_000_000})
    return g


def scaled_mid(n, m, seed=1002, k=1_000_000):
    """The mid generator at another size (parity tests, profiling)."""
    g = chung_lu(n, m, gamma=2.1, max_deg=max(10.0, 1e5 * m / 20_000_000), multi_frac=0.30, seed=seed)
    g.update({"name": "mid_n%d_m%d" % (n, m), "motif": PATH_CHORD, "delta": 3600, "k": k})
    return g


def learned(seed=1004):
    """Learned-proposal configuration: the mid generator at n = 2e7, m = 1e8."""
    g = chung_lu(20_000_000, 100_000_000, gamma=2.1, max_deg=5e5, multi_frac=0.30, seed=seed)
    g.update({"name": "learned", "motif": PATH_CHORD, "delta": 3600, "k": 100_000_000})
    return g


def large(seed=1005):
    """Large transaction-like graph: n = 1e8, m = 3e8, top degree ~1e6,
    pair multiplicities Zipf(1.8), burst starts with daily periodicity."""
    g = chung_lu(100_000_000, 300_000_000, gamma=2.1, max_deg=1e6, seed=seed, daily=True, zipf_repeats=1.8)
    g.update({"name": "large", "motif": C4, "motifs": {"c4": C4, "path_chord": PATH_CHORD}, "delta": 3600,
              "k": 1_000_000_000})
    return g


def large_small(seed=1105):
    """Profiling case of the large graph's kernels: the same generator
    (Zipf(1.8) pair multiplicities, daily periodicity) at n = 1e7, m = 3e7,
    top degree about 1e5 (graph and indexes about 3 GB, many times L2),
    directed 4-cycle, delta = 3600, k = 3e7."""
    g = chung_lu(10_000_000, 30_000_000, gamma=2.1, max_deg=1e5, seed=seed, daily=True, zipf_repeats=1.8)
    g.update({"name": "large_small", "motif": C4, "motifs": {"c4": C4, "path_chord": PATH_CHORD}, "delta": 3600,
              "k": 30_000_000})
    return g


BATCH_DELTAS = (600, 3600, 86400)


def time_slice(g, j, parts=100):
    """Contiguous time slice j of `parts` of graph g, each holding about
    1 / parts of the edges: with t_(i) the i-th smallest time and m edges,
    the edges with t_(j m / parts) <= t < t_((j + 1) m / parts) (no upper
    bound for the last slice), in input order, with the vertices that occur
    renumbered 0..n'-1 in increasing order of their ids (which keeps every
    list order).  Returns a graph dict with the slice's time bounds."""
    t = g["t"]
    m = len(t)
    k0, k1 = j * m // parts, (j + 1) * m // parts
    ks = [k0] + ([k1] if j + 1 < parts else [])
    part = np.partition(t, ks)
    lo = int(part[k0])
    hi = int(part[k1]) if j + 1 < parts else None
    sel = np.flatnonzero((t >= lo) & (t < hi)) if hi is not None else np.flatnonzero(t >= lo)
    src, dst = g["src"][sel], g["dst"][sel]
    verts, inv = np.unique(np.concatenate([src, dst]), return_inverse=True)
    out = {k: v for k, v in g.items() if k not in ("src", "dst", "t", "n")}
    out.update({"name": "%s_slice%d_of%d" % (g.get("name", "graph"), j, parts), "n": int(max(len(verts), 1)),
                "src": inv[:len(sel)].astype(np.int32), "dst": inv[len(sel):].astype(np.int32),
                "t": t[sel].copy(), "t_lo": lo, "t_hi": hi, "m_parent": m})
    return out


def small(seed=1007):
    """Profiling case: the mid generator at n = 5e5, m = 1e7 (graph and index
    about 1 GB, several times L2), path+chord, delta = 3600, k = 1e7."""
    g = chung_lu(500_000, 10_000_000, gamma=2.1, max_deg=5e4, multi_frac=0.30, seed=seed)
    g.update({"name": "small", "motif": PATH_CHORD, "delta": 3600, "k": 10_000_000})
    return g


def batch(seed=1003, n_small=64, big_m=50_000_000, k_range=(1e6, 1e8)):
    """Batched queries: a 50M-edge graph of the mid generator (n = 2.5M)
    queried with all 24 time-rank orders of the directed 4-cycle at each
    delta in BATCH_DELTAS, plus n_small graphs of 1e4 - 2e6 edges
    (log-uniform) with one query each (rank order i mod 24, delta i mod 3).
    Samples per query are log-uniform in [1e6, 1e8].  Queries are
    (graph index, edges, delta, k, seed, sample_offset); graph 0 is the big
    graph."""
    import itertools
    rng = np.random.default_rng(seed)
    graphs = [chung_lu(big_m // 20, big_m, gamma=2.1, max_deg=2.5e5 * big_m / 50_000_000, multi_frac=0.30,
                       seed=seed)]
    sizes = np.exp(rng.uniform(np.log(1e4), np.log(2e6), n_small)).astype(np.int64)
    for i, m_i in enumerate(sizes):
        n_i = int(max(1000, m_i // 20))
        graphs.append(chung_lu(n_i, int(m_i), gamma=2.1, max_deg=max(10.0, 1e5 * m_i / 20_000_000),
                               multi_frac=0.30, seed=seed + 1 + i))
    orders = [[C4[j] for j in p] for p in itertools.permutations(range(4))]
    def k_draw():
        return int(np.exp(rng.uniform(np.log(k_range[0]), np.log(k_range[1]))))
    queries = []
    for o, edges in enumerate(orders):
        for d in BATCH_DELTAS:
            queries.append((0, edges, d, k_draw(), 0, 0))
    for i in range(n_small):
        queries.append((1 + i, orders[i % 24], BATCH_DELTAS[i % 3], k_draw(), 0, 0))
    return {"name": "batch", "graphs": graphs, "queries": queries, "motif": C4, "delta": 3600,
            "k": sum(q[3] for q in queries)}


def batch_small(seed=1008):
    """Profiling case of the batch: a 1e7-edge big graph, 8 small graphs,
    1e5 - 1e7 samples per query."""
    cfg = batch(seed=seed, n_small=8, big_m=10_000_000, k_range=(1e5, 1e7))
    cfg["name"] = "batch_small"
    return cfg


CONFIGS = {"tiny": tiny, "mid": mid, "learned": learned, "large": large, "batch": batch, "small": small,
           "large_small": large_small,
           "batch_small": batch_small}
