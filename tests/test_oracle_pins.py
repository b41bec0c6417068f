"""Pins of the CPU oracle against facts fixed outside itself: published
known answers, closed forms, library routines, literal brute force of the
paper's definitions, and the statistical properties the paper proves.

Every test here runs without a GPU.
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from _graphs import GOLDEN, hand_graphs, path_motifs_all_classes, small_random_graph

C4 = [(0, 1), (1, 2), (2, 3), (3, 0)]           # M4-0, directed 4-cycle
CHORD = [(0, 1), (1, 2), (2, 3), (0, 3)]        # 3-path + closing edge a->d last


# --------------------------------------------------------------------------
# Philox4x32-10: published known-answer vectors (Salmon et al., SC'11)

def test_philox_known_answers():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(x, 16) for x in line.split()])
    assert len(rows) == 3
    for r in rows:
        assert oracle.philox4x32_10(r[0:4], r[4:6]) == r[6:10]


# --------------------------------------------------------------------------
# Lemire's bounded draw (Lemire 2019)

def _x(seed, s, d, a, upper=False):
    o = oracle.philox4x32_10([s & 0xFFFFFFFF, s >> 32, d, a], [seed & 0xFFFFFFFF, seed >> 32])
    return (o[2] | (o[3] << 32)) if upper else (o[0] | (o[1] << 32))


@pytest.mark.parametrize("j", [1, 5, 17, 32, 63])
def test_bounded_power_of_two_is_top_bits(j):
    # 2^64 mod 2^j = 0: nothing is rejected and x * 2^j >> 64 = x >> (64 - j),
    # x from the lower or the upper half of the block
    for s in range(200):
        assert oracle.bounded(7, s, 2, 1 << j) == _x(7, s, 2, 0) >> (64 - j)
        assert oracle.bounded(7, s, 1, 1 << j, upper=True) == _x(7, s, 1, 0, upper=True) >> (64 - j)


def test_bounded_range_one_and_bounds():
    rng = np.random.default_rng(0)
    for s in range(300):
        assert oracle.bounded(1, s, 0, 1) == 0
        R = int(rng.integers(1, 1 << 62)) * 3 + 1
        assert 0 <= oracle.bounded(1, s, 1, R) < R


@pytest.mark.parametrize("R,mod", [(3 << 62, 3), (5 << 61, 5)])
def test_bounded_rejection_removes_bias(R, mod):
    # For R = 3*2^62 the map x -> floor(x R / 2^64) without rejection hits
    # residues r % 3 == 0 twice as often (probability 1/2 instead of 1/3);
    # with the rejection of Lemire's method the residues are uniform.
    N = 30000
    counts = np.zeros(mod)
    for s in range(N):
        counts[oracle.bounded(11, s, 0, R, upper=bool(s & 1)) % mod] += 1
    chi2 = ((counts - N / mod) ** 2 / (N / mod)).sum()
    assert chi2 < 20.0, counts


# --------------------------------------------------------------------------
# ListCount (Alg. 4) against enumeration of tuples

def _tuples(lists):
    return sum(1 for tup in itertools.product(*lists) if all(tup[i] < tup[i + 1] for i in range(len(tup) - 1)))


def test_list_count_bruteforce():
    rng = np.random.default_rng(3)
    for trial in range(300):
        l = int(rng.integers(1, 5))
        lists = [np.sort(rng.integers(0, 12, int(rng.integers(0, 7)))) for _ in range(l)]
        assert oracle.list_count(lists) == _tuples(lists)


def test_list_count_closed_forms():
    assert oracle.list_count([]) == 1
    assert oracle.list_count([[1, 2, 3]]) == 3
    assert oracle.list_count([[1, 2], [5, 6, 7]]) == 6          # all of L1 before L2
    assert oracle.list_count([[5, 6], [1, 2]]) == 0
    vals = list(range(10))
    for l in range(1, 6):                                       # C(10, l)
        assert oracle.list_count([vals] * l) == math.comb(10, l)
    assert oracle.list_count([[4, 4], [4, 4]]) == 0             # ties never count


# --------------------------------------------------------------------------
# Lists: the comparison sorts agree with numpy.lexsort on the full keys

def test_csr_orders_match_lexsort():
    src, dst, t = small_random_graph(5, 30, 400, 50)
    n, m = 30, len(src)
    g = oracle.build_csr(n, src, dst, t)
    idx = np.arange(m)
    assert (g.out_perm == np.lexsort((idx, t, src))).all()
    assert (g.in_perm == np.lexsort((idx, t, dst))).all()
    assert (g.pair_perm == np.lexsort((idx, t, dst, src))).all()
    g2 = oracle.build_csr(n, src, dst, t, sort="lexsort")
    for name in ("out_perm", "out_off", "in_perm", "in_off", "in_eid", "pair_perm", "pair_off", "pair_dst",
                 "pair_eoff"):
        assert (getattr(g, name) == getattr(g2, name)).all(), name
    assert (g.out_off == np.concatenate([[0], np.cumsum(np.bincount(src, minlength=n))])).all()
    assert (g.in_off == np.concatenate([[0], np.cumsum(np.bincount(dst, minlength=n))])).all()
    canon = np.empty(m, np.int64)
    canon[g.out_perm] = idx
    assert (g.in_eid == canon[g.in_perm]).all()
    pairs = sorted(set(zip(src.tolist(), dst.tolist())))
    assert g.P == len(pairs)
    assert g.pair_dst.tolist() == [b for _, b in pairs]
    for p, (a, b) in enumerate(pairs):
        seg = g.pair_perm[g.pair_eoff[p]:g.pair_eoff[p + 1]]
        assert ((src[seg] == a) & (dst[seg] == b)).all()
        assert len(seg) == int(((src == a) & (dst == b)).sum())
        assert g.pair_off[a] <= p < g.pair_off[a + 1]


# --------------------------------------------------------------------------
# Claim 1 / Alg. 1: w_e equals a literal count of delta-centered paths

@pytest.mark.parametrize("closed", [False, True])
def test_weights_equal_path_enumeration_all_classes(closed):
    src, dst, t = small_random_graph(11, 7, 60, 40)
    g = oracle.build_csr(7, src, dst, t)
    for edges in path_motifs_all_classes():
        plan = oracle.compile_motif(edges, closed=closed)
        for delta in (0, 3, 12, 100):
            pw = oracle.path_weights(g, plan, delta)
            brute = np.array(oracle.brute_force_paths(src, dst, t, plan, delta), dtype=np.uint64)
            assert (pw["w"] == brute[g.out_perm]).all(), (plan.cls, delta)
            assert (pw["w"] == pw["d1"].astype(np.uint64) * pw["d3"].astype(np.uint64)).all()


def test_strict_windows_empty_at_delta_zero():
    src, dst, t = small_random_graph(2, 8, 80, 10)
    g = oracle.build_csr(8, src, dst, t)
    pw = oracle.path_weights(g, oracle.compile_motif(C4), 0)
    assert int(pw["w"].sum()) == 0


def test_prefix_sum_and_overflow():
    w = np.array([3, 0, 5, 1 << 40, 7], dtype=np.uint64)
    pre = oracle.prefix_sum(w)
    assert pre.tolist() == [0, 3, 3, 8, 8 + (1 << 40), 15 + (1 << 40)]
    with pytest.raises(oracle.OracleError) as e:
        oracle.prefix_sum(np.array([1 << 63, 1 << 63], dtype=np.uint64))
    assert e.value.status == oracle.STATUS_OVERFLOW
    assert oracle.prefix_sum(np.zeros(0, np.uint64)).tolist() == [0]


# --------------------------------------------------------------------------
# Exact counts: hand derivations, literal brute force, backtracking, and the
# path-sum identity of Claim 2's proof

@pytest.mark.parametrize("case", hand_graphs(), ids=lambda c: c[0])
def test_hand_graphs(case):
    name, edges, delta, count, src, dst, t = case
    g = oracle.build_csr(4, src, dst, t)
    assert oracle.brute_force_count(src, dst, t, edges, delta) == count
    assert oracle.exact_count(g, edges, delta) == count
    assert oracle.path_sum(g, oracle.compile_motif(edges), delta)["C"] == count


def _motif_zoo():
    zoo = [C4, CHORD, [(0, 1), (2, 3), (1, 2)], [(1, 2), (0, 1), (2, 3), (3, 0)],
           [(0, 1), (1, 2), (2, 3), (2, 3)], [(0, 1), (1, 2), (1, 2), (2, 3), (3, 0), (0, 2)],
           [(2, 3), (1, 2), (0, 1), (0, 3)]]
    zoo += path_motifs_all_classes()[::3]
    return zoo


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_path_sum_equals_brute_force(seed):
    src, dst, t = small_random_graph(100 + seed, 5, 32, 30, dup_frac=0.3)
    g = oracle.build_csr(5, src, dst, t)
    for edges in _motif_zoo():
        for delta in (4, 15, 40):
            C = oracle.brute_force_count(src, dst, t, edges, delta)
            assert oracle.exact_count(g, edges, delta) == C
            for closed in (False, True):
                plan = oracle.compile_motif(edges, closed=closed)
                ps = oracle.path_sum(g, plan, delta)
                assert ps["C"] == C, (edges, delta, closed)
                W = int(oracle.prefix_sum(oracle.path_weights(g, plan, delta)["w"])[-1])
                assert ps["paths"] == W


def test_every_anchor_choice_gives_the_count():
    # Claim 2 holds for any anchor containing edge 0; forcing each candidate
    # anchor of the 4-cycle must give the same exact path-sum.
    src, dst, t = small_random_graph(42, 5, 40, 30, dup_frac=0.3)
    g = oracle.build_csr(5, src, dst, t)
    C = oracle.brute_force_count(src, dst, t, C4, 20)
    cands = oracle.core.anchor_candidates(C4)
    assert len(cands) == 3
    for c in cands:
        plan = oracle.compile_motif(C4, anchor=(c[1], c[2], c[3]))
        assert oracle.path_sum(g, plan, 20)["C"] == C


def test_rotation_invariance_of_4cycle_orderings():
    # Relabelling a->b->c->d->a maps an ordering of the directed 4-cycle to
    # another ordering with the same number of matches: 24 orderings fall into
    # 6 orbits of 4 with equal exact counts.
    src, dst, t = small_random_graph(9, 5, 120, 60, dup_frac=0.3)
    g = oracle.build_csr(5, src, dst, t)
    cyc = [(0, 1), (1, 2), (2, 3), (3, 0)]
    counts = {}
    for perm in itertools.permutations(range(4)):
        edges = [cyc[p] for p in perm]             # edge of rank i is cyc[perm[i]]
        counts[perm] = oracle.path_sum(g, oracle.compile_motif(edges), 25)["C"]
    orbits = set()
    for perm in counts:
        orbit = frozenset(tuple((p + s) % 4 for p in perm) for s in range(4))
        orbits.add(orbit)
        vals = {counts[q] for q in orbit}
        assert len(vals) == 1, (orbit, vals)
    assert len(orbits) == 6
    assert sum(counts.values()) > 0


def test_single_pair_multigraph_has_no_match():
    src = np.zeros(20, np.int32)
    dst = np.ones(20, np.int32)
    t = np.arange(20, dtype=np.int64)
    src[::2], dst[::2] = 1, 0
    g = oracle.build_csr(2, src, dst, t)
    plan = oracle.compile_motif(C4)
    pre = oracle.prefix_sum(oracle.path_weights(g, plan, 10)["w"])
    sums, tr = oracle.sample_run(g, plan, 10, pre, 500, 3, trace=True)
    assert int(pre[-1]) > 0 and sums["sum_x"] == 0 and sums["hits"] == 0


def test_empty_graph():
    g = oracle.build_csr(4, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int64))
    plan = oracle.compile_motif(C4)
    pre = oracle.prefix_sum(oracle.path_weights(g, plan, 10)["w"])
    assert pre.tolist() == [0]
    sums, _ = oracle.sample_run(g, plan, 10, pre, 100, 0)
    assert sums["sum_x"] == 0
    assert oracle.estimate(0, 0, 100, 0) == (0.0, 0.0)


# --------------------------------------------------------------------------
# Sampler: Lemma 1 (uniform over the W paths) and per-path counts

def _per_path_counts(src, dst, t, edges, plan, delta):
    """Brute force: for every M-match (Def. 2) the image of the anchor edges,
    keyed by input edge indices (e1, e2, e3)."""
    m, r = len(src), len(edges)
    order = sorted(range(m), key=lambda i: (int(t[i]), i))
    out = {}
    for combo in itertools.combinations(order, r):
        times = [int(t[e]) for e in combo]
        if any(times[i] >= times[i + 1] for i in range(r - 1)) or times[-1] - times[0] > delta:
            continue
        phi, ok = {}, True
        for (x, y), e in zip(edges, combo):
            for lab, vert in ((x, int(src[e])), (y, int(dst[e]))):
                if phi.setdefault(lab, vert) != vert:
                    ok = False
        if ok and len(set(phi.values())) == len(phi):
            key = (combo[plan.e1], combo[plan.mid], combo[plan.e3])
            out[key] = out.get(key, 0) + 1
    return out


def test_sampler_uniform_and_per_path_counts():
    src, dst, t = small_random_graph(21, 5, 28, 25, dup_frac=0.3)
    g = oracle.build_csr(5, src, dst, t)
    plan = oracle.compile_motif(CHORD)
    delta = 12
    pw = oracle.path_weights(g, plan, delta)
    pre = oracle.prefix_sum(pw["w"])
    W = int(pre[-1])
    assert 20 <= W <= 5000
    N = 60 * W
    sums, tr = oracle.sample_run(g, plan, delta, pre, N, 5, trace=True)
    per = _per_path_counts(src, dst, t, CHORD, plan, delta)
    e1_of = g.in_perm if plan.alpha1 < 0 else g.out_perm
    e3_of = g.in_perm if plan.alpha3 < 0 else g.out_perm
    freq = {}
    for i2, p1, p3, X in tr.astype(np.int64).tolist():
        key = (int(e1_of[p1]), int(g.out_perm[i2]), int(e3_of[p3]))
        freq[key] = freq.get(key, 0) + 1
        assert X == per.get(key, 0)                       # X = C_P (Claim 2)
    # each sampled triple is a path of the class (Def. 4/5)
    assert len(freq) <= W
    counts = np.array(list(freq.values()) + [0] * (W - len(freq)), dtype=np.float64)
    chi2 = ((counts - N / W) ** 2 / (N / W)).sum()
    dof = W - 1
    assert chi2 < dof + 4.0 * math.sqrt(2 * dof), (chi2, dof)  # Lemma 1
    assert sums["sum_x"] == int(tr[:, 3].sum())


def test_unbiased_over_1000_seeds():
    # Claim 2: E[C_hat] = C.  Exact per-sample variance from the path sums:
    # Var X = sum_P C_P^2 / W - (C / W)^2; the mean of 1000 estimates of k
    # samples lies within 2.576 standard deviations (99%) of C.
    src, dst, t = small_random_graph(77, 6, 60, 60, dup_frac=0.3)
    g = oracle.build_csr(6, src, dst, t)
    plan = oracle.compile_motif(C4)
    delta = 20
    pre = oracle.prefix_sum(oracle.path_weights(g, plan, delta)["w"])
    W = int(pre[-1])
    ps = oracle.path_sum(g, plan, delta)
    C = ps["C"]
    assert C == oracle.brute_force_count(src, dst, t, C4, delta) and C > 0
    var_x = Fraction(ps["sum_x2"], W) - Fraction(C, W) ** 2
    k, seeds = 200, 1000
    ests = []
    for seed in range(seeds):
        sums, _ = oracle.sample_run(g, plan, delta, pre, k, seed)
        ests.append(oracle.estimate(sums["sum_x"], sums["sum_x2"], k, W)[0])
    sd_mean = W * math.sqrt(float(var_x) / k / seeds)
    assert abs(np.mean(ests) - C) <= 2.576 * sd_mean, (np.mean(ests), C, sd_mean)
    # the per-run standard error estimates the true one
    sd_run = W * math.sqrt(float(var_x) / k)
    assert 0.8 * sd_run < np.std(ests) < 1.2 * sd_run


def test_sample_offsets_compose():
    # samples are keyed by id: two ranges merge into one run exactly
    src, dst, t = small_random_graph(8, 6, 60, 60, dup_frac=0.3)
    g = oracle.build_csr(6, src, dst, t)
    plan = oracle.compile_motif(C4)
    pre = oracle.prefix_sum(oracle.path_weights(g, plan, 20)["w"])
    a, ta = oracle.sample_run(g, plan, 20, pre, 300, 9, 0, trace=True)
    b, tb = oracle.sample_run(g, plan, 20, pre, 200, 9, 300, trace=True)
    c, tc_ = oracle.sample_run(g, plan, 20, pre, 500, 9, 0, trace=True)
    assert (np.concatenate([ta, tb]) == tc_).all()
    for key in ("sum_x", "sum_x2", "hits", "k"):
        assert a[key] + b[key] == c[key]


def test_estimate_exact_integer_division():
    # C_hat = sum_x * W / k formed as q + r/k
    for sx, W, k in [(7, 10, 3), (1 << 40, (1 << 60) + 3, 12345), (0, 5, 9), (5, 1, 1)]:
        c, _ = oracle.estimate(sx, sx * sx, k, W)
        assert c == pytest.approx(float(Fraction(sx * W, k)), rel=1e-15)
    # standard error of a constant sample is zero
    assert oracle.estimate(30, 90, 10, 4)[1] == 0.0


def test_threaded_oracle_equals_serial():
    """The OpenMP loops (weights, sampler with trace, path sum, backtracking
    count) give the serial results exactly."""
    from _graphs import small_random_graph
    src, dst, t = small_random_graph(91, 9, 400, 300, dup_frac=0.3)
    g = oracle.build_csr(9, src, dst, t)
    plan = oracle.compile_motif(C4)
    res = []
    try:
        for threads in (1, 4):
            assert oracle.set_threads(threads) in (1, threads)
            pw = oracle.path_weights(g, plan, 40)
            pre = oracle.prefix_sum(pw["w"])
            sums, tr = oracle.sample_run(g, plan, 40, pre, 5000, 3, 11, trace=True)
            res.append((pw["w"].copy(), pw["lo1"].copy(), pw["d3"].copy(), sums, tr.copy(),
                        oracle.path_sum(g, plan, 40), oracle.exact_count(g, C4, 40)))
    finally:
        oracle.set_threads(1)
    a, b = res
    for x, y in zip(a, b):
        if isinstance(x, np.ndarray):
            assert np.array_equal(x, y)
        else:
            assert x == y
    assert a[5]["C"] == a[6] > 0
