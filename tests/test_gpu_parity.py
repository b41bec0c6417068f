"""Parity of the CUDA path with the CPU oracle, element by element, through
the C ABI.  Integer outputs (lists, weights, prefix, sampled indices, X,
sums) must be bit-exact; the FP64 estimate must agree to 1e-12 relative."""
import numpy as np
import pytest

import oracle
from _graphs import path_motifs_all_classes, small_random_graph

pytestmark = pytest.mark.gpu

C4 = [(0, 1), (1, 2), (2, 3), (3, 0)]
CHORD = [(0, 1), (1, 2), (2, 3), (0, 3)]
M41 = [(0, 1), (1, 2), (2, 3), (3, 2), (2, 1), (1, 0), (0, 1), (1, 2), (2, 3)]
MULTI = [(0, 1), (1, 2), (1, 2), (2, 3), (3, 0), (0, 2)]   # two lists in one gap, one in another
LATE_MID = [(2, 3), (1, 2), (0, 1), (0, 3)]                 # middle edge not of rank 1
REL_TOL = 1e-12


@pytest.fixture(scope="module")
def tc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_08975_gb300 import _build
    _build.build()
    from paper_2409_08975_gb300 import tc as tcmod
    tcmod.lib()
    return tcmod


def _dev(a, dt):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)


def _build_both(tc, n, src, dst, t):
    import torch
    g = tc.tc_build_temporal_csr(n, _dev(src, torch.int32), _dev(dst, torch.int32), _dev(t, torch.int64))
    og = oracle.build_csr(n, src, dst, t)
    return g, og


def _u64(x):
    return x.cpu().numpy().view(np.uint64)


def _graphs():
    out = []
    s, d, t = small_random_graph(3, 9, 300, 200, dup_frac=0.3)
    out.append(("small", 9, s, d, t))
    from paper_2409_08975_gb300 import synth
    g = synth.tiny()
    out.append(("tiny", g["n"], g["src"], g["dst"], g["t"]))
    g = synth.dense_tiny()
    out.append(("dense24", g["n"], g["src"], g["dst"], g["t"]))
    g = synth.dense_tiny(seed=1012, n=200, bursty=True)
    out.append(("dense200b", g["n"], g["src"], g["dst"], g["t"]))
    # several sort/scan tiles and a ragged tail
    g = synth.scaled_mid(5000, 61_237, seed=7)
    out.append(("cl61k", g["n"], g["src"], g["dst"], g["t"]))
    return out


GRAPHS = _graphs()


def _check_csr(tc, g, og):
    m = og.m
    oe = g.array("out_edges").view(-1, 4).cpu().numpy()
    src, dst, t = og.src, og.dst, og.t
    assert (oe[:, 0] == src[og.out_perm]).all()
    assert (oe[:, 1] == dst[og.out_perm]).all()
    assert (oe[:, 2:].copy().view(np.int64)[:, 0] == t[og.out_perm]).all()
    assert (g.array("edge_perm").cpu().numpy() == og.out_perm).all()
    assert (g.array("out_off").cpu().numpy() == og.out_off).all()
    ie = g.array("in_edges").view(-1, 4).cpu().numpy()
    assert (ie[:, 0] == src[og.in_perm]).all()
    assert (ie[:, 1] == og.dst[og.in_perm]).all()
    assert (g.array("in_eid").cpu().numpy().astype(np.int64) == og.in_eid).all()
    assert (ie[:, 2:].copy().view(np.int64)[:, 0] == t[og.in_perm]).all()
    assert (g.array("in_off").cpu().numpy() == og.in_off).all()
    assert g.num_pairs == og.P
    assert (g.array("pair_off").cpu().numpy() == og.pair_off).all()
    assert (g.array("pair_dst").cpu().numpy() == og.pair_dst).all()
    assert (g.array("pair_eoff").cpu().numpy() == og.pair_eoff).all()
    assert (g.array("pair_t").cpu().numpy() == t[og.pair_perm]).all()
    canon = np.empty(m, np.int64)
    canon[og.out_perm] = np.arange(m)
    assert (g.array("pair_eid").cpu().numpy() == canon[og.pair_perm]).all()


@pytest.mark.parametrize("case", GRAPHS, ids=lambda c: c[0])
def test_csr_bit_exact(tc, case):
    name, n, src, dst, t = case
    g, og = _build_both(tc, n, src, dst, t)
    _check_csr(tc, g, og)
    # the canonical edge order as int64 (tc_graph_edge_order)
    assert (tc.tc_graph_edge_order(g).cpu().numpy() == og.out_perm).all()


def _records(w):
    idx = w.index.cpu().numpy()
    m = (len(w.prefix) - 1)
    rec = idx[256:256 + 16 * m].view(np.uint32).reshape(m, 4)
    return rec


@pytest.mark.parametrize("case", GRAPHS, ids=lambda c: c[0])
def test_weights_prefix_bit_exact(tc, case):
    name, n, src, dst, t = case
    g, og = _build_both(tc, n, src, dst, t)
    motifs = [C4, CHORD, LATE_MID] + path_motifs_all_classes()
    deltas = (0, 7, 50_000) if name in ("small",) else (10_000,)
    for edges in motifs:
        for window in (0, 1):
            plan = oracle.compile_motif(edges, closed=bool(window))
            mot = tc.make_motif(edges, window=window)
            for delta in deltas:
                ow = oracle.path_weights(og, plan, delta)
                opre = oracle.prefix_sum(ow["w"])
                w = tc.tc_path_weights(g, mot, delta, want_w=True)
                assert w.W == int(opre[-1])
                assert (_u64(w.w)[:og.m] == ow["w"]).all(), (edges, window, delta)
                assert (_u64(w.prefix) == opre).all()
                rec = _records(w)
                assert (rec[:, 0] == ow["lo1"]).all() and (rec[:, 1] == ow["d1"]).all()
                assert (rec[:, 2] == ow["lo3"]).all() and (rec[:, 3] == ow["d3"]).all()


@pytest.mark.parametrize("case", GRAPHS, ids=lambda c: c[0])
def test_sampler_trace_and_sums_bit_exact(tc, case):
    name, n, src, dst, t = case
    g, og = _build_both(tc, n, src, dst, t)
    for edges in (C4, CHORD, M41, MULTI, LATE_MID):
        for window in (0, 1):
            delta = 10_000 if name != "small" else 60
            plan = oracle.compile_motif(edges, closed=bool(window))
            mot = tc.make_motif(edges, window=window)
            w = tc.tc_path_weights(g, mot, delta)
            opre = oracle.prefix_sum(oracle.path_weights(og, plan, delta)["w"])
            if w.W == 0:
                continue
            k, seed, off = 20_000, 12345, 777
            tr = _u64(tc.tc_sample_trace(g, mot, delta, w, k, seed, off))
            osums, otr = oracle.sample_run(og, plan, delta, opre, k, seed, off, trace=True)
            assert (tr == otr).all(), (edges, window)
            est = tc.tc_sample_estimate(g, mot, delta, w, k, seed, off)
            for key in ("sum_x", "sum_x2", "hits", "k"):
                assert est[key] == osums[key], key
            c_hat, se = oracle.estimate(osums["sum_x"], osums["sum_x2"], k, int(opre[-1]))
            assert est["estimate"] == pytest.approx(c_hat, rel=REL_TOL, abs=0)
            assert est["std_err"] == pytest.approx(se, rel=REL_TOL, abs=0)


@pytest.mark.parametrize("case", GRAPHS[2:], ids=lambda c: c[0])
def test_key_sorted_sampling_bit_exact(tc, case):
    # from 2^16 samples on, the library processes each chunk's samples sorted
    # by middle-edge key; ids, indices and X must still match the oracle
    name, n, src, dst, t = case
    g, og = _build_both(tc, n, src, dst, t)
    for edges in (CHORD, MULTI):
        plan = oracle.compile_motif(edges)
        mot = tc.make_motif(edges)
        w = tc.tc_path_weights(g, mot, 10_000)
        opre = oracle.prefix_sum(oracle.path_weights(og, plan, 10_000)["w"])
        k, seed, off = 70_001, 99, 1 << 40
        tr = _u64(tc.tc_sample_trace(g, mot, 10_000, w, k, seed, off))
        osums, otr = oracle.sample_run(og, plan, 10_000, opre, k, seed, off, trace=True)
        assert (tr == otr).all()
        est = tc.tc_sample_estimate(g, mot, 10_000, w, k, seed, off)
        for key in ("sum_x", "sum_x2", "hits"):
            assert est[key] == osums[key]


@pytest.mark.parametrize("case", GRAPHS, ids=lambda c: c[0])
def test_exact_count_matches_path_sum(tc, case):
    # the exhaustive GPU path sum equals the oracle's path sum (itself pinned
    # to the literal count of Def. 2 on tiny graphs by the CPU tests)
    name, n, src, dst, t = case
    g, og = _build_both(tc, n, src, dst, t)
    delta = 10_000 if name != "small" else 60
    for edges in (C4, CHORD, MULTI, LATE_MID):
        for window in (0, 1):
            plan = oracle.compile_motif(edges, closed=bool(window))
            mot = tc.make_motif(edges, window=window)
            w = tc.tc_path_weights(g, mot, delta)
            r = tc.tc_exact_count(g, mot, delta, w)
            ps = oracle.path_sum(og, plan, delta)
            assert r["sum_x"] == ps["C"] and r["sum_x2"] == ps["sum_x2"] and r["k"] == ps["paths"] == w.W


def test_exact_count_hand_graphs(tc):
    import torch
    from _graphs import hand_graphs
    for name, edges, delta, count, src, dst, t in hand_graphs():
        g = tc.tc_build_temporal_csr(4, _dev(src, torch.int32), _dev(dst, torch.int32), _dev(t, torch.int64))
        mot = tc.make_motif(edges)
        w = tc.tc_path_weights(g, mot, delta)
        assert tc.tc_exact_count(g, mot, delta, w)["sum_x"] == count, name


def test_tiny_config_estimate(tc):
    from paper_2409_08975_gb300 import synth
    cfg = synth.tiny()
    g, og = _build_both(tc, cfg["n"], cfg["src"], cfg["dst"], cfg["t"])
    plan = oracle.compile_motif(cfg["motif"])
    mot = tc.make_motif(cfg["motif"])
    w = tc.tc_path_weights(g, mot, cfg["delta"])
    opre = oracle.prefix_sum(oracle.path_weights(og, plan, cfg["delta"])["w"])
    est = tc.tc_sample_estimate(g, mot, cfg["delta"], w, cfg["k"], 0, 0)
    osums, _ = oracle.sample_run(og, plan, cfg["delta"], opre, cfg["k"], 0, 0)
    assert est["sum_x"] == osums["sum_x"] and est["sum_x2"] == osums["sum_x2"] and est["hits"] == osums["hits"]
    assert est["W"] == int(opre[-1])


def test_unbiased_over_1000_seeds_gpu(tc):
    # Claim 2 on the device path: the mean of 1000 estimates lies within the
    # 99% interval of the exact count (exact variance from the path sums).
    from fractions import Fraction
    import math
    src, dst, t = small_random_graph(77, 6, 60, 60, dup_frac=0.3)
    g, og = _build_both(tc, 6, src, dst, t)
    plan = oracle.compile_motif(C4)
    ps = oracle.path_sum(og, plan, 20)
    C = oracle.brute_force_count(src, dst, t, C4, 20)
    assert ps["C"] == C > 0
    mot = tc.make_motif(C4)
    w = tc.tc_path_weights(g, mot, 20)
    W = w.W
    var_x = Fraction(ps["sum_x2"], W) - Fraction(C, W) ** 2
    k = 200
    ests = [tc.tc_sample_estimate(g, mot, 20, w, k, seed)["estimate"] for seed in range(1000)]
    sd_mean = W * math.sqrt(float(var_x) / k / 1000)
    assert abs(np.mean(ests) - C) <= 2.576 * sd_mean


def test_disjoint_ranges_merge(tc):
    from paper_2409_08975_gb300 import synth
    cfg = synth.dense_tiny()
    g, _ = _build_both(tc, cfg["n"], cfg["src"], cfg["dst"], cfg["t"])
    mot = tc.make_motif(CHORD)
    w = tc.tc_path_weights(g, mot, 10_000)
    a = tc.tc_sample_estimate(g, mot, 10_000, w, 300_000, 5, 0)
    b = tc.tc_sample_estimate(g, mot, 10_000, w, 700_000, 5, 300_000)
    c = tc.tc_sample_estimate(g, mot, 10_000, w, 1_000_000, 5, 0)
    for key in ("sum_x", "sum_x2", "hits", "k"):
        assert a[key] + b[key] == c[key]
    # the merged sums through the library's estimate equal the single run bit for bit
    est, se = tc.tc_estimate_from_sums(a["sum_x"] + b["sum_x"], a["sum_x2"] + b["sum_x2"], 1_000_000, w.W)
    assert est == c["estimate"] and se == c["std_err"]


# ---------------------------------------------------------------------------
# edge cases and errors


def test_empty_graph_and_zero_delta(tc):
    import torch
    e32 = torch.zeros(0, dtype=torch.int32, device="cuda")
    e64 = torch.zeros(0, dtype=torch.int64, device="cuda")
    g = tc.tc_build_temporal_csr(5, e32, e32, e64)
    assert g.m == 0 and g.num_pairs == 0
    mot = tc.make_motif(C4)
    w = tc.tc_path_weights(g, mot, 100)
    assert w.W == 0
    est = tc.tc_sample_estimate(g, mot, 100, w, 1000, 0)
    assert est["estimate"] == 0.0 and est["sum_x"] == 0
    # delta = 0 with strict windows: no path at all
    src, dst, t = small_random_graph(4, 8, 200, 30)
    g, og = _build_both(tc, 8, src, dst, t)
    assert tc.tc_path_weights(g, mot, 0).W == 0


def test_single_vertex_pair_multigraph(tc):
    src = np.array([0, 1] * 50, np.int32)
    dst = np.array([1, 0] * 50, np.int32)
    t = np.arange(100, dtype=np.int64)
    g, og = _build_both(tc, 2, src, dst, t)
    mot = tc.make_motif(C4)
    w = tc.tc_path_weights(g, mot, 10)
    assert w.W > 0
    est = tc.tc_sample_estimate(g, mot, 10, w, 10_000, 1)
    assert est["sum_x"] == 0 and est["hits"] == 0


def test_bad_vertex_id_rejected(tc):
    import torch
    src = _dev(np.array([0, 1, 7], np.int32), torch.int32)
    dst = _dev(np.array([1, 2, 0], np.int32), torch.int32)
    t = _dev(np.array([1, 2, 3], np.int64), torch.int64)
    with pytest.raises(tc.TcError) as e:
        tc.tc_build_temporal_csr(5, src, dst, t)
    assert e.value.status == 1


def test_index_mismatch_rejected(tc):
    src, dst, t = small_random_graph(5, 8, 300, 100)
    g, _ = _build_both(tc, 8, src, dst, t)
    w = tc.tc_path_weights(g, tc.make_motif(C4), 30)
    with pytest.raises(tc.TcError) as e:          # other delta
        tc.tc_sample_estimate(g, tc.make_motif(C4), 31, w, 100, 0)
    assert e.value.status == 1
    with pytest.raises(tc.TcError) as e:          # other class
        tc.tc_sample_estimate(g, tc.make_motif(LATE_MID), 30, w, 100, 0)
    assert e.value.status == 1


def test_weight_overflow_detected(tc):
    # three groups of 2^22 parallel edges a->b, b->c, c->d at one time with
    # closed windows: every b->c edge has w = 2^22 * 2^22, W = 2^66 > 2^64
    import torch
    q = 1 << 22
    src = np.concatenate([np.full(q, 0), np.full(q, 1), np.full(q, 2)]).astype(np.int32)
    dst = np.concatenate([np.full(q, 1), np.full(q, 2), np.full(q, 3)]).astype(np.int32)
    t = np.zeros(3 * q, np.int64)
    g = tc.tc_build_temporal_csr(4, _dev(src, torch.int32), _dev(dst, torch.int32), _dev(t, torch.int64))
    mot = tc.make_motif([(0, 1), (1, 2), (2, 3)], window=1)
    with pytest.raises(tc.TcError) as e:
        tc.tc_path_weights(g, mot, 5)
    assert e.value.status == 3


def test_host_entry_point_matches_device_path(tc):
    from paper_2409_08975_gb300 import synth
    cfg = synth.dense_tiny(seed=1013, n=64)
    g, _ = _build_both(tc, cfg["n"], cfg["src"], cfg["dst"], cfg["t"])
    mot = tc.make_motif(C4)
    w = tc.tc_path_weights(g, mot, 10_000)
    a = tc.tc_sample_estimate(g, mot, 10_000, w, 200_000, 3, 0)
    b = tc.tc_estimate_from_host(cfg["n"], cfg["src"], cfg["dst"], cfg["t"], mot, 10_000, 200_000, 3)
    assert a == b


def test_weights_with_times_beyond_32_bits(tc):
    # a time span of 2^40 s: the window searches read the 64-bit list times
    # (the 32-bit offsets are only built when the span fits)
    src, dst, t = small_random_graph(19, 9, 400, 300, dup_frac=0.3)
    t = t * (1 << 32) - (1 << 40)
    g, og = _build_both(tc, 9, src, dst, t)
    for edges in (C4, CHORD, LATE_MID, [(0, 1), (0, 2), (1, 2)]):
        for window in (0, 1):
            plan = oracle.compile_motif(edges, closed=bool(window))
            mot = tc.make_motif(edges, window=window)
            for delta in (0, 3 << 32, 40 << 32):
                ow = oracle.path_weights(og, plan, delta)
                w = tc.tc_path_weights(g, mot, delta, want_w=True)
                assert (_u64(w.w)[:og.m] == ow["w"]).all(), (edges, window, delta)
                assert w.W == int(oracle.prefix_sum(ow["w"])[-1])
