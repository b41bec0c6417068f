"""Wedge sampling for 3-vertex motifs on the GPU against the oracle, element
by element: weights, prefix and window records bit-exact, traced samples
(base edge, second-edge position, X) and sums bit-exact in id order and in
key order, the exhaustive wedge sum equal to the oracle's (itself pinned to
the literal count), and wedge queries inside a batch equal to single runs."""
import numpy as np
import pytest

import oracle
from _graphs import small_random_graph

pytestmark = pytest.mark.gpu

FF = [(0, 1), (0, 2), (1, 2)]
CYC = [(0, 1), (1, 2), (2, 0)]
IN_DST = [(0, 1), (2, 1), (0, 2)]
IN_SRC = [(0, 1), (2, 0), (2, 1)]
WEDGE2 = [(0, 1), (0, 2)]
MULTI3 = [(0, 1), (0, 2), (0, 1), (1, 2), (0, 2)]
GAP0 = [(0, 1), (1, 0), (0, 1), (1, 2), (2, 1)]
ZOO = [FF, CYC, IN_DST, IN_SRC, WEDGE2, MULTI3, GAP0]
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


def _u64(x):
    return x.cpu().numpy().view(np.uint64)


def _graphs():
    from paper_2409_08975_gb300 import synth
    out = []
    s, d, t = small_random_graph(3, 9, 300, 200, dup_frac=0.3)
    out.append(("small", 9, s, d, t, 60))
    g = synth.dense_tiny()
    out.append(("dense24", g["n"], g["src"], g["dst"], g["t"], 10_000))
    g = synth.dense_tiny(seed=1012, n=200, bursty=True)
    out.append(("dense200b", g["n"], g["src"], g["dst"], g["t"], 10_000))
    g = synth.scaled_mid(5000, 61_237, seed=7)
    out.append(("cl61k", g["n"], g["src"], g["dst"], g["t"], 3600))
    return out


GRAPHS = _graphs()


def _build_both(tc, n, src, dst, t):
    import torch
    g = tc.tc_build_temporal_csr(n, _dev(src, torch.int32), _dev(dst, torch.int32), _dev(t, torch.int64))
    return g, oracle.build_csr(n, src, dst, t)


def test_wedge_plan_matches_oracle(tc):
    for edges in ZOO:
        anchor, cls = tc.tc_motif_plan(tc.make_motif(edges))
        p = oracle.compile_motif(edges)
        assert anchor == (p.e1, p.mid, p.e3)
        assert cls == (p.alpha1, p.alpha3, p.beta1, p.beta3)


@pytest.mark.parametrize("case", GRAPHS, ids=lambda c: c[0])
def test_wedge_weights_and_sampler_bit_exact(tc, case):
    name, n, src, dst, t, delta = case
    g, og = _build_both(tc, n, src, dst, t)
    for edges in ZOO:
        for window in (0, 1):
            plan = oracle.compile_motif(edges, closed=bool(window))
            mot = tc.make_motif(edges, window=window)
            ow = oracle.path_weights(og, plan, delta)
            opre = oracle.prefix_sum(ow["w"])
            w = tc.tc_path_weights(g, mot, delta, want_w=True)
            assert w.W == int(opre[-1])
            m = og.m
            assert (_u64(w.w)[:m] == ow["w"]).all(), (edges, window)
            assert (_u64(w.prefix) == opre).all()
            rec = w.index.cpu().numpy()[256:256 + 16 * m].view(np.uint32).reshape(m, 4)
            assert (rec[:, 0] == ow["lo1"]).all() and (rec[:, 1] == ow["d1"]).all()
            assert (rec[:, 2] == ow["lo3"]).all() and (rec[:, 3] == ow["d3"]).all()
            if w.W == 0:
                continue
            k, seed, off = 20_000, 4242, 31
            tr = _u64(tc.tc_sample_trace(g, mot, delta, w, k, seed, off))
            osums, otr = oracle.sample_run(og, plan, delta, opre, k, seed, off, trace=True)
            assert (tr == otr).all(), (edges, window)
            est = tc.tc_sample_estimate(g, mot, delta, w, k, seed, off)
            for key in ("sum_x", "sum_x2", "hits", "k"):
                assert est[key] == osums[key], key
            c_hat, se = oracle.estimate(osums["sum_x"], osums["sum_x2"], k, int(opre[-1]))
            assert est["estimate"] == pytest.approx(c_hat, rel=REL_TOL, abs=0)


@pytest.mark.parametrize("case", GRAPHS[1:], ids=lambda c: c[0])
def test_wedge_key_sorted_and_exact_sum(tc, case):
    name, n, src, dst, t, delta = case
    g, og = _build_both(tc, n, src, dst, t)
    for edges in (FF, CYC, MULTI3):
        plan = oracle.compile_motif(edges)
        mot = tc.make_motif(edges)
        w = tc.tc_path_weights(g, mot, delta)
        opre = oracle.prefix_sum(oracle.path_weights(og, plan, delta)["w"])
        k, seed, off = 70_001, 7, 1 << 35
        osums, _ = oracle.sample_run(og, plan, delta, opre, k, seed, off)
        est = tc.tc_sample_estimate(g, mot, delta, w, k, seed, off)
        for key in ("sum_x", "sum_x2", "hits"):
            assert est[key] == osums[key]
        r = tc.tc_exact_count(g, mot, delta, w)
        ps = oracle.path_sum(og, plan, delta)
        assert r["sum_x"] == ps["C"] and r["sum_x2"] == ps["sum_x2"] and r["k"] == ps["paths"] == w.W


def test_wedge_exact_count_equals_literal_count(tc):
    import torch
    for seed in range(3):
        src, dst, t = small_random_graph(300 + seed, 5, 40, 30, dup_frac=0.4)
        g = tc.tc_build_temporal_csr(5, _dev(src, torch.int32), _dev(dst, torch.int32), _dev(t, torch.int64))
        for edges in (FF, CYC, IN_DST, IN_SRC, WEDGE2):
            for delta in (4, 15):
                mot = tc.make_motif(edges)
                w = tc.tc_path_weights(g, mot, delta)
                C = oracle.brute_force_count(src, dst, t, edges, delta)
                assert tc.tc_exact_count(g, mot, delta, w)["sum_x"] == C, (seed, edges, delta)


def test_wedge_queries_in_a_batch(tc):
    case = GRAPHS[3]
    g, _ = _build_both(tc, *case[1:5])
    qs = [(g, e, d, k, 5, 0) for e in ZOO for d, k in ((600, 80_000), (3600, 3000))]
    qs.append((g, [(0, 1), (1, 2), (2, 3), (0, 3)], 3600, 100_000, 1, 0))
    res = tc.Batch(qs, block_size=256, tile=2048).run()
    for (gq, edges, delta, k, seed, off), r in zip(qs, res):
        mot = tc.make_motif(edges)
        w = tc.tc_path_weights(g, mot, delta)
        a = tc.tc_sample_estimate(g, mot, delta, w, k, seed, off)
        for key in ("W", "sum_x", "sum_x2", "hits", "checked"):
            assert r[key] == a[key], (edges, delta, key)
