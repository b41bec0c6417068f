"""Parity at the benchmark's full size: the 20M-edge Chung-Lu graph with the
path+chord motif, delta = 3600, in the launch configuration the benchmark
times.  The oracle builds its lists with numpy's lexsort (pinned equal to its
qsort build), so lists, weights, window records and prefix are compared in
full; sampling is compared on 200,000 traced samples and on the sums of the
untraced kernel over a sample-id range, and the 1e8-sample run is checked by
the exact merge of two disjoint halves."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_08975_gb300 import _build, synth, tc
    _build.build()
    cfg = synth.mid()
    n, src, dst, t = cfg["n"], cfg["src"], cfg["dst"], cfg["t"]
    dev = lambda a, dt: torch.from_numpy(a).to(device="cuda", dtype=dt)
    g = tc.tc_build_temporal_csr(n, dev(src, torch.int32), dev(dst, torch.int32), dev(t, torch.int64))
    og = oracle.build_csr(n, src, dst, t, sort="lexsort")
    plan = oracle.compile_motif(cfg["motif"])
    ow = oracle.path_weights(og, plan, cfg["delta"])
    opre = oracle.prefix_sum(ow["w"])
    mot = tc.make_motif(cfg["motif"])
    w = tc.tc_path_weights(g, mot, cfg["delta"], want_w=True)
    yield tc, cfg, g, og, plan, ow, opre, mot, w
    g.destroy()


def test_lists_full_size(setup):
    tc, cfg, g, og, *_ = setup
    oe = g.array("out_edges").view(-1, 4).cpu().numpy()
    assert (g.array("edge_perm").cpu().numpy() == og.out_perm).all()
    assert (oe[:, 0] == og.src[og.out_perm]).all() and (oe[:, 1] == og.dst[og.out_perm]).all()
    assert (g.array("out_off").cpu().numpy() == og.out_off).all()
    ie = g.array("in_edges").view(-1, 4).cpu().numpy()
    assert (ie[:, 1] == og.dst[og.in_perm]).all()
    assert (g.array("in_eid").cpu().numpy().astype(np.int64) == og.in_eid).all()
    assert (g.array("in_off").cpu().numpy() == og.in_off).all()
    assert g.num_pairs == og.P
    assert (g.array("pair_off").cpu().numpy() == og.pair_off).all()
    assert (g.array("pair_dst").cpu().numpy() == og.pair_dst).all()
    assert (g.array("pair_eoff").cpu().numpy() == og.pair_eoff).all()
    assert (g.array("pair_t").cpu().numpy() == og.t[og.pair_perm]).all()


def test_weights_full_size(setup):
    tc, cfg, g, og, plan, ow, opre, mot, w = setup
    m = og.m
    assert w.W == int(opre[-1]) > 0
    assert (w.w.cpu().numpy().view(np.uint64)[:m] == ow["w"]).all()
    assert (w.prefix.cpu().numpy().view(np.uint64) == opre).all()
    rec = w.index.cpu().numpy()[256:256 + 16 * m].view(np.uint32).reshape(m, 4)
    assert (rec[:, 0] == ow["lo1"]).all() and (rec[:, 1] == ow["d1"]).all()
    assert (rec[:, 2] == ow["lo3"]).all() and (rec[:, 3] == ow["d3"]).all()


def test_sampler_full_size(setup):
    tc, cfg, g, og, plan, ow, opre, mot, w = setup
    delta = cfg["delta"]
    seed = 0
    k = 200_000
    tr = tc.tc_sample_trace(g, mot, delta, w, k, seed, 0).cpu().numpy().view(np.uint64)
    osums, otr = oracle.sample_run(og, plan, delta, opre, k, seed, 0, trace=True)
    assert (tr == otr).all()
    # the untraced kernel (the benchmark's) over the same ids and over a late range
    est = tc.tc_sample_estimate(g, mot, delta, w, k, seed, 0)
    for key in ("sum_x", "sum_x2", "hits"):
        assert est[key] == osums[key]
    late = 99_000_000
    o2, _ = oracle.sample_run(og, plan, delta, opre, 50_000, seed, late)
    e2 = tc.tc_sample_estimate(g, mot, delta, w, 50_000, seed, late)
    for key in ("sum_x", "sum_x2", "hits"):
        assert e2[key] == o2[key]


def test_bench_launch_merges_exactly(setup):
    tc, cfg, g, og, plan, ow, opre, mot, w = setup
    K = cfg["k"]
    full = tc.tc_sample_estimate(g, mot, cfg["delta"], w, K, 0, 0)
    a = tc.tc_sample_estimate(g, mot, cfg["delta"], w, K // 2, 0, 0)
    b = tc.tc_sample_estimate(g, mot, cfg["delta"], w, K - K // 2, 0, K // 2)
    for key in ("sum_x", "sum_x2", "hits", "k"):
        assert a[key] + b[key] == full[key]
    assert full["hits"] > 0 and full["estimate"] > 0
    # the estimate's standard error is small at this k
    assert full["std_err"] < 0.05 * full["estimate"]
    # exact count by the exhaustive path sum: the estimate lies within five
    # standard errors, and the sum of squares gives that standard error
    ex = tc.tc_exact_count(g, mot, cfg["delta"], w)
    C, W = ex["sum_x"], ex["W"]
    assert abs(full["estimate"] - C) < 5 * full["std_err"]
    var = ex["sum_x2"] / W - (C / W) ** 2
    exact_se = W * (var / K) ** 0.5
    assert 0.9 * exact_se < full["std_err"] < 1.1 * exact_se
