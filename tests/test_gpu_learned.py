"""Learned proposal on the GPU against the oracle: features (within one bf16
step), network forward and gradients (tolerances from bf16 arithmetic),
proposal prefix, sampled indices and per-h bins (bit-exact, with the oracle
taking the GPU's h as input), unbiasedness, and the variance the trained
network saves over the plain proposal."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import learned as L
from _graphs import small_random_graph

pytestmark = pytest.mark.gpu

C4 = [(0, 1), (1, 2), (2, 3), (3, 0)]
CHORD = [(0, 1), (1, 2), (2, 3), (0, 3)]


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


def _setup(tc, n, src, dst, t, motif, delta):
    import torch
    g = tc.tc_build_temporal_csr(n, _dev(src, torch.int32), _dev(dst, torch.int32), _dev(t, torch.int64))
    og = oracle.build_csr(n, src, dst, t)
    mot = tc.make_motif(motif)
    plan = oracle.compile_motif(motif)
    w = tc.tc_path_weights(g, mot, delta, want_w=True)
    feat = tc.tc_edge_features(g, mot, delta, w)
    return g, og, mot, plan, w, feat


def _graph_bursty():
    from paper_2409_08975_gb300 import synth
    c = synth.scaled_mid(3000, 60_000, seed=21)
    return c["n"], c["src"], c["dst"], c["t"]


def _f32(feat):
    import torch
    return feat.to(torch.float32).cpu().numpy()


def test_features_within_one_bf16_step(tc):
    n, src, dst, t = _graph_bursty()
    g, og, mot, plan, w, feat = _setup(tc, n, src, dst, t, CHORD, 3600)
    got = _f32(feat)
    exp = L.features_bf16(L.edge_features(og, plan, 3600))
    assert got.shape == exp.shape
    assert (got[:, 12:] == 0).all()
    # an edge with w = 0 is never drawn: its row is zero; the others are the oracle's
    live = oracle.path_weights(og, plan, 3600)["w"] > 0
    assert live.any() and not live.all()
    assert (got[~live] == 0).all()
    got, exp = got[live], exp[live]
    diff = np.abs(got - exp)
    step = np.maximum(np.abs(exp), 1e-30) * 2.0 ** -7
    assert (diff <= step).all()
    assert (diff == 0).mean() > 0.999


def test_sample_features_match_oracle(tc):
    # columns 12..15 from 50,000 plain samples, against the oracle's
    # statistics of the same samples, within one bf16 step
    n, src, dst, t = _graph_bursty()
    g, og, mot, plan, w, feat = _setup(tc, n, src, dst, t, CHORD, 3600)
    before = _f32(feat)[:, :12].copy()
    tc.tc_sample_features(g, mot, 3600, w, feat, 50_000, seed=11, offset=3)
    got = _f32(feat)
    assert (got[:, :12] == before).all()
    ow = oracle.path_weights(og, plan, 3600)["w"]
    pre = oracle.prefix_sum(ow)
    exp = L.features_bf16(L.edge_features(og, plan, 3600), L.sample_features(og, plan, 3600, pre, 50_000, 11, 3))
    live = ow > 0
    assert (got[~live] == 0).all()  # rows of edges that are never drawn stay zero
    got, exp = got[live], exp[live]
    diff = np.abs(got[:, 12:] - exp[:, 12:])
    step = np.maximum(np.abs(exp[:, 12:]), 1e-30) * 2.0 ** -7
    assert (diff <= step).all()
    assert (diff == 0).mean() > 0.999
    assert (got[:, 15] > 0).any() and (got[:, 15] == 0).any()


def test_forward_and_gradient_match_fp64(tc):
    import torch
    n, src, dst, t = _graph_bursty()
    g, og, mot, plan, w, feat = _setup(tc, n, src, dst, t, CHORD, 3600)
    tc.tc_sample_features(g, mot, 3600, w, feat, 50_000, seed=11)
    params = L.init_params(np.random.default_rng(9))
    flat = L.pack(params).astype(np.float32)
    mlp = tc.MLP(seed=1)
    mlp.set_params(flat)
    assert np.array_equal(mlp.get_params(), flat)
    p32 = L.unpack(flat.astype(np.float64))
    rng = np.random.default_rng(2)
    rows = rng.integers(0, g.m, 5000).astype(np.int32)
    x = _f32(feat)[rows]
    z_gpu = tc.tc_mlp_forward(mlp, feat, _dev(rows, torch.int32)).cpu().numpy()
    z_ref, _ = L.mlp_forward(p32, x)
    assert np.abs(z_gpu - z_ref).max() < 2e-2
    assert np.abs(z_gpu - z_ref).mean() < 1e-3
    y = np.where(rng.random(5000) < 0.8, 0, rng.integers(1, 6, 5000)).astype(np.float32)  # closure counts
    grad, loss = tc.tc_mlp_grad(mlp, feat, _dev(rows, torch.int32), _dev(y, torch.float32))
    gref, lref = L.mlp_backward(p32, x, y.astype(np.float64))
    gref_flat = L.pack(gref)
    gg = grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gg - gref_flat) <= 1e-2 * np.linalg.norm(gref_flat)
    assert abs(loss - lref) < 1e-3
    # the binary cross-entropy on the closure outcome 1[X > 0]: the oracle's
    # closure loss on labels clipped to 1
    grad, loss = tc.tc_mlp_grad(mlp, feat, _dev(rows, torch.int32), _dev(y, torch.float32), objective="bce")
    gref, lref = L.mlp_backward(p32, x, np.minimum(y, 1).astype(np.float64))
    gref_flat = L.pack(gref)
    gg = grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gg - gref_flat) <= 1e-2 * np.linalg.norm(gref_flat)
    assert abs(loss - lref) < 1e-3


def test_variance_objective_gradient_matches_fp64(tc):
    import torch
    n, src, dst, t = _graph_bursty()
    g, og, mot, plan, w, feat = _setup(tc, n, src, dst, t, CHORD, 3600)
    tc.tc_sample_features(g, mot, 3600, w, feat, 50_000, seed=11)
    params = L.init_params(np.random.default_rng(19))
    flat = L.pack(params).astype(np.float32)
    mlp = tc.MLP(seed=1)
    mlp.set_params(flat)
    p32 = L.unpack(flat.astype(np.float64))
    rng = np.random.default_rng(12)
    for nrows in (5000, 77):        # several tiles, and one ragged tile
        rows = rng.integers(0, g.m, nrows).astype(np.int32)
        x = _f32(feat)[rows]
        y = np.where(rng.random(nrows) < 0.8, 0, rng.integers(1, 6, nrows)).astype(np.float32)
        grad, loss = tc.tc_mlp_grad(mlp, feat, _dev(rows, torch.int32), _dev(y, torch.float32),
                                    objective="variance", eps=0.05)
        gref, lref = L.mlp_backward(p32, x, y.astype(np.float64), objective="variance", eps=0.05)
        gref_flat = L.pack(gref)
        gg = grad.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(gg - gref_flat) <= 1e-2 * np.linalg.norm(gref_flat), nrows
        assert loss == pytest.approx(lref, rel=1e-3)
    with pytest.raises(tc.TcError):
        tc.tc_mlp_grad(mlp, feat, _dev(rows, torch.int32), _dev(y, torch.float32), objective="variance", eps=0.0)


def _trained(tc, setup, n_train, seed=3, objective="closure"):
    g, og, mot, plan, w, feat = setup
    delta = 3600 if og.n > 100 else 10_000
    tc.tc_sample_features(g, mot, delta, w, feat, n_train, seed=seed + 1000)  # samples disjoint from training
    mlp = tc.MLP(seed=seed)
    first, last = tc.tc_mlp_train(mlp, g, mot, delta, w, feat, n_train, seed=seed, batch=4096, lr=3e-3,
                                  objective=objective)
    return mlp, first, last


def test_training_lowers_loss(tc):
    n, src, dst, t = _graph_bursty()
    setup = _setup(tc, n, src, dst, t, CHORD, 3600)
    w1_init = L.unpack(tc.MLP(seed=3).get_params())["W1"]
    mlp, first, last = _trained(tc, setup, 400_000)
    assert last < 0.8 * first
    # every input column, the sample statistics included, is trained
    w1 = L.unpack(mlp.get_params())["W1"]
    assert (np.abs(w1 - w1_init).max(axis=0) > 1e-3).all()


def test_proposal_prefix_and_sampler_bit_exact(tc):
    n, src, dst, t = _graph_bursty()
    g, og, mot, plan, w, feat = setup = _setup(tc, n, src, dst, t, CHORD, 3600)
    mlp, _, _ = _trained(tc, setup, 200_000)
    prop = tc.tc_proposal_weights(mlp, g, mot, 3600, w, feat)
    h = prop.h.cpu().numpy().view(np.uint16)
    ow = oracle.path_weights(og, plan, 3600)["w"]
    live = ow > 0
    assert live.any() and not live.all()
    assert h[live].min() >= 51 and h[live].max() <= 1075   # eps = 0.05, scale = 1024
    assert (h[~live] == 1).all()                            # never drawn: the network is not run on them
    qpre = L.qprefix(ow, h)
    assert prop.Q == int(qpre[-1])
    assert (prop.qprefix.cpu().numpy().view(np.uint64) == qpre).all()
    for k, off in ((30_000, 5), (100_000, 1 << 33)):        # id order, key order
        out = tc.tc_sample_estimate_q(g, mot, 3600, w, prop, k, seed=7, offset=off, want_bins=True, trace=True)
        osum, otr = L.sample_run_q(og, plan, 3600, qpre, h, k, 7, off, trace=True)
        assert (out["trace"].cpu().numpy().view(np.uint64) == otr).all()
        lo = osum["h_lo"]
        bins = out["bins"]
        for j, (b, b2) in enumerate(zip(osum["B"], osum["B2"])):
            assert int(bins[lo + j, 0]) == b
            assert int(bins[lo + j, 1]) | (int(bins[lo + j, 2]) << 64) == b2
        est, se = L.estimate_q(osum["B"], osum["B2"], lo, prop.Q, k)
        assert out["estimate"] == pytest.approx(est, rel=1e-12)
        assert out["std_err"] == pytest.approx(se, rel=1e-9)
        assert out["hits"] == osum["hits"]


def test_proposal_unbiased_over_1000_seeds(tc):
    src, dst, t = small_random_graph(77, 6, 60, 60, dup_frac=0.3)
    g, og, mot, plan, w, feat = setup = _setup(tc, 6, src, dst, t, C4, 20)
    mlp = tc.MLP(seed=4)
    tc.tc_sample_features(g, mot, 20, w, feat, 20_000, seed=5)
    tc.tc_mlp_train(mlp, g, mot, 20, w, feat, 20_000, seed=4, batch=512, lr=1e-2)
    prop = tc.tc_proposal_weights(mlp, g, mot, 20, w, feat, eps=0.05, scale=64)
    h = prop.h.cpu().numpy().view(np.uint16)
    C = oracle.brute_force_count(src, dst, t, C4, 20)
    h_lo, S1, S2 = L.path_sum_q(og, plan, 20, h)
    assert sum(S1) == C > 0
    var = L.exact_variance_q(prop.Q, C, h_lo, S2)
    k = 200
    ests = [tc.tc_sample_estimate_q(g, mot, 20, w, prop, k, seed=s)["estimate"] for s in range(1000)]
    assert abs(np.mean(ests) - C) <= 2.576 * math.sqrt(float(var) / k / 1000)


@pytest.mark.parametrize("objective", ["closure", "variance", "bce"])
def test_trained_network_reduces_variance(tc, objective):
    # exact per-sample variances from all paths: plain W sum C_P^2 - C^2,
    # learned Q sum C_P^2 / h_P - C^2, after training on plain samples
    n, src, dst, t = _graph_bursty()
    g, og, mot, plan, w, feat = setup = _setup(tc, n, src, dst, t, CHORD, 3600)
    mlp, _, _ = _trained(tc, setup, 400_000, objective=objective)
    prop = tc.tc_proposal_weights(mlp, g, mot, 3600, w, feat)
    h = prop.h.cpu().numpy().view(np.uint16)
    ps = oracle.path_sum(og, plan, 3600)
    C, W = ps["C"], w.W
    var_plain = Fraction(W) * ps["sum_x2"] - C * C
    h_lo, S1, S2 = L.path_sum_q(og, plan, 3600, h)
    assert sum(S1) == C
    var_learned = L.exact_variance_q(prop.Q, C, h_lo, S2)
    assert var_learned < 0.9 * var_plain, (float(var_learned / var_plain))
