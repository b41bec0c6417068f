"""The network's inference on the fifth-generation tensor cores (tcgen05 MMAs
into TMEM accumulators) against the oracle's forward pass and against the
warp-level mma.sync kernel: logits within the bf16 tolerances of the other
forward tests, for row counts at and around the 128-row MMA tile and the
2048-row scan tile; the proposal's q-prefix bit-exact with the oracle's on
the GPU's own h; h equal to the one the oracle derives from the logits
wherever a logit is not within rounding of a bin edge; the variance
objective's gradient (whose logits come from the inference kernel)."""
import numpy as np
import pytest

import oracle
from oracle import learned as L

pytestmark = pytest.mark.gpu

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
    before = tcmod.tc_mlp_kernel()
    yield tcmod
    tcmod.tc_mlp_kernel(before)


def _dev(a, dt):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)


@pytest.fixture(scope="module")
def setup(tc):
    import torch
    from paper_2409_08975_gb300 import synth
    c = synth.scaled_mid(3000, 60_000, seed=21)
    g = tc.tc_build_temporal_csr(c["n"], _dev(c["src"], torch.int32), _dev(c["dst"], torch.int32),
                                 _dev(c["t"], torch.int64))
    og = oracle.build_csr(c["n"], c["src"], c["dst"], c["t"])
    mot = tc.make_motif(CHORD)
    plan = oracle.compile_motif(CHORD)
    w = tc.tc_path_weights(g, mot, 3600, want_w=True)
    feat = tc.tc_edge_features(g, mot, 3600, w)
    tc.tc_sample_features(g, mot, 3600, w, feat, 50_000, seed=11)
    mlp = tc.MLP(seed=1)
    flat = L.pack(L.init_params(np.random.default_rng(9))).astype(np.float32)
    mlp.set_params(flat)
    return g, og, mot, plan, w, feat, mlp, L.unpack(flat.astype(np.float64))


def _logits(tc, kind, mlp, feat, rows):
    import torch
    assert tc.tc_mlp_kernel(kind) == kind
    r = None if rows is None else _dev(rows, torch.int32)
    return tc.tc_mlp_forward(mlp, feat, r, n=None if rows is not None else feat.shape[0]).cpu().numpy()


@pytest.mark.parametrize("nrows", [1, 127, 128, 129, 2047, 2048, 2049, 5000])
def test_logits_match_oracle_and_mma(tc, setup, nrows):
    g, og, mot, plan, w, feat, mlp, p32 = setup
    rows = np.random.default_rng(nrows).integers(0, g.m, nrows).astype(np.int32)
    x = feat.to(dtype=__import__("torch").float32).cpu().numpy()[rows]
    z_ref, _ = L.mlp_forward(p32, x)
    z5 = _logits(tc, "tcgen05", mlp, feat, rows)
    zm = _logits(tc, "mma", mlp, feat, rows)
    assert z5.shape == (nrows,)
    assert np.isfinite(z5).all()
    assert np.abs(z5 - z_ref).max() < 2e-2
    assert np.abs(z5 - z_ref).mean() < 1e-3
    # the two kernels differ only in the order of FP32 sums
    assert np.abs(z5 - zm).max() < 2e-2
    assert np.abs(z5 - zm).mean() < 1e-3


def test_logits_of_every_edge(tc, setup):
    g, og, mot, plan, w, feat, mlp, p32 = setup
    x = feat.to(dtype=__import__("torch").float32).cpu().numpy()
    z_ref, _ = L.mlp_forward(p32, x)
    z5 = _logits(tc, "tcgen05", mlp, feat, None)
    assert z5.shape == (g.m,) and g.m % 2048 != 0 and g.m > 2048 * 16
    assert np.abs(z5 - z_ref).max() < 2e-2
    assert np.abs(z5 - z_ref).mean() < 1e-3


def test_proposal_bit_exact_on_its_h(tc, setup):
    g, og, mot, plan, w, feat, mlp, p32 = setup
    tc.tc_mlp_kernel("tcgen05")
    prop = tc.tc_proposal_weights(mlp, g, mot, 3600, w, feat)
    h5 = prop.h.cpu().numpy().view(np.uint16).astype(np.int64)
    ow = oracle.path_weights(og, plan, 3600)["w"]
    qpre = L.qprefix(ow, h5)
    assert prop.Q == int(qpre[-1])
    assert (prop.qprefix.cpu().numpy().view(np.uint64) == qpre).all()
    # h from the kernel's logits: the oracle's rule on the tcgen05 logits,
    # except where sigmoid rounding puts a logit on the other side of a bin
    z5 = _logits(tc, "tcgen05", mlp, feat, None)
    g32 = (np.float32(1) / (np.float32(1) + np.exp(-z5.astype(np.float32)))).astype(np.float32)
    h_ref = np.where(ow > 0, L.proposal_h(g32, 0.05, 1024).astype(np.int64), 1)  # w = 0: never drawn, h = 1
    assert np.abs(h5 - h_ref).max() <= 1
    assert (h5 != h_ref).mean() < 1e-3
    # and against the mma.sync kernel's proposal
    tc.tc_mlp_kernel("mma")
    prop_m = tc.tc_proposal_weights(mlp, g, mot, 3600, w, feat)
    hm = prop_m.h.cpu().numpy().view(np.uint16).astype(np.int64)
    assert np.abs(h5 - hm).max() <= 1
    assert (h5 != hm).mean() < 1e-3
    # the sampler on the tcgen05 proposal, bit-exact with the oracle on its h
    tc.tc_mlp_kernel("tcgen05")
    out = tc.tc_sample_estimate_q(g, mot, 3600, w, prop, 20_000, seed=7, trace=True)
    _, otr = L.sample_run_q(og, plan, 3600, qpre, h5, 20_000, 7, 0, trace=True)
    assert (out["trace"].cpu().numpy().view(np.uint64) == otr).all()


def test_variance_gradient_through_tcgen05(tc, setup):
    import torch
    g, og, mot, plan, w, feat, mlp, p32 = setup
    tc.tc_mlp_kernel("tcgen05")
    rng = np.random.default_rng(12)
    for nrows in (5000, 77):
        rows = rng.integers(0, g.m, nrows).astype(np.int32)
        x = feat.to(torch.float32).cpu().numpy()[rows]
        y = np.where(rng.random(nrows) < 0.8, 0, rng.integers(1, 6, nrows)).astype(np.float32)
        grad, loss = tc.tc_mlp_grad(mlp, feat, _dev(rows, torch.int32), _dev(y, torch.float32),
                                    objective="variance", eps=0.05)
        gref, lref = L.mlp_backward(p32, x, y.astype(np.float64), objective="variance", eps=0.05)
        gref_flat = L.pack(gref)
        gg = grad.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(gg - gref_flat) <= 1e-2 * np.linalg.norm(gref_flat), nrows
        assert loss == pytest.approx(lref, rel=1e-3)
