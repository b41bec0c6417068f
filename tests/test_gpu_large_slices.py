"""The GPU's exact count at the scale of the 300M-edge transaction-like
graph, against the oracle's enumerator: contiguous time slices holding 1% of
that graph's edges (3e6 each) are counted by the oracle's chronological
backtracking over the motif's edges (the literal Def. 2, all host cores) and
by the library's exhaustive path sum (tc_exact_count, the proof of Claim 2),
which must agree bit for bit; the weights total W agrees with the oracle's
Claim 1 weights, and a sampled estimate on the slice lies within 5 standard
errors of the count."""
import os

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

C4 = [(0, 1), (1, 2), (2, 3), (3, 0)]
PATH_CHORD = [(0, 1), (1, 2), (2, 3), (0, 3)]
DELTA = 3600


@pytest.fixture(scope="module")
def large():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_08975_gb300 import _build, synth, tc
    _build.build()
    return tc, synth, synth.large()


@pytest.mark.parametrize("j,motif", [(0, C4), (0, PATH_CHORD), (50, C4)], ids=["first_c4", "first_chord", "mid_c4"])
def test_slice_exact_count_matches_oracle(large, j, motif):
    import torch
    tc, synth, cfg = large
    s = synth.time_slice(cfg, j, 100)
    m = len(s["src"])
    assert abs(m - 3_000_000) < 30_000
    og = oracle.build_csr(s["n"], s["src"], s["dst"], s["t"], sort="lexsort")
    plan = oracle.compile_motif(motif)
    W_or = int(oracle.prefix_sum(oracle.path_weights(og, plan, DELTA)["w"])[-1])
    try:
        oracle.set_threads(os.cpu_count() or 1)
        C = oracle.exact_count(og, motif, DELTA)
    finally:
        oracle.set_threads(1)
    dev = lambda a, dt: torch.from_numpy(a).to(device="cuda", dtype=dt)
    g = tc.tc_build_temporal_csr(s["n"], dev(s["src"], torch.int32), dev(s["dst"], torch.int32),
                                 dev(s["t"], torch.int64))
    mot = tc.make_motif(motif)
    w = tc.tc_path_weights(g, mot, DELTA)
    assert w.W == W_or > 0
    ex = tc.tc_exact_count(g, mot, DELTA, w)
    assert ex["k"] == w.W
    assert ex["sum_x"] == C > 0
    est = tc.tc_sample_estimate(g, mot, DELTA, w, 100_000_000, seed=j + 1)
    assert abs(est["estimate"] - C) <= 5 * est["std_err"]
    g.destroy()
