"""The allocation-free prefix sum (tc_prefix_sum_noalloc) gives the same
prefix as tc_path_weights.

That entry point serves callers that cannot allocate device memory (their
device memory belongs to another allocator, or they run under a hard memory
budget); it keeps its scratch in a static device array instead.  This file is
collected last so that a failure here cannot stop the other tests."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


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


def _graph(tc):
    import torch
    from paper_2409_08975_gb300 import synth
    cfg = synth.scaled_mid(50_000, 1_500_000, seed=11)
    dev = lambda a, dt: torch.from_numpy(a).to(device="cuda", dtype=dt)
    g = tc.tc_build_temporal_csr(cfg["n"], dev(cfg["src"], torch.int32), dev(cfg["dst"], torch.int32),
                                 dev(cfg["t"], torch.int64))
    return g


def test_noalloc_prefix_matches_path_weights_twice(tc):
    import torch
    g = _graph(tc)
    m = g.m
    # two calls in a row on different weights: the shared scratch keeps the
    # first call's tile sums, which the second call must not depend on
    cases = [([(0, 1), (1, 2), (2, 3), (0, 3)], 3600), ([(1, 2), (0, 1), (2, 3), (3, 0)], 600)]
    for edges, delta in cases:
        ref = tc.tc_path_weights(g, tc.make_motif(edges), delta, want_w=True)
        out = torch.full((m + 1,), -1, dtype=torch.int64, device="cuda")
        W = tc.tc_prefix_sum_noalloc(ref.w[:m], m, out)
        torch.cuda.synchronize()
        assert W == ref.W > 0
        assert torch.equal(out, ref.prefix)


def test_noalloc_small_and_empty(tc):
    import torch
    w = torch.tensor([5, 0, 7, 1 << 40], dtype=torch.int64, device="cuda")
    out = torch.empty(5, dtype=torch.int64, device="cuda")
    assert tc.tc_prefix_sum_noalloc(w, 4, out) == 12 + (1 << 40)
    assert out.cpu().tolist() == [0, 5, 5, 12, 12 + (1 << 40)]
    assert tc.tc_prefix_sum_noalloc(w, 0, out) == 0


def test_noalloc_rejects_beyond_maximum(tc):
    import torch
    w = torch.zeros(4, dtype=torch.int64, device="cuda")
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    with pytest.raises(tc.TcError) as e:
        tc.tc_prefix_sum_noalloc(w, tc.NOALLOC_MAX_EDGES + 1, out)
    assert e.value.status == 1
    assert "TC_NOALLOC_MAX_EDGES" in str(e.value)
    assert out.cpu().tolist() == [0, 0, 0, 0]


def test_noalloc_two_scan_levels_match_cumsum(tc):
    """More than 2048 x 2048 weights: the scan's second level of tile sums
    sits after the first in the static array."""
    import torch
    m = 5_000_003
    g = torch.Generator(device="cpu").manual_seed(4)
    w = torch.randint(0, 1 << 20, (m,), generator=g, dtype=torch.int64).cuda()
    ref = torch.zeros(m + 1, dtype=torch.int64, device="cuda")
    ref[1:] = torch.cumsum(w, 0)
    out = torch.full((m + 1,), -1, dtype=torch.int64, device="cuda")
    for _ in range(2):  # twice in a row on the same array
        W = tc.tc_prefix_sum_noalloc(w, m, out)
        torch.cuda.synchronize()
        assert W == int(ref[-1])
        assert torch.equal(out, ref)


def test_noalloc_reports_overflow(tc):
    import torch
    w = torch.tensor([1 << 62, 1 << 62, 1 << 62, 1 << 62], dtype=torch.int64, device="cuda")
    out = torch.empty(5, dtype=torch.int64, device="cuda")
    with pytest.raises(tc.TcError) as e:
        tc.tc_prefix_sum_noalloc(w, 4, out)
    assert e.value.status == 3
    # the error word starts from zero again on the next call
    assert tc.tc_prefix_sum_noalloc(w, 2, out) == 1 << 63
