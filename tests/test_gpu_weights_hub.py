"""Path weights on lists longer than an anchor's range word can tell.

The weights kernel takes a list's bounds from 16-bit distances stored with
each window anchor and reads the list's offsets only where a distance is
saturated (65,535 or more entries away).  Here a hub sends and receives
150,000 edges each, so the u and v sides of every anchor kind (u's in-list,
u's out-list, v's in-list, v's out-list) search lists of both kinds; the
weights and windows of all sixteen anchor classes (Def. 5), strict and
closed, must equal the oracle's bit for bit."""
import numpy as np
import pytest

import oracle
from _graphs import path_motifs_all_classes

pytestmark = pytest.mark.gpu

HUB_EDGES = 150_000
LEAVES = 39


def _hub_graph(seed=31):
    rng = np.random.default_rng(seed)
    leaf_out = rng.integers(1, LEAVES + 1, HUB_EDGES)     # hub -> leaf
    leaf_in = rng.integers(1, LEAVES + 1, HUB_EDGES)      # leaf -> hub
    src = np.concatenate([np.zeros(HUB_EDGES, np.int32), leaf_in.astype(np.int32)])
    dst = np.concatenate([leaf_out.astype(np.int32), np.zeros(HUB_EDGES, np.int32)])
    t = rng.integers(0, 1_000_000, 2 * HUB_EDGES).astype(np.int64)  # ties included
    perm = rng.permutation(2 * HUB_EDGES)
    return LEAVES + 1, src[perm], dst[perm], t[perm]


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


def test_hub_weights_all_classes_bit_exact(tc):
    import torch
    n, src, dst, t = _hub_graph()
    og = oracle.build_csr(n, src, dst, t)
    assert np.diff(og.out_off)[0] == HUB_EDGES and np.diff(og.in_off)[0] == HUB_EDGES
    dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)
    g = tc.tc_build_temporal_csr(n, dev(src, torch.int32), dev(dst, torch.int32), dev(t, torch.int64))
    for edges in path_motifs_all_classes():
        for window in (0, 1):
            plan = oracle.compile_motif(edges, closed=bool(window))
            ow = oracle.path_weights(og, plan, 200)
            w = tc.tc_path_weights(g, tc.make_motif(edges, window=window), 200, want_w=True)
            assert w.W == int(ow["w"].sum(dtype=np.uint64)), (edges, window)
            assert (w.w.cpu().numpy().view(np.uint64)[:og.m] == ow["w"]).all(), (edges, window)
            rec = w.index.cpu().numpy()[256:256 + 16 * og.m].view(np.uint32).reshape(og.m, 4)
            assert (rec[:, 0] == ow["lo1"]).all() and (rec[:, 1] == ow["d1"]).all(), (edges, window)
            assert (rec[:, 2] == ow["lo3"]).all() and (rec[:, 3] == ow["d3"]).all(), (edges, window)
    g.destroy()
