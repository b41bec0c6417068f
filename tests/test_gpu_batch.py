"""Batched queries (tc_batch_*): every query's sums from the one persistent
launch (replayed from a CUDA graph or issued directly) equal, bit for bit,
those of the same query run alone through tc_sample_estimate, and a subset
equals the CPU oracle's; replays repeat exactly."""
import itertools

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

C4 = [(0, 1), (1, 2), (2, 3), (3, 0)]
CHORD = [(0, 1), (1, 2), (2, 3), (0, 3)]
M41 = [(0, 1), (1, 2), (2, 3), (3, 2), (2, 1), (1, 0), (0, 1), (1, 2), (2, 3)]
MULTI = [(0, 1), (1, 2), (1, 2), (2, 3), (3, 0), (0, 2)]
KEYS = ("W", "k", "sum_x", "sum_x2", "hits", "checked")


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


@pytest.fixture(scope="module")
def graphs(tc):
    import torch
    from paper_2409_08975_gb300 import synth
    out = []
    for cfg in (synth.dense_tiny(), synth.dense_tiny(seed=1012, n=200, bursty=True),
                synth.scaled_mid(5000, 61_237, seed=7)):
        g = tc.tc_build_temporal_csr(cfg["n"], _dev(cfg["src"], torch.int32), _dev(cfg["dst"], torch.int32),
                                     _dev(cfg["t"], torch.int64))
        out.append((g, cfg))
    yield out
    for g, _ in out:
        g.destroy()


def _queries(tc, graphs):
    """All 24 rank orders of the directed 4-cycle on the largest graph at two
    windows, other motifs and window kinds on the others, with k spanning
    empty, id-order (below 65536) and key-order runs."""
    rng = np.random.default_rng(5)
    ks = [0, 1, 999, 4096, 65_536, 70_001, 200_000]
    qs = []
    g_big = graphs[2][0]
    for i, perm in enumerate(itertools.permutations(range(4))):
        edges = [C4[j] for j in perm]
        for delta in (600, 10_000):
            qs.append((g_big, edges, delta, ks[(i + delta) % len(ks)], 11 + i, int(rng.integers(0, 1 << 40))))
    for g, _ in graphs[:2]:
        for edges in (CHORD, M41, MULTI):
            for window in (0, 1):
                mot = tc.make_motif(edges, window=window)
                qs.append((g, mot, 10_000, ks[len(qs) % len(ks)], len(qs), 0))
    return qs


def _alone(tc, q):
    g, motif, delta, k, seed, offset = q
    mot = motif if isinstance(motif, tc.tc_motif) else tc.make_motif(motif)
    w = tc.tc_path_weights(g, mot, delta)
    return tc.tc_sample_estimate(g, mot, delta, w, k, seed, offset)


def _same(a, b):
    for key in KEYS:
        assert a[key] == b[key], key
    if a["k"] and a["W"]:
        assert a["estimate"] == b["estimate"]


def test_batch_matches_single_queries(tc, graphs):
    qs = _queries(tc, graphs)
    alone = [_alone(tc, q) for q in qs]
    for opts in (dict(block_size=128, tile=2048), dict(block_size=512, tile=32768),
                 dict(block_size=256, tile=8192, use_graph=False)):
        b = tc.Batch(qs, **opts)
        res = b.run()
        for q, r, a in zip(qs, res, alone):
            _same(r, a)
        again = b.run()
        for r, a in zip(res, again):
            _same(r, a)
        info = b.info()
        assert info["block_size"] == opts["block_size"] and info["tile"] == opts["tile"]
        assert info["launches_per_run"] > 0
        # one weights key per (graph, anchor class, window kind, delta)
        keys = set()
        for g, motif, delta, *_ in qs:
            mot = motif if isinstance(motif, tc.tc_motif) else tc.make_motif(motif)
            keys.add((id(g), tc.tc_motif_plan(mot)[1], mot.window, delta))
        assert info["weight_slots"] == len(keys)
        run_ms, samp_ms = b.timing()
        assert 0 < samp_ms <= run_ms
        b.destroy()


def test_batch_autotune_and_launch_count(tc, graphs):
    qs = _queries(tc, graphs)[:20]
    b = tc.Batch(qs)
    info = b.info()
    assert info["block_size"] in (128, 256, 512) and info["tile"] in (2048, 8192, 32768)
    assert info["use_graph"]
    before = tc.tc_kernel_launches()
    res = b.run()
    assert tc.tc_kernel_launches() - before == info["launches_per_run"]
    for q, r in zip(qs, res):
        _same(r, _alone(tc, q))
    b.destroy()


def test_batch_matches_oracle(tc, graphs):
    """Two queries on the 24-vertex dense graph against the oracle's sums."""
    g, cfg = graphs[0]
    og = oracle.build_csr(cfg["n"], cfg["src"], cfg["dst"], cfg["t"])
    qs = [(g, C4, 10_000, 100_000, 3, 7), (g, CHORD, 500, 70_000, 4, 1 << 33)]
    res = tc.Batch(qs, block_size=256, tile=2048).run()
    for (gq, edges, delta, k, seed, offset), r in zip(qs, res):
        plan = oracle.compile_motif(edges)
        opre = oracle.prefix_sum(oracle.path_weights(og, plan, delta)["w"])
        osums, _ = oracle.sample_run(og, plan, delta, opre, k, seed, offset)
        assert r["W"] == int(opre[-1])
        for key in ("sum_x", "sum_x2", "hits"):
            assert r[key] == osums[key], key


def test_batch_edge_cases(tc, graphs):
    g = graphs[0][0]
    empty = tc.Batch([])
    assert empty.run() == []
    empty.destroy()
    with pytest.raises(tc.TcError) as e:
        tc.Batch([(g, C4, 100, 10, 0, 0)], block_size=64, tile=2048)
    assert e.value.status == 1
    with pytest.raises(tc.TcError) as e:
        tc.Batch([(g, C4, 100, 10, 0, 0)], block_size=256, tile=1000)
    assert e.value.status == 1
    with pytest.raises(tc.TcError) as e:
        tc.Batch([(g, [(0, 1), (2, 3), (0, 1), (2, 3)], 100, 10, 0, 0)], block_size=256, tile=2048)
    assert e.value.status == 5
    with pytest.raises(tc.TcError) as e:
        tc.Batch([(g, C4, -1, 10, 0, 0)], block_size=256, tile=2048)
    assert e.value.status == 1
    # one query repeated: identical results, one weights slot
    qs = [(g, C4, 10_000, 80_000, 9, 0)] * 3
    res = tc.Batch(qs, block_size=256, tile=2048).run()
    _same(res[0], res[1])
    _same(res[1], res[2])


def test_chunked_sort_beyond_2_28_samples(tc, graphs):
    # above 2^28 samples the sample ids are put in key order chunk by chunk;
    # the sums must equal those of the two ranges run separately, single
    # call and batch alike
    g = graphs[2][0]
    chunk = 1 << 28
    k = chunk + 123_457
    mot = tc.make_motif(C4)
    w = tc.tc_path_weights(g, mot, 10_000)
    full = tc.tc_sample_estimate(g, mot, 10_000, w, k, 21, 5)
    a = tc.tc_sample_estimate(g, mot, 10_000, w, chunk, 21, 5)
    b = tc.tc_sample_estimate(g, mot, 10_000, w, k - chunk, 21, 5 + chunk)
    for key in ("sum_x", "sum_x2", "hits", "checked"):
        assert full[key] == a[key] + b[key], key
    r = tc.Batch([(g, C4, 10_000, k, 21, 5), (g, C4, 10_000, 70_000, 21, 5)], block_size=256, tile=32768).run()
    for key in ("sum_x", "sum_x2", "hits", "checked"):
        assert r[0][key] == full[key], key
