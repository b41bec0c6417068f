"""The seeded synthetic inputs have the shapes their recipes state (the
stand-ins for the paper's datasets): sizes, id and time ranges, no
self-loops, the share of repeated pairs, the degree cap, Zipf
multiplicities, the daily modulation of burst starts, and determinism in the
seed."""
import numpy as np
import pytest

from paper_2409_08975_gb300 import synth


def _pair_counts(src, dst):
    key = src.astype(np.int64) * (1 << 32) + dst.astype(np.int64)
    _, counts = np.unique(key, return_counts=True)
    return counts


def test_tiny_recipe():
    g = synth.tiny()
    src, dst, t = g["src"], g["dst"], g["t"]
    assert g["n"] == 2000 and len(src) == len(dst) == len(t) == 20_000
    assert src.min() >= 0 and max(src.max(), dst.max()) < 2000 and (src != dst).all()
    assert t.min() >= 0 and t.max() < 1_000_000
    counts = _pair_counts(src, dst)
    # a pair repeats with probability 0.10, 2-5 times (the last pair may be trimmed)
    assert 0.08 < (counts > 1).mean() < 0.12
    assert counts.max() <= 5
    assert g["motif"] == synth.C4 and g["delta"] == 10_000 and g["k"] == 100_000


def test_dense_tiny_recipe():
    for bursty in (False, True):
        g = synth.dense_tiny(bursty=bursty)
        src, dst, t = g["src"], g["dst"], g["t"]
        assert len(src) == 20_000 and (src != dst).all() and max(src.max(), dst.max()) < 24
        assert t.min() >= 0 and t.max() < 1_000_000


@pytest.mark.parametrize("zipf", [None, 1.8])
def test_chung_lu_recipe(zipf):
    n, m, max_deg = 20_000, 400_000, 2_000
    g = synth.chung_lu(n, m, max_deg=max_deg, seed=5, daily=zipf is not None, zipf_repeats=zipf)
    src, dst, t = g["src"], g["dst"], g["t"]
    assert len(src) == len(dst) == len(t) == m
    assert (src != dst).all() and src.min() >= 0 and max(src.max(), dst.max()) < n
    assert t.min() >= 0 and t.max() < 100_000_000
    counts = _pair_counts(src, dst)
    repeated_edges = 1.0 - len(counts) / m       # edges beyond the first of their pair
    out_deg = np.bincount(src, minlength=n)
    if zipf is None:
        assert 0.29 < repeated_edges < 0.45       # 30% repeats plus pairs that bursts join twice
        assert 0.5 * max_deg < out_deg.max() < 2.0 * max_deg
    else:
        # Zipf(1.8) multiplicity per burst edge (capped at ZIPF_CAP; a pair
        # that several burst edges join adds their multiplicities): heavy tail
        assert counts.max() > 100
        assert (counts == 1).mean() > 0.5
        assert 0.3 * max_deg < out_deg.max() < 3.0 * max_deg
    # power law: the top 1% of vertices hold far more than 1% of the edges
    top = np.sort(out_deg)[::-1][: n // 100].sum() / m
    assert top > 0.1


def test_daily_modulation_of_burst_starts():
    # burst starts are accepted with probability (1 + 0.5 sin(2 pi t / 86400)) / 1.5:
    # the half-day where the sine is positive holds about (1 + 1/pi) / 2 of them
    g = synth.chung_lu(50_000, 500_000, max_deg=5_000, seed=9, daily=True, zipf_repeats=1.8,
                       mean_burst_edges=1)
    phase = (g["t"] % 86_400) / 86_400.0
    share = (phase < 0.5).mean()
    assert abs(share - (1 + 1 / np.pi) / 2) < 0.03, share


def test_generators_are_deterministic_in_the_seed():
    a, b = synth.scaled_mid(5000, 50_000, seed=3), synth.scaled_mid(5000, 50_000, seed=3)
    c = synth.scaled_mid(5000, 50_000, seed=4)
    for key in ("src", "dst", "t"):
        assert np.array_equal(a[key], b[key])
    assert not np.array_equal(a["t"], c["t"])


def test_batch_queries_shape():
    cfg = synth.batch(seed=3, n_small=4, big_m=200_000, k_range=(1e3, 1e4))
    assert len(cfg["graphs"]) == 5
    big = [q for q in cfg["queries"] if q[0] == 0]
    assert len(big) == 24 * len(synth.BATCH_DELTAS)        # every rank order of the 4-cycle at every delta
    orders = {tuple(q[1]) for q in big}
    assert len(orders) == 24 and all(sorted(o) == sorted(synth.C4) for o in orders)
    assert all(1e3 <= q[3] <= 1e4 for q in cfg["queries"])
    assert cfg["k"] == sum(q[3] for q in cfg["queries"])


def test_time_slices_partition_the_graph():
    """Contiguous time slices of about 1 / parts of the edges each: every edge
    falls in exactly one slice, inside its time bounds, and renumbering keeps
    the vertex order."""
    g = synth.scaled_mid(20_000, 300_000, seed=5)
    parts = 10
    total = 0
    seen = np.zeros(len(g["t"]), np.int64)
    for j in range(parts):
        s = synth.time_slice(g, j, parts)
        m = len(s["src"])
        total += m
        assert abs(m - len(g["t"]) / parts) <= 0.05 * len(g["t"]) / parts
        assert (s["t"] >= s["t_lo"]).all()
        if s["t_hi"] is not None:
            assert (s["t"] < s["t_hi"]).all()
        sel = np.flatnonzero((g["t"] >= s["t_lo"]) & ((g["t"] < s["t_hi"]) if s["t_hi"] is not None else True))
        seen[sel] += 1
        assert np.array_equal(s["t"], g["t"][sel])
        ids = np.unique(np.concatenate([g["src"][sel], g["dst"][sel]]))
        assert np.array_equal(ids[s["src"]], g["src"][sel]) and np.array_equal(ids[s["dst"]], g["dst"][sel])
        assert s["n"] == len(ids)
    assert total == len(g["t"]) and (seen == 1).all()
