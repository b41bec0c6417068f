"""Pins of the oracle's wedge sampling for 3-vertex motifs (wedge anchor:
base = motif edge 0, second edge later in time at the shared vertex).  The
wedge weights equal a literal count of second edges per base edge, the sum
of CheckMotif over all wedges equals the literal Def. 2 count (brute force
and backtracking), and the estimator is unbiased over seeds."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from _graphs import small_random_graph

FF = [(0, 1), (0, 2), (1, 2)]                      # a->b, a->c, b->c: <+,>> at the base's source
CYC = [(0, 1), (1, 2), (2, 0)]                     # cyclic triangle: second edge leaves the base's head
IN_DST = [(0, 1), (2, 1), (0, 2)]                  # second edge enters the base's head
IN_SRC = [(0, 1), (2, 0), (2, 1)]                  # second edge enters the base's tail
WEDGE2 = [(0, 1), (0, 2)]                          # the wedge alone
MULTI3 = [(0, 1), (0, 2), (0, 1), (1, 2), (0, 2)]  # three lists after the second edge
GAP0 = [(0, 1), (1, 0), (0, 1), (1, 2), (2, 1)]    # second edge is rank 3: two lists before it
ZOO = [FF, CYC, IN_DST, IN_SRC, WEDGE2, MULTI3, GAP0]


def test_wedge_anchor_rule():
    p = oracle.compile_motif(FF)
    assert (p.kind, p.e1, p.mid, p.e3, p.alpha1, p.beta1, p.labels) == (1, 1, 0, -1, +1, +1, (2, 0, 1, -1))
    p = oracle.compile_motif(CYC)
    assert (p.kind, p.e1, p.mid, p.e3, p.alpha3, p.beta3, p.labels) == (2, -1, 0, 1, +1, +1, (-1, 0, 1, 2))
    p = oracle.compile_motif(IN_DST)
    assert (p.kind, p.e3, p.alpha3) == (2, 1, -1)
    p = oracle.compile_motif(IN_SRC)
    assert (p.kind, p.e1, p.alpha1) == (1, 1, -1)
    p = oracle.compile_motif(GAP0)
    assert (p.kind, p.e3, p.gaps) == (2, 3, [[1, 2], [4]])
    with pytest.raises(ValueError):
        oracle.compile_motif([(0, 1), (1, 0), (0, 1)])  # two labels
    with pytest.raises(ValueError):
        oracle.compile_motif([(0, 1)])


@pytest.mark.parametrize("closed", [False, True])
def test_wedge_weights_equal_literal_count(closed):
    src, dst, t = small_random_graph(11, 7, 80, 40, dup_frac=0.3)
    g = oracle.build_csr(7, src, dst, t)
    for edges in (FF, CYC, IN_DST, IN_SRC):
        plan = oracle.compile_motif(edges, closed=closed)
        for delta in (0, 3, 12, 100):
            pw = oracle.path_weights(g, plan, delta)
            brute = np.array(oracle.brute_force_paths(src, dst, t, plan, delta), dtype=np.uint64)
            assert (pw["w"] == brute[g.out_perm]).all(), (edges, delta)
            # the unused side is the single dummy position
            side_d = pw["d3"] if plan.kind == 1 else pw["d1"]
            assert (side_d == 1).all()


def test_wedge_weight_by_hand():
    # base (0,1,10); out-edges of 0 at 5, 10, 11, 20, 21; delta 10:
    # strict (10, 20] holds 11 and 20; closed [10, 20] adds the base itself
    src = np.array([0, 0, 0, 0, 0, 0], np.int32)
    dst = np.array([1, 2, 3, 2, 3, 1], np.int32)
    t = np.array([10, 5, 11, 20, 21, 10], np.int64)
    g = oracle.build_csr(4, src, dst, t)
    for closed, want in ((False, 2), (True, 4)):
        pw = oracle.path_weights(g, oracle.compile_motif(FF, closed=closed), 10)
        i = int(np.nonzero(g.out_perm == 0)[0][0])
        assert int(pw["w"][i]) == want


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_wedge_path_sum_equals_brute_force(seed):
    for edges in ZOO:
        # the literal count enumerates all edge tuples: fewer edges for longer motifs
        src, dst, t = small_random_graph(300 + seed, 5, 40 if len(edges) <= 3 else 22, 30, dup_frac=0.4)
        g = oracle.build_csr(5, src, dst, t)
        for delta in (0, 4, 15, 40):
            C = oracle.brute_force_count(src, dst, t, edges, delta)
            assert oracle.exact_count(g, edges, delta) == C
            for closed in (False, True):
                plan = oracle.compile_motif(edges, closed=closed)
                ps = oracle.path_sum(g, plan, delta)
                assert ps["C"] == C, (edges, delta, closed)
                W = int(oracle.prefix_sum(oracle.path_weights(g, plan, delta)["w"])[-1])
                assert ps["paths"] == W


def test_every_wedge_anchor_gives_the_count():
    src, dst, t = small_random_graph(46, 4, 26, 30, dup_frac=0.4)
    g = oracle.build_csr(4, src, dst, t)
    C = oracle.brute_force_count(src, dst, t, MULTI3, 20)
    assert C > 0
    js = oracle.core.wedge_candidates(MULTI3)
    assert js == [1, 3, 4]
    kinds = []
    for j in js:  # edges 1 and 4 share the base's source, edge 3 its head
        anchor = (j, 0, -1) if j != 3 else (-1, 0, j)
        plan = oracle.compile_motif(MULTI3, anchor=anchor)
        assert (plan.e1, plan.mid, plan.e3) == anchor
        kinds.append(plan.kind)
        assert oracle.path_sum(g, plan, 20)["C"] == C
    assert kinds == [1, 2, 1]


def test_wedge_triangle_by_hand():
    # edges (0,1,1), (0,2,2), (1,2,3), (1,0,4), (2,0,5), (0,1,50); feed-forward
    # a->b, a->c, b->c: {(0,1,1), (0,2,2), (1,2,3)} and {(1,2,3), (1,0,4), (2,0,5)}
    src = np.array([0, 0, 1, 1, 2, 0], np.int32)
    dst = np.array([1, 2, 2, 0, 0, 1], np.int32)
    t = np.array([1, 2, 3, 4, 5, 50], np.int64)
    g = oracle.build_csr(3, src, dst, t)
    assert oracle.path_sum(g, oracle.compile_motif(FF), 10)["C"] == 2
    assert oracle.path_sum(g, oracle.compile_motif(FF), 1)["C"] == 0
    assert oracle.path_sum(g, oracle.compile_motif(FF), 2)["C"] == 2
    # cyclic a->b, b->c, c->a: (0,1,1), (1,2,3), (2,0,5) is one; so is
    # (1,2,3), (2,0,5), (0,1,50) only when delta >= 47
    assert oracle.path_sum(g, oracle.compile_motif(CYC), 10)["C"] == 1
    assert oracle.path_sum(g, oracle.compile_motif(CYC), 47)["C"] == 2
    assert oracle.brute_force_count(src, dst, t, CYC, 47) == 2


def test_wedge_unbiased_over_seeds():
    src, dst, t = small_random_graph(78, 6, 80, 50, dup_frac=0.3)
    g = oracle.build_csr(6, src, dst, t)
    delta = 20
    for edges in (FF, CYC):
        plan = oracle.compile_motif(edges)
        pre = oracle.prefix_sum(oracle.path_weights(g, plan, delta)["w"])
        W = int(pre[-1])
        ps = oracle.path_sum(g, plan, delta)
        C = ps["C"]
        assert C == oracle.brute_force_count(src, dst, t, edges, delta) and C > 0
        var_x = Fraction(ps["sum_x2"], W) - Fraction(C, W) ** 2
        k, seeds = 100, 600
        ests = []
        for seed in range(seeds):
            sums, _ = oracle.sample_run(g, plan, delta, pre, k, seed)
            ests.append(oracle.estimate(sums["sum_x"], sums["sum_x2"], k, W)[0])
        sd_mean = W * math.sqrt(float(var_x) / k / seeds)
        assert abs(np.mean(ests) - C) <= 2.576 * sd_mean, (edges, np.mean(ests), C, sd_mean)


def test_wedge_trace_positions_in_window():
    src, dst, t = small_random_graph(5, 6, 100, 40, dup_frac=0.3)
    g = oracle.build_csr(6, src, dst, t)
    for edges in (FF, CYC):
        plan = oracle.compile_motif(edges)
        pw = oracle.path_weights(g, plan, 15)
        pre = oracle.prefix_sum(pw["w"])
        sums, tr = oracle.sample_run(g, plan, 15, pre, 3000, 9, trace=True)
        for i2, p1, p3, X in tr.astype(np.int64).tolist():
            if plan.kind == 1:
                assert pw["lo1"][i2] <= p1 < pw["lo1"][i2] + pw["d1"][i2] and p3 == 0
            else:
                assert pw["lo3"][i2] <= p3 < pw["lo3"][i2] + pw["d3"][i2] and p1 == 0
        assert sums["sum_x"] == int(tr[:, 3].sum())
