"""The C ABI library builds, loads without a GPU, and exports every function
that include/tc.h declares; host-only entry points behave as documented."""
import ctypes
import os
import re

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "tc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(tc_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libtc():
    from paper_2409_08975_gb300 import _build
    _build.build()
    from paper_2409_08975_gb300 import tc
    return tc.lib()


def test_header_declares_the_path(libtc):
    names = declared_functions()
    for required in ("tc_build_temporal_csr", "tc_path_weights", "tc_sample_estimate", "tc_last_error"):
        assert required in names
    for name in names:
        assert hasattr(libtc, name), name


def test_motif_plan_host_only(libtc):
    from paper_2409_08975_gb300 import tc
    import oracle
    from _graphs import path_motifs_all_classes
    # the library's motif compiler agrees with the oracle's on anchor and class
    zoo = path_motifs_all_classes() + [[(0, 1), (1, 2), (2, 3), (3, 0)], [(0, 1), (1, 2), (2, 3), (0, 3)],
                                       [(1, 2), (0, 1), (2, 3), (3, 0)], [(2, 3), (1, 2), (0, 1), (0, 3)],
                                       [(0, 1), (1, 2), (2, 3), (3, 2), (2, 1), (1, 0), (0, 1), (1, 2), (2, 3)],
                                       # 3-vertex motifs: wedge anchors at the base's source and head
                                       [(0, 1), (0, 2), (1, 2)], [(0, 1), (1, 2), (2, 0)], [(0, 1), (2, 1), (0, 2)],
                                       [(0, 1), (2, 0), (2, 1)], [(0, 1), (0, 2)],
                                       [(0, 1), (1, 0), (0, 1), (1, 2), (2, 1)]]
    for edges in zoo:
        anchor, cls = tc.tc_motif_plan(tc.make_motif(edges))
        p = oracle.compile_motif(edges)
        assert anchor == (p.e1, p.mid, p.e3)
        assert cls == (p.alpha1, p.alpha3, p.beta1, p.beta3)


@pytest.mark.parametrize("edges,status", [
    ([(0, 1)], 1),                               # too few edges
    ([(0, 1), (2, 3)], 1),                       # four labels need three edges
    ([(0, 1), (1, 1), (2, 3)], 1),               # self-loop
    ([(0, 1), (1, 0), (0, 1)], 1),               # only two labels
    ([(0, 1), (2, 3), (0, 1), (2, 3)], 5),       # no 3-path through edge 0
])
def test_motif_errors(libtc, edges, status):
    from paper_2409_08975_gb300 import tc
    with pytest.raises(tc.TcError) as e:
        tc.tc_motif_plan(tc.make_motif(edges))
    assert e.value.status == status
    assert libtc.tc_last_error()


def test_null_arguments_rejected(libtc):
    from paper_2409_08975_gb300 import tc
    out = ctypes.c_void_p()
    assert libtc.tc_build_temporal_csr(10, 5, None, None, None, None, ctypes.byref(out)) == 1
    assert libtc.tc_build_temporal_csr(0, 0, None, None, None, None, ctypes.byref(out)) == 1
    assert libtc.tc_graph_destroy(None) == 0
    m = tc.make_motif([(0, 1), (1, 2), (2, 3), (3, 0)])
    assert libtc.tc_path_weights(None, ctypes.byref(m), 5, None, None, None, None, None) == 1
    est = tc.tc_estimate()
    assert libtc.tc_sample_estimate(None, ctypes.byref(m), 5, None, None, 1, 0, 0, ctypes.byref(est), None) == 1


def test_estimate_from_sums_matches_the_oracle(libtc):
    """Alg. 5's final step through the ABI (host only) against the oracle's
    exact-rational form, including sums of squares above 2^64 and the
    degenerate k = 0, k = 1 and W = 0 cases."""
    import math
    import random
    from paper_2409_08975_gb300 import tc
    import oracle
    rng = random.Random(3)
    cases = [(0, 0, 0, 5), (7, 49, 1, 9), (0, 0, 10, 0), (3, 9, 2, 1 << 63)]
    for _ in range(200):
        k = rng.randrange(2, 1 << 40)
        sx = rng.randrange(0, 1 << 63)
        sx2 = rng.randrange(sx, 1 << 127)
        cases.append((sx, sx2, k, rng.randrange(1, 1 << 64)))
    for sx, sx2, k, W in cases:
        est, se = tc.tc_estimate_from_sums(sx, sx2, k, W)
        ref, rse = oracle.estimate(sx, sx2, k, W)
        assert est == ref, (sx, sx2, k, W)
        if math.isnan(rse):
            assert math.isnan(se)
        else:
            assert se == pytest.approx(rse, rel=1e-12, abs=0.0)


def test_mlp_kernel_selector_host_only(libtc):
    before = libtc.tc_mlp_kernel(-1)
    assert before in (0, 1)
    assert libtc.tc_mlp_kernel(7) == -1 and libtc.tc_mlp_kernel(-1) == before
    assert libtc.tc_mlp_kernel(1) == 1 and libtc.tc_mlp_kernel(0) == 0
    assert libtc.tc_mlp_kernel(before) == before
