"""Oracle implementation (test infrastructure; see the package docstring).

The heavy loops live in ``tc_oracle.c`` (plain serial C); this module holds the
motif compiler, the literal brute-force counter and the host arithmetic of the
estimate, and wraps the C functions with numpy arrays.
"""
import ctypes
import itertools
import math

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        _declare(_lib)
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _declare(L):
    vp, i64, u64, i32, u32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32, ctypes.c_uint32
    L.or_build_csr.argtypes = [i64, i64, ctypes.c_int] + [vp] * 3 + [vp] * 9 + [vp]
    L.or_build_csr.restype = ctypes.c_int
    L.or_path_weights.argtypes = [i64, i64] + [vp] * 7 + [vp, i64] + [vp] * 5
    L.or_path_weights.restype = ctypes.c_int
    L.or_prefix.argtypes = [i64, vp, vp]
    L.or_prefix.restype = ctypes.c_int
    L.or_philox4x32_10.argtypes = [vp, vp, vp]
    L.or_philox4x32_10.restype = None
    L.or_bounded.argtypes = [u64, u64, u32, u64, ctypes.POINTER(u64)]
    L.or_bounded.restype = ctypes.c_int
    L.or_bounded_hi.argtypes = [u64, u64, u32, u64, ctypes.POINTER(u64)]
    L.or_bounded_hi.restype = ctypes.c_int
    L.or_list_count.argtypes = [ctypes.c_int, vp, vp, ctypes.POINTER(ctypes.c_int)]
    L.or_list_count.restype = u64
    L.or_sample_run.argtypes = [i64, i64] + [vp] * 3 + [vp] * 8 + [vp, i64, vp, u64, u64, u64, vp, vp]
    L.or_sample_run.restype = ctypes.c_int
    L.or_path_sum.argtypes = [i64, i64] + [vp] * 3 + [vp] * 8 + [vp, i64, vp]
    L.or_path_sum.restype = ctypes.c_int
    L.or_exact_count.argtypes = [i64, i64] + [vp] * 3 + [vp] * 8 + [i32, vp, vp, i64, ctypes.POINTER(u64)]
    L.or_exact_count.restype = ctypes.c_int
    L.or_set_threads.argtypes = [ctypes.c_int]
    L.or_set_threads.restype = ctypes.c_int


def set_threads(n):
    """Threads of the oracle's parallel loops (weights, sampler, path sum,
    backtracking count); 1 (the default) runs them serially.  Results do not
    depend on it.  Returns the number in use (1 without OpenMP)."""
    return int(lib().or_set_threads(int(n)))


class OracleError(RuntimeError):
    def __init__(self, status, what):
        super().__init__("%s failed with status %d" % (what, status))
        self.status = status


STATUS_OVERFLOW = 3
STATUS_RNG_EXHAUSTED = 6

# ---------------------------------------------------------------------------
# Motif compiler (Alg. 5: choose an anchor 3-path that contains the edge of
# smallest time order; Def. 5: its class <alpha1, alpha3, beta1, beta3>).


class Plan:
    """Anchor choice and class of a motif.  Edge i of the motif has rank i."""

    def __init__(self, edges, e1, mid, e3, labels, closed):
        self.edges = [tuple(e) for e in edges]
        self.r = len(edges)
        self.e1, self.mid, self.e3 = e1, mid, e3
        U, V = self.edges[mid]
        a, c = self.edges[e1], self.edges[e3]
        # alpha: '-' (in-list) when the end edge points into the middle's
        # endpoint, '+' (out-list) when it leaves it (Def. 5)
        self.alpha1 = -1 if a[1] == U else +1
        self.alpha3 = +1 if c[0] == V else -1
        # beta: '<' when the end edge precedes the middle edge in time order
        self.beta1 = -1 if e1 < mid else +1
        self.beta3 = -1 if e3 < mid else +1
        self.labels = labels  # motif labels of (u', u, v, v')
        self.closed = int(bool(closed))
        self.kind = 0
        ranks = sorted((e1, mid, e3))
        self.gaps = [
            [f for f in range(ranks[0] + 1, ranks[1])],
            [f for f in range(ranks[1] + 1, ranks[2])],
            [f for f in range(ranks[2] + 1, self.r)],
        ]

    @property
    def cls(self):
        s = {-1: "-", 1: "+", 0: "0"}
        b = {-1: "<", 1: ">", 0: "0"}
        return (s[self.alpha1], s[self.alpha3], b[self.beta1], b[self.beta3])

    def array(self):
        a = np.zeros(46, dtype=np.int32)
        a[0] = self.r
        for i, (x, y) in enumerate(self.edges):
            a[1 + i] = x
            a[17 + i] = y
        a[33:36] = (self.e1, self.mid, self.e3)
        a[36:40] = (self.alpha1, self.alpha3, self.beta1, self.beta3)
        a[40] = self.closed
        a[41:45] = self.labels
        a[45] = self.kind
        return a


class WedgePlan(Plan):
    """Anchor of a 3-vertex motif (wedge sampling, Sec. "Brief Description of
    Wedge Sampling"): the base is motif edge 0, the edge sampled in
    proportion to its weight; the second edge is motif edge j, which shares
    exactly one vertex s with the base and is later in time order, so it lies
    in s's out-list (alpha = +1, the paper's <+,>> wedge when s is the base's
    source) or in-list (alpha = -1) within (t, t + delta] of the base.  The
    weight of a base edge is the size of that window.  kind 1: s is the
    base's source (second edge stored as e1); kind 2: its destination (e3)."""

    def __init__(self, edges, j, closed):
        self.edges = [tuple(e) for e in edges]
        self.r = len(edges)
        A, B = self.edges[0]
        x, y = self.edges[j]
        shared = A if A in (x, y) else B
        third = y if x == shared else x
        alpha = +1 if x == shared else -1
        self.kind = 1 if shared == A else 2
        self.mid = 0
        if self.kind == 1:
            self.e1, self.e3 = j, -1
            self.alpha1, self.beta1, self.alpha3, self.beta3 = alpha, +1, 0, 0
            self.labels = (third, A, B, -1)
        else:
            self.e1, self.e3 = -1, j
            self.alpha1, self.beta1, self.alpha3, self.beta3 = 0, 0, alpha, +1
            self.labels = (-1, A, B, third)
        self.closed = int(bool(closed))
        self.gaps = [[f for f in range(1, j)], [f for f in range(j + 1, self.r)]]


def anchor_candidates(edges):
    """All (sorted ranks, e1, mid, e3, labels) 3-paths over the four vertices
    that contain motif edge 0 (the edge of smallest time order)."""
    out = []
    r = len(edges)
    for trip in itertools.combinations(range(r), 3):
        if 0 not in trip:
            continue
        for mid in trip:
            U, V = edges[mid]
            rest = [x for x in trip if x != mid]
            for e1, e3 in (rest, rest[::-1]):
                a, c = edges[e1], edges[e3]
                if U not in a or V in a or V not in c or U in c:
                    continue
                Up = a[0] if a[1] == U else a[1]
                Vp = c[0] if c[1] == V else c[1]
                if len({Up, U, V, Vp}) != 4:
                    continue
                out.append((tuple(sorted(trip)), e1, mid, e3, (Up, U, V, Vp)))
    return out


def wedge_candidates(edges):
    """Motif edges j > 0 that share exactly one vertex with edge 0."""
    return [j for j in range(1, len(edges)) if len(set(edges[0]) & set(edges[j])) == 1]


def compile_motif(edges, anchor=None, closed=False):
    """Anchor rule: among the candidate 3-paths containing edge 0, take the one
    whose sorted triple of ranks is lexicographically smallest (Alg. 5 leaves
    the choice open; any choice is unbiased by Claim 2).  ``anchor`` may force
    (e1, mid, e3).  A motif on three vertex labels gets a wedge anchor: edge 0
    as the base and the smallest j whose edge shares one vertex with it
    (forced as (j, 0, -1) or (-1, 0, j))."""
    edges = [tuple(int(v) for v in e) for e in edges]
    labs = set()
    for x, y in edges:
        if x == y or not (0 <= x < 4 and 0 <= y < 4):
            raise ValueError("motif edges join two distinct labels in 0..3")
        labs |= {x, y}
    if len(labs) == 3:
        if not 2 <= len(edges) <= 16:
            raise ValueError("a 3-vertex motif needs 2..16 edges")
        js = wedge_candidates(edges)
        if anchor is not None:
            js = [j for j in js if tuple(anchor) in ((j, 0, -1), (-1, 0, j))]
        if not js:
            raise ValueError("no wedge anchor containing edge 0")
        return WedgePlan(edges, js[0], closed)
    if not 3 <= len(edges) <= 16:
        raise ValueError("motif needs 3..16 edges")
    if labs != {0, 1, 2, 3}:
        raise ValueError("motif must use three or all four vertex labels")
    cands = anchor_candidates(edges)
    if anchor is not None:
        cands = [c for c in cands if (c[1], c[2], c[3]) == tuple(anchor)]
    if not cands:
        raise ValueError("no anchor 3-path containing edge 0")
    best = min(cands, key=lambda c: c[0])
    _, e1, mid, e3, labels = best
    return Plan(edges, e1, mid, e3, labels, closed)


# ---------------------------------------------------------------------------
# Graph lists


class Graph:
    """Time-sorted out-, in- and pair-lists (Sec. III, Sec. III-B) built by
    comparison sorts with the full keys: C qsort by default, or numpy's
    lexsort on the same keys (sort="lexsort") for large graphs."""

    def __init__(self, n, src, dst, t, sort="qsort"):
        self.n = int(n)
        self.src = np.ascontiguousarray(src, dtype=np.int32)
        self.dst = np.ascontiguousarray(dst, dtype=np.int32)
        self.t = np.ascontiguousarray(t, dtype=np.int64)
        m = self.m = len(self.src)
        self.out_perm = np.empty(m, np.int64)
        self.out_off = np.empty(n + 1, np.int64)
        self.in_perm = np.empty(m, np.int64)
        self.in_off = np.empty(n + 1, np.int64)
        self.in_eid = np.empty(m, np.int64)
        self.pair_perm = np.empty(m, np.int64)
        self.pair_off = np.empty(n + 1, np.int64)
        self.pair_dst = np.empty(max(m, 1), np.int32)
        self.pair_eoff = np.empty(m + 1, np.int64)
        presorted = 0
        if sort == "lexsort":
            idx = np.arange(m, dtype=np.int64)
            self.out_perm[:] = np.lexsort((idx, self.t, self.src))
            self.in_perm[:] = np.lexsort((idx, self.t, self.dst))
            self.pair_perm[:] = np.lexsort((idx, self.t, self.dst, self.src))
            presorted = 1
        P = ctypes.c_int64(0)
        st = lib().or_build_csr(n, m, presorted, _p(self.src), _p(self.dst), _p(self.t), _p(self.out_perm),
                                _p(self.out_off), _p(self.in_perm), _p(self.in_off), _p(self.in_eid),
                                _p(self.pair_perm), _p(self.pair_off), _p(self.pair_dst),
                                _p(self.pair_eoff), ctypes.byref(P))
        if st:
            raise OracleError(st, "build_csr")
        self.P = P.value
        self.pair_dst = self.pair_dst[: self.P]
        self.pair_eoff = self.pair_eoff[: self.P + 1].copy()

    def _ptrs(self):
        return [_p(self.src), _p(self.dst), _p(self.t), _p(self.out_perm), _p(self.out_off),
                _p(self.in_perm), _p(self.in_off), _p(self.pair_perm), _p(self.pair_off),
                _p(self.pair_dst if self.P else np.zeros(1, np.int32)), _p(self.pair_eoff)]


def build_csr(n, src, dst, t, sort="qsort"):
    return Graph(n, src, dst, t, sort)


def path_weights(g, plan, delta):
    """Claim 1 / Alg. 1: per canonical edge, w = d1 * d3 with the list
    positions of both windows.  Returns dict of arrays."""
    m = g.m
    w = np.empty(m, np.uint64)
    lo1, d1, lo3, d3 = (np.empty(m, np.int64) for _ in range(4))
    st = lib().or_path_weights(g.n, m, _p(g.src), _p(g.dst), _p(g.t), _p(g.out_perm), _p(g.out_off),
                               _p(g.in_perm), _p(g.in_off), _p(plan.array()), int(delta), _p(w),
                               _p(lo1), _p(d1), _p(lo3), _p(d3))
    if st:
        raise OracleError(st, "path_weights")
    return {"w": w, "lo1": lo1, "d1": d1, "lo3": lo3, "d3": d3}


def prefix_sum(w):
    """prefix[0] = 0, prefix[i+1] = prefix[i] + w[i]; W = prefix[m] (Alg. 1)."""
    w = np.ascontiguousarray(w, dtype=np.uint64)
    pre = np.empty(len(w) + 1, np.uint64)
    st = lib().or_prefix(len(w), _p(w), _p(pre))
    if st:
        raise OracleError(st, "prefix")
    return pre


def philox4x32_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    o = np.empty(4, np.uint32)
    lib().or_philox4x32_10(_p(c), _p(k), _p(o))
    return [int(x) for x in o]


def bounded(seed, s, draw, rng, upper=False):
    """Lemire's bounded draw in [0, rng) from block (s, draw, attempt): x from
    words 0-1, or words 2-3 when upper."""
    r = ctypes.c_uint64(0)
    st = (lib().or_bounded_hi if upper else lib().or_bounded)(seed, s, draw, rng, ctypes.byref(r))
    if st:
        raise OracleError(st, "bounded")
    return r.value


def list_count(lists):
    """ListCount (Alg. 4): number of tuples, one element per list, with
    strictly increasing times (Def. 2 needs strict order)."""
    arrs = [np.ascontiguousarray(x, dtype=np.int64) for x in lists]
    ptrs = (ctypes.c_void_p * max(len(arrs), 1))(*[a.ctypes.data for a in arrs])
    lens = np.array([len(a) for a in arrs] or [0], dtype=np.int64)
    ovf = ctypes.c_int(0)
    c = lib().or_list_count(len(arrs), ctypes.cast(ptrs, ctypes.c_void_p), _p(lens), ctypes.byref(ovf))
    if ovf.value:
        raise OracleError(STATUS_OVERFLOW, "list_count")
    return int(c)


def sample_run(g, plan, delta, prefix, k, seed, offset=0, trace=False):
    """Alg. 5's loop for sample ids offset..offset+k-1.  Returns (sums, trace)
    with sums = dict(sum_x, sum_x2, hits, k) and trace an array (k,4) of
    (canonical middle edge, e1 list position, e3 list position, X)."""
    prefix = np.ascontiguousarray(prefix, dtype=np.uint64)
    tr = np.empty((k, 4), np.uint64) if trace else None
    sums = np.zeros(5, np.uint64)
    st = lib().or_sample_run(g.n, g.m, *g._ptrs(), _p(plan.array()), int(delta), _p(prefix),
                             int(k), int(seed), int(offset), _p(tr) if trace else None, _p(sums))
    if st:
        raise OracleError(st, "sample_run")
    out = {"sum_x": int(sums[0]), "sum_x2": int(sums[1]) | (int(sums[2]) << 64),
           "hits": int(sums[3]), "k": int(sums[4])}
    return out, tr


def path_sum(g, plan, delta):
    """Proof of Claim 2: sum over all class paths of CheckMotif = C.  Returns
    dict(C, sum_x2, paths)."""
    out = np.zeros(4, np.uint64)
    st = lib().or_path_sum(g.n, g.m, *g._ptrs(), _p(plan.array()), int(delta), _p(out))
    if st:
        raise OracleError(st, "path_sum")
    return {"C": int(out[0]), "sum_x2": int(out[1]) | (int(out[2]) << 64), "paths": int(out[3])}


def exact_count(g, edges, delta):
    """Def. 2 by chronological backtracking over the motif's edges."""
    ms = np.array([e[0] for e in edges], np.int32)
    md = np.array([e[1] for e in edges], np.int32)
    c = ctypes.c_uint64(0)
    st = lib().or_exact_count(g.n, g.m, *g._ptrs(), len(edges), _p(ms), _p(md), int(delta), ctypes.byref(c))
    if st:
        raise OracleError(st, "exact_count")
    return c.value


def brute_force_count(src, dst, t, edges, delta):
    """Literal Def. 2 (tiny graphs only): count edge tuples (g_0..g_{r-1}) with
    strictly increasing times, span <= delta and a consistent one-to-one map
    phi from motif labels to graph vertices.  With a total time order the
    i-th motif edge must map to the i-th earliest edge of the tuple."""
    m, r = len(src), len(edges)
    order = sorted(range(m), key=lambda i: (int(t[i]), i))
    count = 0
    for combo in itertools.combinations(order, r):
        times = [int(t[e]) for e in combo]
        if any(times[i] >= times[i + 1] for i in range(r - 1)):
            continue
        if times[-1] - times[0] > delta:
            continue
        phi = {}
        ok = True
        for (x, y), e in zip(edges, combo):
            for lab, vert in ((x, int(src[e])), (y, int(dst[e]))):
                if phi.setdefault(lab, vert) != vert:
                    ok = False
        if ok and len(set(phi.values())) == len(phi):
            count += 1
    return count


def brute_force_paths(src, dst, t, plan, delta):
    """Literal Def. 4/5: all (e1, e2, e3) edge triples of the anchor's class,
    per middle edge (input index); for a wedge anchor, all second edges per
    base edge.  Tiny graphs only."""
    m = len(src)
    per_mid = [0] * m
    for e2 in range(m):
        u, v, tm = int(src[e2]), int(dst[e2]), int(t[e2])
        # a wedge's unused end (alpha = 0) counts as one position
        c1 = 1 if plan.alpha1 == 0 else 0
        c3 = 1 if plan.alpha3 == 0 else 0
        for e in range(m):
            te = int(t[e])
            for alpha, beta, x, which in ((plan.alpha1, plan.beta1, u, 1), (plan.alpha3, plan.beta3, v, 3)):
                if alpha == 0:
                    continue
                inc = (int(dst[e]) == x) if alpha < 0 else (int(src[e]) == x)
                if not inc:
                    continue
                if beta < 0:
                    ok = (tm - delta <= te < tm) if not plan.closed else (tm - delta <= te <= tm)
                else:
                    ok = (tm < te <= tm + delta) if not plan.closed else (tm <= te <= tm + delta)
                if ok:
                    if which == 1:
                        c1 += 1
                    else:
                        c3 += 1
        per_mid[e2] = c1 * c3
    return per_mid


# ---------------------------------------------------------------------------
# Estimate (Alg. 5): C_hat = (cnt / k) * W, formed from exact integers.


def estimate(sum_x, sum_x2, k, W):
    """C_hat = sum_x * W / k by exact integer division, q + r/k in FP64; the
    standard error W * sqrt(s^2 / k) with the unbiased sample variance
    s^2 = (sum_x2 - sum_x^2 / k) / (k - 1), in FP64."""
    if k == 0 or W == 0:
        return 0.0, 0.0
    q, r = divmod(int(sum_x) * int(W), int(k))
    c_hat = float(q) + float(r) / float(k)
    if k < 2:
        return c_hat, float("nan")
    sx, sx2, kf = float(sum_x), float(sum_x2), float(k)
    s2 = (sx2 - sx * sx / kf) / (kf - 1.0)
    if s2 < 0.0:
        s2 = 0.0
    return c_hat, float(W) * math.sqrt(s2 / kf)
