"""Helpers shared by the tests: parsing the hand-built graph fixtures and
small random graphs.  No estimator arithmetic lives here."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def parse_motif(s):
    return [tuple(int(v) for v in e.split(">")) for e in s.split(",")]


def hand_graphs():
    """Yield (name, edges(list of (a,b)), delta, count, src, dst, t)."""
    path = os.path.join(GOLDEN, "hand_graphs.txt")
    cur = None
    rows = []

    def flush():
        if cur is not None:
            a = np.array(rows, dtype=np.int64).reshape(-1, 3)
            return (cur[0], cur[1], cur[2], cur[3], a[:, 0].astype(np.int32),
                    a[:, 1].astype(np.int32), a[:, 2].astype(np.int64))
        return None

    out = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if line.startswith("#"):
                continue
            if not line:
                g = flush()
                if g:
                    out.append(g)
                cur, rows = None, []
                continue
            tok = line.split()
            if tok[0] == "graph":
                cur = (tok[1], parse_motif(tok[3]), int(tok[5]), int(tok[7]))
            else:
                rows.append([int(x) for x in tok])
    g = flush()
    if g:
        out.append(g)
    return out


def small_random_graph(seed, n, m, tmax, dup_frac=0.2):
    """Tiny multigraph without self-loops, some repeated pairs and tied times."""
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n, m)
    dst = rng.integers(0, n, m)
    keep = src != dst
    src, dst = src[keep], dst[keep]
    k = int(len(src) * dup_frac)
    if k and len(src):
        pick = rng.integers(0, len(src), k)
        src = np.concatenate([src, src[pick]])
        dst = np.concatenate([dst, dst[pick]])
    t = rng.integers(0, tmax, len(src))
    return src.astype(np.int32), dst.astype(np.int32), t.astype(np.int64)


def path_motifs_all_classes():
    """Sixteen 3-edge path motifs a-b-c-d whose anchor (the whole motif)
    covers each class <alpha1, alpha3, beta1, beta3> once (Def. 5)."""
    out = []
    # rank arrangements (rank e1, rank mid, rank e3)
    arrangements = [(0, 1, 2), (2, 0, 1), (1, 2, 0), (2, 1, 0)]
    for e1_in in (True, False):          # e1 = a->b (into b) or b->a
        for e3_out in (True, False):     # e3 = c->d (out of c) or d->c
            for r1, rm, r3 in arrangements:
                e = [None] * 3
                e[r1] = (0, 1) if e1_in else (1, 0)
                e[rm] = (1, 2)
                e[r3] = (2, 3) if e3_out else (3, 2)
                out.append(e)
    return out
