"""Oracle of the learned proposal (test infrastructure).

The paper has no learned part; what it fixes is the estimator (Alg. 5) and
its unbiasedness (Claim 2), which holds for any proposal q_e = w_e * h_e with
integer h_e >= 1: the path P with middle edge e is drawn with probability
(w_e h_e / Q)(1 / w_e) = h_e / Q, so Y = X Q / h_e has E[Y] = C, where
Q = sum_e w_e h_e.  Here:
  * ``edge_features``   the 12 per-edge counts (plain definitions)
  * ``sample_features`` four per-edge statistics of the plain sampler's
    outcomes (columns 12..15)
  * ``bf16`` / ``features_bf16``   log1p then bf16 rounding (to nearest even)
  * ``mlp_forward`` / ``mlp_backward``   16 -> 64 -> 64 -> 1 network in FP64
    on bf16 weights and inputs, activations rounded to bf16 between layers
  * ``proposal_h``      h = max(1, floor(S (eps + g) + 1/2))
  * ``sample_run_q``    Alg. 2 / 3 / 5 with the proposal, per-h exact bins
  * ``estimate_q``      C_hat = Q / k * sum_h B_h / h (ascending h)
"""
import ctypes
import math
from fractions import Fraction

import numpy as np

from .core import OracleError, _p, lib

N_FEAT = 12
HIDDEN = 64
K_PAD = 16


def _declare():
    L = lib()
    if getattr(L, "_learned_declared", False):
        return L
    vp, i64, u64, u32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32
    L.or_edge_features.argtypes = [i64, i64] + [vp] * 3 + [vp] * 8 + [vp, i64, vp]
    L.or_edge_features.restype = ctypes.c_int
    L.or_sample_run_q.argtypes = [i64, i64] + [vp] * 3 + [vp] * 8 + [vp, i64, vp, vp, u32, u32, u64, u64, u64,
                                                                      vp, vp, vp]
    L.or_sample_run_q.restype = ctypes.c_int
    L.or_path_sum_q.argtypes = [i64, i64] + [vp] * 3 + [vp] * 8 + [vp, i64, vp, u32, u32, vp]
    L.or_path_sum_q.restype = ctypes.c_int
    L._learned_declared = True
    return L


def edge_features(g, plan, delta):
    """Counts of the 12 features per canonical edge, FP64 [m, 12]."""
    L = _declare()
    f = np.zeros((g.m, N_FEAT), np.float64)
    st = L.or_edge_features(g.n, g.m, *g._ptrs(), _p(plan.array()), int(delta), _p(f))
    if st:
        raise OracleError(st, "edge_features")
    return f


def sample_features(g, plan, delta, prefix, n, seed, offset=0):
    """Sample-statistics features (columns 12..15 of a feature row) of every
    canonical edge e = (u, v, t), from n samples of the plain sampler (ids
    offset .. offset + n - 1 of seed; Alg. 2, 3).  With the time bucket
    b(t) = (floor(t / D) - floor(t_min / D)) mod 2^32, D = max(delta, 1),
    t_min the graph's earliest time, and the keys K1 = (u, v), K2 = (u, b(t)),
    K3 = (v, b(t)): n_K is the number of samples whose middle edge has key K
    and s_K the sum of their X^2; prior = (sum of all X^2) / n.  Returns FP64
    [m, 4]: (s_K1 + prior) / (n_K1 + 1), the same for K2 and K3, and n_K1
    (log1p is applied with the other features)."""
    from .core import sample_run
    m = g.m
    out = np.zeros((m, 4), np.float64)
    if m == 0 or n == 0:
        return out
    _, tr = sample_run(g, plan, delta, prefix, n, seed, offset, trace=True)
    i2 = tr[:, 0].astype(np.int64)
    x2 = tr[:, 3].astype(np.float64) ** 2
    prior = float(x2.sum()) / n
    u = g.src[g.out_perm].astype(np.uint64)
    v = g.dst[g.out_perm].astype(np.uint64)
    t = g.t[g.out_perm]
    D = max(int(delta), 1)
    b = ((t // D) - (int(g.t.min()) // D)).astype(np.int64).astype(np.uint64) & np.uint64(0xFFFFFFFF)
    sh = np.uint64(32)
    for col, key in enumerate(((u << sh) | v, (u << sh) | b, (v << sh) | b)):
        ks, inv = np.unique(key[i2], return_inverse=True)
        cnt = np.bincount(inv, minlength=len(ks)).astype(np.float64)
        sx2 = np.bincount(inv, weights=x2, minlength=len(ks))
        pos = np.minimum(np.searchsorted(ks, key), len(ks) - 1)
        hit = ks[pos] == key
        n_e = np.where(hit, cnt[pos], 0.0)
        s_e = np.where(hit, sx2[pos], 0.0)
        out[:, col] = (s_e + prior) / (n_e + 1.0)
        if col == 0:
            out[:, 3] = n_e
    return out


def bf16(x):
    """Round to bfloat16 (through float32, both to nearest even); returns
    float32 values that are exactly representable in bfloat16."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).reshape(f.shape)


def features_bf16(counts, sample_stats=None):
    """log1p of the counts, rounded to bf16, in 16 columns; the four
    sample-statistics values (``sample_features``) fill columns 12..15 when
    given, else those columns are zero."""
    out = np.zeros((counts.shape[0], K_PAD), np.float32)
    out[:, :N_FEAT] = bf16(np.log1p(counts))
    if sample_stats is not None:
        out[:, N_FEAT:] = bf16(np.log1p(sample_stats))
    return out


def init_params(rng):
    """FP64 parameters (used by the tests only; the library has its own init)."""
    def u(shape, fan_in):
        b = 1.0 / math.sqrt(fan_in)
        return rng.uniform(-b, b, shape)
    return {"W1": u((HIDDEN, K_PAD), K_PAD), "b1": u(HIDDEN, K_PAD), "W2": u((HIDDEN, HIDDEN), HIDDEN),
            "b2": u(HIDDEN, HIDDEN),
            "W3": u(HIDDEN, HIDDEN), "b3": u(1, HIDDEN)}


def pack(params):
    """Flat FP32 layout shared with the library's tc_mlp_get/set_params:
    W1[64][16], b1[64], W2[64][64], b2[64], W3[64], b3[1]."""
    return np.concatenate([params["W1"].ravel(), params["b1"].ravel(), params["W2"].ravel(), params["b2"].ravel(),
                           params["W3"].ravel(), params["b3"].ravel()]).astype(np.float64)


def unpack(flat):
    flat = np.asarray(flat, np.float64)
    o = 0
    out = {}
    for name, shape in (("W1", (HIDDEN, K_PAD)), ("b1", (HIDDEN,)), ("W2", (HIDDEN, HIDDEN)), ("b2", (HIDDEN,)),
                        ("W3", (HIDDEN,)), ("b3", (1,))):
        size = int(np.prod(shape))
        out[name] = flat[o:o + size].reshape(shape)
        o += size
    return out


N_PARAMS = HIDDEN * K_PAD + HIDDEN + HIDDEN * HIDDEN + HIDDEN + HIDDEN + 1


def mlp_forward(params, x, round_acts=True, quantized=True):
    """z3 (logits) for rows x [B, 16].  Weights and inputs are taken as bf16
    and biases as FP32 (quantized); products and sums in FP64; the hidden
    activations are rounded to bf16 like the library's tensor-core path when
    round_acts.  quantized=False, round_acts=False is the plain FP64 network."""
    if quantized:
        W1, W2, W3 = (bf16(params[k]).astype(np.float64) for k in ("W1", "W2", "W3"))
        b1, b2, b3 = (np.float32(params[k]).astype(np.float64) for k in ("b1", "b2", "b3"))
        x = bf16(x).astype(np.float64)
    else:
        W1, W2, W3, b1, b2, b3 = (np.asarray(params[k], np.float64) for k in ("W1", "W2", "W3", "b1", "b2", "b3"))
        x = np.asarray(x, np.float64)
    z1 = x @ W1.T + b1
    a1 = np.maximum(z1, 0.0)
    if round_acts:
        a1 = bf16(a1).astype(np.float64)
    z2 = a1 @ W2.T + b2
    a2 = np.maximum(z2, 0.0)
    if round_acts:
        a2 = bf16(a2).astype(np.float64)
    z3 = a2 @ W3 + b3[0]
    return z3, (x, z1, a1, z2, a2)


def closure_loss(z3, y):
    """Mean closure loss of g = sigmoid(z3) against closure counts y >= 0:
    y softplus(-z3) = -y log g where y > 0, softplus(z3) = -log(1 - g) where
    y = 0.  For labels 0 and 1 it is the binary cross-entropy; its minimiser
    per input is g = E[y] / (E[y] + P(y = 0))."""
    y = np.asarray(y, np.float64)
    return float(np.mean(np.where(y > 0, y * np.logaddexp(0.0, -z3), np.logaddexp(0.0, z3))))


def variance_loss(z3, X, eps):
    """Estimator-variance objective over a batch of plain samples (paths drawn
    with probability w_e / W, closure counts X): with h = eps + sigmoid(z3),
    the second moment of one importance-weighted sample under q ~ w h is
    (Q / W) * E_plain[X^2 / h] with Q / W = E_plain[h]; the objective is the
    batch estimate mean(h) * mean(X^2 / h).  Its minimiser over per-edge h is
    h proportional to sqrt(E[X^2 | e]) (Cauchy-Schwarz)."""
    h = eps + 1.0 / (1.0 + np.exp(-np.asarray(z3, np.float64)))
    X = np.asarray(X, np.float64)
    return float(np.mean(h) * np.mean(X * X / h))


def variance_dz(z3, X, eps):
    """d variance_loss / d z3 for each row: with A = mean(h), B = mean(X^2/h)
    and g' = g (1 - g), (B - A X^2 / h^2) g' / n."""
    g = 1.0 / (1.0 + np.exp(-np.asarray(z3, np.float64)))
    h = eps + g
    X = np.asarray(X, np.float64)
    A, Bm = np.mean(h), np.mean(X * X / h)
    return (Bm - A * X * X / (h * h)) * g * (1.0 - g) / len(X)


def mlp_backward(params, x, y, round_acts=True, quantized=True, objective="closure", eps=0.05):
    """Gradients of closure_loss(mlp_forward(x), y) -- or, for objective
    "variance", of variance_loss(mlp_forward(x), y, eps) -- with respect to
    the FP32 parameters (the bf16 roundings are treated as identity in the
    chain rule, as in the library's backward)."""
    z3, (xb, z1, a1, z2, a2) = mlp_forward(params, x, round_acts, quantized)
    B = len(y)
    if quantized:
        W2 = bf16(params["W2"]).astype(np.float64)
        W3 = bf16(params["W3"]).astype(np.float64)
    else:
        W2 = np.asarray(params["W2"], np.float64)
        W3 = np.asarray(params["W3"], np.float64)
    y = np.asarray(y, np.float64)
    if objective == "variance":
        dz3 = variance_dz(z3, y, eps)
    else:
        g3 = 1.0 / (1.0 + np.exp(-z3))
        dz3 = np.where(y > 0, -y * (1.0 - g3), g3) / B
    g = {"W3": a2.T @ dz3, "b3": np.array([dz3.sum()])}
    dz2 = np.outer(dz3, W3) * (z2 > 0)
    g["W2"] = dz2.T @ a1
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ W2) * (z1 > 0)
    g["W1"] = dz1.T @ xb
    g["b1"] = dz1.sum(0)
    return g, (variance_loss(z3, y, eps) if objective == "variance" else closure_loss(z3, y))


def proposal_h(g, eps, scale):
    """h = max(1, floor(scale * (eps + g) + 1/2)) in FP32, as the library."""
    v = np.floor(np.float32(scale) * (np.float32(eps) + np.asarray(g, np.float32)) + np.float32(0.5))
    return np.maximum(1, v).astype(np.uint16)


def qprefix(w, h):
    q = np.asarray(w, np.uint64) * np.asarray(h, np.uint64)
    from .core import prefix_sum
    return prefix_sum(q)


def sample_run_q(g, plan, delta, qpre, h, k, seed, offset=0, trace=False):
    L = _declare()
    h = np.ascontiguousarray(h, dtype=np.uint16)
    h_lo, h_hi = int(h.min()) if len(h) else 1, int(h.max()) if len(h) else 1
    bins = np.zeros(3 * (h_hi - h_lo + 1), np.uint64)
    sums = np.zeros(3, np.uint64)
    tr = np.empty((k, 4), np.uint64) if trace else None
    qpre = np.ascontiguousarray(qpre, dtype=np.uint64)
    st = L.or_sample_run_q(g.n, g.m, *g._ptrs(), _p(plan.array()), int(delta), _p(qpre), _p(h), h_lo, h_hi, int(k),
                           int(seed), int(offset), _p(tr) if trace else None, _p(bins), _p(sums))
    if st:
        raise OracleError(st, "sample_run_q")
    b = bins.reshape(-1, 3)
    out = {"h_lo": h_lo, "B": [int(v) for v in b[:, 0]],
           "B2": [int(lo) | (int(hi) << 64) for lo, hi in zip(b[:, 1], b[:, 2])],
           "hits": int(sums[0]), "k": int(k), "Q": int(qpre[-1])}
    return out, tr


def estimate_q(B, B2, h_lo, Q, k):
    """C_hat = Q / k * sum over ascending h of B_h / h (FP64 in that order);
    SE from sum Y = Q sum B_h / h and sum Y^2 = Q^2 sum B2_h / h^2."""
    if k == 0 or Q == 0:
        return 0.0, 0.0
    s1 = 0.0
    s2 = 0.0
    for j, (b, b2) in enumerate(zip(B, B2)):
        h = float(h_lo + j)
        s1 += float(b) / h
        s2 += float(b2) / (h * h)
    Qf, kf = float(Q), float(k)
    est = Qf / kf * s1
    if k < 2:
        return est, float("nan")
    sy, sy2 = Qf * s1, Qf * Qf * s2
    var = max((sy2 - sy * sy / kf) / (kf - 1.0), 0.0)
    return est, math.sqrt(var / kf)


def path_sum_q(g, plan, delta, h):
    """Per-h exhaustive sums of C_P and C_P^2 over all class paths."""
    L = _declare()
    h = np.ascontiguousarray(h, dtype=np.uint16)
    h_lo, h_hi = int(h.min()), int(h.max())
    acc = np.zeros(3 * (h_hi - h_lo + 1), np.uint64)
    st = L.or_path_sum_q(g.n, g.m, *g._ptrs(), _p(plan.array()), int(delta), _p(h), h_lo, h_hi, _p(acc))
    if st:
        raise OracleError(st, "path_sum_q")
    a = acc.reshape(-1, 3)
    return h_lo, [int(v) for v in a[:, 0]], [int(lo) | (int(hi) << 64) for lo, hi in zip(a[:, 1], a[:, 2])]


def exact_variance_q(Q, C, h_lo, S2):
    """Var(Y) = Q sum_P C_P^2 / h_P - C^2 (exact rational)."""
    return Fraction(Q) * sum(Fraction(s2, h_lo + j) for j, s2 in enumerate(S2)) - Fraction(C) ** 2
