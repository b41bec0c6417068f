"""Python binding of the tc C ABI (include/tc.h).

Argument marshalling only: every step of the method runs in the CUDA library
``libtc.so``.  Device buffers are torch CUDA tensors; torch provides memory
and streams, nothing else.  If the library is missing the import fails loudly;
there is no CPU fallback.
"""
import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtc.so")

TC_OK = 0
STATUS_NAMES = {0: "TC_OK", 1: "TC_ERR_INVALID_ARG", 2: "TC_ERR_OOM", 3: "TC_ERR_OVERFLOW", 4: "TC_ERR_CUDA",
                5: "TC_ERR_UNSUPPORTED_MOTIF", 6: "TC_ERR_RNG_EXHAUSTED", 7: "TC_ERR_TIMEOUT",
                8: "TC_ERR_BOUNDS"}
WINDOW_STRICT, WINDOW_CLOSED = 0, 1

ARRAYS = {"out_off": 0, "out_edges": 1, "edge_perm": 2, "in_off": 3, "in_edges": 4, "pair_off": 5,
          "pair_dst": 6, "pair_eoff": 7, "pair_t": 8, "pair_eid": 9, "in_eid": 10}


class TcError(RuntimeError):
    def __init__(self, status, what, msg):
        super().__init__("%s: %s (%s)" % (what, STATUS_NAMES.get(status, status), msg))
        self.status = status


class tc_motif(ctypes.Structure):
    _fields_ = [("num_edges", ctypes.c_int32), ("src", ctypes.c_int8 * 16), ("dst", ctypes.c_int8 * 16),
                ("anchor", ctypes.c_int32 * 3), ("window", ctypes.c_int32)]


class tc_estimate(ctypes.Structure):
    _fields_ = [("W", ctypes.c_uint64), ("k", ctypes.c_uint64), ("sum_x", ctypes.c_uint64),
                ("sum_x2_lo", ctypes.c_uint64), ("sum_x2_hi", ctypes.c_uint64), ("hits", ctypes.c_uint64),
                ("checked", ctypes.c_uint64), ("estimate", ctypes.c_double), ("std_err", ctypes.c_double)]


class tc_query(ctypes.Structure):
    _fields_ = [("graph", ctypes.c_void_p), ("motif", tc_motif), ("delta", ctypes.c_int64), ("k", ctypes.c_uint64),
                ("seed", ctypes.c_uint64), ("sample_offset", ctypes.c_uint64)]


class tc_batch_options(ctypes.Structure):
    _fields_ = [("block_size", ctypes.c_int32), ("tile", ctypes.c_uint32), ("use_graph", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class tc_graph_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("num_pairs", ctypes.c_int64),
                ("t_min", ctypes.c_int64), ("t_max", ctypes.c_int64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libtc.so is not built; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, u64, i32, st = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int
        sz = ctypes.c_size_t
        sig = {
            "tc_build_temporal_csr": [i64, i64, vp, vp, vp, vp, ctypes.POINTER(vp)],
            "tc_graph_destroy": [vp],
            "tc_graph_info_get": [vp, ctypes.POINTER(tc_graph_info)],
            "tc_graph_copy": [vp, i32, vp, vp],
            "tc_graph_edge_order": [vp, vp, vp],
            "tc_estimate_from_sums": [u64, u64, u64, u64, u64, ctypes.POINTER(tc_estimate)],
            "tc_sample_index_bytes": [vp, ctypes.POINTER(sz)],
            "tc_path_weights": [vp, ctypes.POINTER(tc_motif), i64, vp, vp, vp, ctypes.POINTER(u64), vp],
            "tc_sample_estimate": [vp, ctypes.POINTER(tc_motif), i64, vp, vp, u64, u64, u64,
                                   ctypes.POINTER(tc_estimate), vp],
            "tc_sample_trace": [vp, ctypes.POINTER(tc_motif), i64, vp, vp, u64, u64, u64, vp, vp],
            "tc_estimate_from_host": [i64, i64, vp, vp, vp, ctypes.POINTER(tc_motif), i64, u64, u64,
                                      ctypes.POINTER(tc_estimate), vp],
            "tc_motif_plan": [ctypes.POINTER(tc_motif), vp, vp],
            "tc_prefix_sum_noalloc": [vp, u64, vp, ctypes.POINTER(u64), vp],
            "tc_exact_count": [vp, ctypes.POINTER(tc_motif), i64, vp, vp, ctypes.POINTER(tc_estimate), vp],
            "tc_mlp_create": [u64, ctypes.POINTER(vp)],
            "tc_mlp_destroy": [vp],
            "tc_mlp_get_params": [vp, vp],
            "tc_mlp_set_params": [vp, vp],
            "tc_edge_features": [vp, ctypes.POINTER(tc_motif), i64, vp, vp, vp],
            "tc_sample_features": [vp, ctypes.POINTER(tc_motif), i64, vp, vp, u64, u64, u64, vp, vp],
            "tc_mlp_forward": [vp, vp, vp, u64, vp, vp],
            "tc_mlp_grad": [vp, vp, vp, vp, u64, vp, ctypes.POINTER(ctypes.c_float), vp],
            "tc_mlp_train": [vp, vp, ctypes.POINTER(tc_motif), i64, vp, vp, vp, u64, u64, ctypes.c_uint32,
                             ctypes.c_float, vp, vp],
            "tc_mlp_grad_ex": [vp, vp, vp, vp, u64, ctypes.c_int32, ctypes.c_float, vp,
                               ctypes.POINTER(ctypes.c_float), vp],
            "tc_mlp_train_ex": [vp, vp, ctypes.POINTER(tc_motif), i64, vp, vp, vp, u64, u64, ctypes.c_uint32,
                                ctypes.c_float, ctypes.c_int32, ctypes.c_float, vp, vp],
            "tc_proposal_index_bytes": [vp, ctypes.POINTER(sz)],
            "tc_proposal_weights": [vp, vp, ctypes.POINTER(tc_motif), i64, vp, vp, ctypes.c_float, ctypes.c_uint32,
                                    vp, vp, vp, ctypes.POINTER(u64), vp],
            "tc_sample_estimate_q": [vp, ctypes.POINTER(tc_motif), i64, vp, vp, vp, vp, u64, u64, u64,
                                     ctypes.POINTER(tc_estimate), vp, vp, vp],
            "tc_batch_create": [ctypes.POINTER(tc_query), i64, ctypes.POINTER(tc_batch_options), vp,
                                ctypes.POINTER(vp)],
            "tc_batch_run": [vp, ctypes.POINTER(tc_estimate), vp],
            "tc_batch_info": [vp, ctypes.POINTER(tc_batch_options), ctypes.POINTER(u64), ctypes.POINTER(u64),
                              ctypes.POINTER(u64)],
            "tc_batch_timing": [vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)],
            "tc_batch_destroy": [vp],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = st
        L.tc_kernel_launches.argtypes = []
        L.tc_kernel_launches.restype = ctypes.c_uint64
        L.tc_set_timing.argtypes = [ctypes.c_int32]
        L.tc_set_timing.restype = st
        L.tc_last_sampler_ms.argtypes = []
        L.tc_last_sampler_ms.restype = ctypes.c_float
        L.tc_last_phase_ms.argtypes = [ctypes.c_int32]
        L.tc_last_phase_ms.restype = ctypes.c_float
        L.tc_mlp_kernel.argtypes = [ctypes.c_int32]
        L.tc_mlp_kernel.restype = ctypes.c_int32
        L.tc_last_error.argtypes = []
        L.tc_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(status, what):
    if status != TC_OK:
        raise TcError(status, what, lib().tc_last_error().decode())


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def tc_kernel_launches():
    return int(lib().tc_kernel_launches())


def tc_set_timing(enabled):
    _check(lib().tc_set_timing(1 if enabled else 0), "tc_set_timing")


def tc_last_sampler_ms():
    return float(lib().tc_last_sampler_ms())


PHASES = {"weights": 0, "index": 1, "order": 2, "sample": 3, "proposal": 4}


MLP_KERNELS = {"mma": 0, "tcgen05": 1}


def tc_mlp_kernel(kind=None):
    """Select ("mma" or "tcgen05") or, with None, query the kernel that runs
    the network's inference in this process; returns the name in effect."""
    k = -1 if kind is None else MLP_KERNELS[kind]
    r = int(lib().tc_mlp_kernel(k))
    return {v: n for n, v in MLP_KERNELS.items()}[r]


def tc_last_phase_ms(phase):
    """Device ms of a phase ("weights": a1 + a2, "index", "order", "sample",
    "proposal": network + h + q + q-prefix) in the last call on this thread
    that ran it with timing enabled."""
    return float(lib().tc_last_phase_ms(PHASES[phase]))


def make_motif(edges, anchor=None, window=WINDOW_STRICT):
    """Motif M = (H, pi) from a list of (src_label, dst_label); edge i has
    time rank i (Def. 1)."""
    m = tc_motif()
    m.num_edges = len(edges)
    for i, (a, b) in enumerate(edges):
        m.src[i] = int(a)
        m.dst[i] = int(b)
    a = anchor if anchor is not None else (-1, -1, -1)
    for i in range(3):
        m.anchor[i] = int(a[i])
    m.window = int(window)
    return m


def tc_motif_plan(motif):
    anchor = (ctypes.c_int32 * 3)()
    cls = (ctypes.c_int32 * 4)()
    _check(lib().tc_motif_plan(ctypes.byref(motif), ctypes.cast(anchor, ctypes.c_void_p),
                               ctypes.cast(cls, ctypes.c_void_p)), "tc_motif_plan")
    return tuple(anchor), tuple(cls)


class Graph:
    """Owner of a device-resident tc_graph."""

    def __init__(self, handle):
        self._h = handle
        info = tc_graph_info()
        _check(lib().tc_graph_info_get(handle, ctypes.byref(info)), "tc_graph_info_get")
        self.n, self.m, self.num_pairs = info.n, info.m, info.num_pairs
        self.t_min, self.t_max = info.t_min, info.t_max

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("graph destroyed")
        return self._h

    def destroy(self):
        if self._h is not None:
            lib().tc_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def array(self, name, stream=None):
        """Copy an internal array to a new CUDA tensor (layouts in tc.h)."""
        n1, m, P = self.n + 1, self.m, self.num_pairs
        shapes = {"out_off": (n1, torch.int32), "out_edges": (4 * m, torch.int32), "edge_perm": (m, torch.int32),
                  "in_off": (n1, torch.int32), "in_edges": (4 * m, torch.int32), "pair_off": (n1, torch.int32),
                  "pair_dst": (P, torch.int32), "pair_eoff": (P + 1, torch.int32), "pair_t": (m, torch.int64),
                  "pair_eid": (m, torch.int32), "in_eid": (m, torch.int32)}
        size, dt = shapes[name]
        out = torch.empty(max(size, 1), dtype=dt, device="cuda")
        _check(lib().tc_graph_copy(self.handle, ARRAYS[name], _ptr(out), _stream(stream)), "tc_graph_copy")
        return out[:size]


def tc_build_temporal_csr(n, src, dst, t, stream=None):
    """src, dst: int32 CUDA tensors, t: int64 CUDA tensor, input order."""
    assert src.is_cuda and dst.is_cuda and t.is_cuda
    assert src.dtype == torch.int32 and dst.dtype == torch.int32 and t.dtype == torch.int64
    src, dst, t = src.contiguous(), dst.contiguous(), t.contiguous()
    h = ctypes.c_void_p()
    _check(lib().tc_build_temporal_csr(int(n), int(src.numel()), _ptr(src), _ptr(dst), _ptr(t), _stream(stream),
                                       ctypes.byref(h)), "tc_build_temporal_csr")
    return Graph(h)


def tc_graph_edge_order(g, stream=None):
    """int64 CUDA tensor: input index of the edge at each canonical position."""
    out = torch.empty(max(g.m, 1), dtype=torch.int64, device="cuda")
    _check(lib().tc_graph_edge_order(g.handle, _ptr(out), _stream(stream)), "tc_graph_edge_order")
    return out[:g.m]


def tc_sample_index_bytes(g):
    b = ctypes.c_size_t()
    _check(lib().tc_sample_index_bytes(g.handle, ctypes.byref(b)), "tc_sample_index_bytes")
    return b.value


class Weights:
    """Prefix sums and sampling index of one (graph, motif, delta)."""

    def __init__(self, prefix, index, w, W):
        self.prefix, self.index, self.w, self.W = prefix, index, w, W


def alloc_weights(g, want_w=False):
    m = g.m
    prefix = torch.empty(m + 1, dtype=torch.int64, device="cuda")
    index = torch.empty(tc_sample_index_bytes(g), dtype=torch.uint8, device="cuda")
    w = torch.empty(max(m, 1), dtype=torch.int64, device="cuda") if want_w else None
    return Weights(prefix, index, w, None)


def tc_path_weights(g, motif, delta, out=None, want_W=True, want_w=False, stream=None):
    """Claim 1 / Alg. 1 on the device; returns a Weights with W (host) when
    want_W (which synchronises)."""
    if out is None:
        out = alloc_weights(g, want_w)
    W = ctypes.c_uint64(0)
    _check(lib().tc_path_weights(g.handle, ctypes.byref(motif), int(delta), _ptr(out.w), _ptr(out.prefix),
                                 _ptr(out.index), ctypes.byref(W) if want_W else None, _stream(stream)),
           "tc_path_weights")
    if want_W:
        out.W = W.value
    return out


def _est_dict(e):
    return {"W": e.W, "k": e.k, "sum_x": e.sum_x, "sum_x2": e.sum_x2_lo | (e.sum_x2_hi << 64), "hits": e.hits,
            "checked": e.checked, "estimate": e.estimate, "std_err": e.std_err}


def tc_sample_estimate(g, motif, delta, weights, k, seed=0, offset=0, stream=None):
    e = tc_estimate()
    _check(lib().tc_sample_estimate(g.handle, ctypes.byref(motif), int(delta), _ptr(weights.prefix),
                                    _ptr(weights.index), int(k), int(seed), int(offset), ctypes.byref(e),
                                    _stream(stream)), "tc_sample_estimate")
    return _est_dict(e)


def tc_exact_count(g, motif, delta, weights, stream=None):
    """Exact count C by summing CheckMotif over all W class paths."""
    e = tc_estimate()
    _check(lib().tc_exact_count(g.handle, ctypes.byref(motif), int(delta), _ptr(weights.prefix), _ptr(weights.index),
                                ctypes.byref(e), _stream(stream)), "tc_exact_count")
    return _est_dict(e)


def tc_sample_trace(g, motif, delta, weights, count, seed=0, offset=0, stream=None):
    """(count, 4) int64 tensor of (middle edge, e1 position, e3 position, X)."""
    tr = torch.empty((max(count, 1), 4), dtype=torch.int64, device="cuda")
    _check(lib().tc_sample_trace(g.handle, ctypes.byref(motif), int(delta), _ptr(weights.prefix),
                                 _ptr(weights.index), int(count), int(seed), int(offset), _ptr(tr), _stream(stream)),
           "tc_sample_trace")
    return tr[:count]


def tc_estimate_from_host(n, src, dst, t, motif, delta, k, seed=0, stream=None):
    """Whole method from host arrays (numpy or CPU tensors, ideally pinned)."""
    def hp(a, dt):
        if isinstance(a, torch.Tensor):
            assert not a.is_cuda and a.dtype == dt and a.is_contiguous()
            return a, ctypes.c_void_p(a.data_ptr())
        a = np.ascontiguousarray(a, dtype={torch.int32: np.int32, torch.int64: np.int64}[dt])
        return a, a.ctypes.data_as(ctypes.c_void_p)
    ks, ps = hp(src, torch.int32)
    kd, pd = hp(dst, torch.int32)
    kt, pt = hp(t, torch.int64)
    e = tc_estimate()
    _check(lib().tc_estimate_from_host(int(n), int(len(ks)), ps, pd, pt, ctypes.byref(motif), int(delta), int(k),
                                       int(seed), ctypes.byref(e), _stream(stream)), "tc_estimate_from_host")
    return _est_dict(e)


NOALLOC_MAX_EDGES = 1 << 28


def tc_prefix_sum_noalloc(w, m, prefix, want_W=True, stream=None):
    """Prefix sum of w[:m] into prefix[:m+1] without device allocation (for
    callers that cannot allocate device memory).  Returns W when want_W."""
    W = ctypes.c_uint64(0)
    _check(lib().tc_prefix_sum_noalloc(_ptr(w), int(m), _ptr(prefix), ctypes.byref(W) if want_W else None,
                                       _stream(stream)), "tc_prefix_sum_noalloc")
    return W.value if want_W else None


def tc_estimate_from_sums(sum_x, sum_x2, k, W):
    """Alg. 5's estimate and standard error from exact sums (for example the
    sums of runs over disjoint sample-id ranges, added up), formed by the
    library; sum_x2 is a Python int below 2^128.  Host only."""
    sum_x2 = int(sum_x2)
    e = tc_estimate()
    _check(lib().tc_estimate_from_sums(int(sum_x), sum_x2 & 0xFFFFFFFFFFFFFFFF, sum_x2 >> 64, int(k), int(W),
                                       ctypes.byref(e)), "tc_estimate_from_sums")
    return e.estimate, e.std_err


# ---------------------------------------------------------------------------
# Learned proposal

MLP_PARAMS = 5313
FEATURE_STRIDE = 16
PROPOSAL_MAX_H = 4095


class MLP:
    """Owner of a device-resident tc_mlp (12 -> 64 -> 64 -> 1 network)."""

    def __init__(self, seed=0):
        h = ctypes.c_void_p()
        _check(lib().tc_mlp_create(int(seed), ctypes.byref(h)), "tc_mlp_create")
        self._h = h

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("mlp destroyed")
        return self._h

    def destroy(self):
        if self._h is not None:
            lib().tc_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def get_params(self):
        out = np.empty(MLP_PARAMS, np.float32)
        _check(lib().tc_mlp_get_params(self.handle, out.ctypes.data_as(ctypes.c_void_p)), "tc_mlp_get_params")
        return out

    def set_params(self, params):
        arr = np.ascontiguousarray(params, dtype=np.float32)
        assert arr.size == MLP_PARAMS
        _check(lib().tc_mlp_set_params(self.handle, arr.ctypes.data_as(ctypes.c_void_p)), "tc_mlp_set_params")


def alloc_features(g):
    """A zeroed feature buffer for tc_edge_features (int16 [m, 16], the bf16 bits)."""
    return torch.zeros((max(g.m, 1), FEATURE_STRIDE), dtype=torch.int16, device="cuda")


def tc_edge_features(g, motif, delta, weights, out=None, stream=None):
    """bf16 feature rows [m, 16] (returned as a torch.bfloat16 CUDA tensor),
    into out (from alloc_features) when given."""
    feat = alloc_features(g) if out is None else out
    _check(lib().tc_edge_features(g.handle, ctypes.byref(motif), int(delta), _ptr(weights.index), _ptr(feat),
                                  _stream(stream)), "tc_edge_features")
    return feat[:g.m].view(torch.bfloat16)


def tc_sample_features(g, motif, delta, weights, feat, n_samples, seed=0, offset=0, stream=None):
    """Fill columns 12..15 of feat (bf16 rows [m, 16]) from n_samples plain samples."""
    _check(lib().tc_sample_features(g.handle, ctypes.byref(motif), int(delta), _ptr(weights.prefix),
                                    _ptr(weights.index), int(n_samples), int(seed), int(offset), _ptr(feat),
                                    _stream(stream)), "tc_sample_features")
    return feat


def tc_mlp_forward(mlp, feat, rows=None, n=None, stream=None):
    n = int(n if n is not None else (rows.numel() if rows is not None else feat.shape[0]))
    out = torch.empty(max(n, 1), dtype=torch.float32, device="cuda")
    _check(lib().tc_mlp_forward(mlp.handle, _ptr(feat), _ptr(rows), n, _ptr(out), _stream(stream)),
           "tc_mlp_forward")
    return out[:n]


OBJECTIVES = {"closure": 0, "variance": 1, "bce": 2}


def tc_mlp_grad(mlp, feat, rows, labels, objective="closure", eps=0.05, stream=None):
    n = int(labels.numel())
    grad = torch.empty(MLP_PARAMS, dtype=torch.float32, device="cuda")
    loss = ctypes.c_float(0.0)
    _check(lib().tc_mlp_grad_ex(mlp.handle, _ptr(feat), _ptr(rows), _ptr(labels), n, OBJECTIVES[objective],
                                float(eps), _ptr(grad), ctypes.byref(loss), _stream(stream)), "tc_mlp_grad")
    return grad, loss.value


def tc_mlp_train(mlp, g, motif, delta, weights, feat, n_samples, seed=0, batch=16384, lr=2e-3, objective="closure",
                 eps=0.05, stream=None):
    """Returns the loss of the first and the last batch (the mean closure
    loss, or the variance objective)."""
    losses = np.zeros(2, np.float32)
    _check(lib().tc_mlp_train_ex(mlp.handle, g.handle, ctypes.byref(motif), int(delta), _ptr(weights.prefix),
                                 _ptr(weights.index), _ptr(feat), int(n_samples), int(seed), int(batch), float(lr),
                                 OBJECTIVES[objective], float(eps), losses.ctypes.data_as(ctypes.c_void_p),
                                 _stream(stream)), "tc_mlp_train")
    return float(losses[0]), float(losses[1])


class Proposal:
    def __init__(self, h, qprefix, qindex, Q):
        self.h, self.qprefix, self.qindex, self.Q = h, qprefix, qindex, Q


def tc_proposal_weights(mlp, g, motif, delta, weights, feat, eps=0.05, scale=1024, stream=None):
    m = g.m
    b = ctypes.c_size_t()
    _check(lib().tc_proposal_index_bytes(g.handle, ctypes.byref(b)), "tc_proposal_index_bytes")
    h = torch.empty(max(m, 1), dtype=torch.int16, device="cuda")
    qprefix = torch.empty(m + 1, dtype=torch.int64, device="cuda")
    qindex = torch.empty(b.value, dtype=torch.uint8, device="cuda")
    Q = ctypes.c_uint64(0)
    _check(lib().tc_proposal_weights(mlp.handle, g.handle, ctypes.byref(motif), int(delta), _ptr(weights.prefix),
                                     _ptr(feat), float(eps), int(scale), _ptr(h), _ptr(qprefix), _ptr(qindex),
                                     ctypes.byref(Q), _stream(stream)), "tc_proposal_weights")
    return Proposal(h[:m], qprefix, qindex, Q.value)


def tc_sample_estimate_q(g, motif, delta, weights, proposal, k, seed=0, offset=0, want_bins=False, trace=False,
                         stream=None):
    e = tc_estimate()
    bins = np.zeros(3 * (PROPOSAL_MAX_H + 1), np.uint64) if want_bins else None
    tr = torch.empty((max(k, 1), 4), dtype=torch.int64, device="cuda") if trace else None
    _check(lib().tc_sample_estimate_q(g.handle, ctypes.byref(motif), int(delta), _ptr(weights.index),
                                      _ptr(proposal.h), _ptr(proposal.qprefix), _ptr(proposal.qindex), int(k),
                                      int(seed), int(offset), ctypes.byref(e),
                                      bins.ctypes.data_as(ctypes.c_void_p) if want_bins else None, _ptr(tr),
                                      _stream(stream)), "tc_sample_estimate_q")
    out = _est_dict(e)
    if want_bins:
        b = bins.reshape(-1, 3)
        out["bins"] = b
    if trace:
        out["trace"] = tr[:k]
    return out


class Batch:
    """A fixed list of queries answered together (tc_batch_*).  queries: a
    list of (graph, motif edges or tc_motif, delta, k, seed, sample_offset);
    the graphs must outlive the batch."""

    def __init__(self, queries, block_size=0, tile=0, use_graph=True, stream=None):
        self._graphs = [q[0] for q in queries]
        arr = (tc_query * max(1, len(queries)))()
        for i, (g, motif, delta, k, seed, offset) in enumerate(queries):
            arr[i].graph = g.handle
            arr[i].motif = motif if isinstance(motif, tc_motif) else make_motif(motif)
            arr[i].delta = int(delta)
            arr[i].k = int(k)
            arr[i].seed = int(seed)
            arr[i].sample_offset = int(offset)
        opts = tc_batch_options(int(block_size), int(tile), 1 if use_graph else 0, 0)
        h = ctypes.c_void_p()
        _check(lib().tc_batch_create(arr, len(queries), ctypes.byref(opts), _stream(stream), ctypes.byref(h)),
               "tc_batch_create")
        self._h = h
        self.nq = len(queries)

    @property
    def handle(self):
        if not self._h:
            raise ValueError("batch destroyed")
        return self._h

    def run(self, stream=None):
        out = (tc_estimate * max(1, self.nq))()
        _check(lib().tc_batch_run(self.handle, out, _stream(stream)), "tc_batch_run")
        return [_est_dict(out[i]) for i in range(self.nq)]

    def info(self):
        o = tc_batch_options()
        launches, nbytes, slots = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(lib().tc_batch_info(self.handle, ctypes.byref(o), ctypes.byref(launches), ctypes.byref(nbytes),
                                   ctypes.byref(slots)), "tc_batch_info")
        return {"block_size": o.block_size, "tile": o.tile, "use_graph": bool(o.use_graph),
                "launches_per_run": launches.value, "device_bytes": nbytes.value, "weight_slots": slots.value}

    def timing(self):
        """Device milliseconds of the last run: (whole run, sampling launch)."""
        run, samp = ctypes.c_float(), ctypes.c_float()
        _check(lib().tc_batch_timing(self.handle, ctypes.byref(run), ctypes.byref(samp)), "tc_batch_timing")
        return run.value, samp.value

    def destroy(self):
        if self._h:
            lib().tc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
