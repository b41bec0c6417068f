/*
 * tc.h -- C ABI of the GB300 temporal 3-path sampling library.
 *
 * Implements the estimator of Pu, Wang, Seshadhri, Aiken, Ganesh, Kolda,
 * Phillips, "Accurate and Fast Estimation of Temporal Motifs using Path
 * Sampling" (ICDM 2024):
 *   - input: a directed temporal multigraph of edges (u, v, t)      (Sec. I-A)
 *   - motif M = (H, pi, delta) on four vertices                     (Def. 1, 2)
 *   - path weights w_e = product of windowed degrees               (Claim 1, Alg. 1)
 *   - sampling of delta-centered 3-paths proportional to w_e       (Alg. 2, Lemma 1)
 *   - CheckMotif / ListCount completion count per sampled path     (Alg. 3, Alg. 4)
 *   - estimate C_hat = (sum X / k) * W                             (Alg. 5, Claim 2)
 *
 * Conventions for every call:
 *   - "d_" pointers are CUDA device pointers, "h_" pointers host pointers.
 *     Device pointers passed in are borrowed: the library never keeps them
 *     after the call returns.
 *   - stream is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Work is enqueued on it; calls that return host values synchronise it.
 *   - Library objects (tc_graph) own device memory taken with
 *     cudaMallocAsync on the creating stream; *_destroy frees it.
 *   - No C++ exception crosses the ABI.  Every call returns a tc_status; on
 *     failure tc_last_error() returns a message for the calling thread.
 *   - Conditions detected inside kernels (an overflow of the 64-bit counts,
 *     a vertex id out of range, an exhausted RNG rejection loop) are collected
 *     in a device error word and returned as a status at the next point where
 *     the call synchronises.
 *   - Integer counts are exact: weights, prefix sums and per-sample counts are
 *     uint64; the sum of squares is 128 bits.  FP64 is used only for the final
 *     estimate and its standard error, on the host.
 *   - Limits: 0 <= m < 2^32 - 1 edges, 1 <= n < 2^31 vertices, delta >= 0.
 *     Windows t - delta and t + delta saturate at the int64 range.
 *
 * Edge orders (fixed by this ABI, needed to read back positions):
 *   canonical order = out-lists: edges sorted by (src, t, input index)
 *   in-lists        = edges sorted by (dst, t, input index)
 *   pair lists      = edges sorted by (src, dst, t, input index)
 */
#ifndef TC_H
#define TC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TC_OK = 0,
  TC_ERR_INVALID_ARG = 1,      /* bad size, pointer, id, motif or mismatched index */
  TC_ERR_OOM = 2,              /* device allocation failed */
  TC_ERR_OVERFLOW = 3,         /* a uint64 count (W, sum of X, X) overflowed */
  TC_ERR_CUDA = 4,             /* a CUDA runtime call failed */
  TC_ERR_UNSUPPORTED_MOTIF = 5,/* no anchor 3-path containing edge 0 */
  TC_ERR_RNG_EXHAUSTED = 6,    /* 64 rejected draws in a row (probability ~0) */
  TC_ERR_TIMEOUT = 7,          /* a bounded device wait gave up */
  TC_ERR_BOUNDS = 8            /* a device index check failed */
} tc_status;

/* Opaque, device-resident temporal graph: out-, in- and pair-lists. */
typedef struct tc_graph tc_graph;

#define TC_MAX_MOTIF_EDGES 16
#define TC_WINDOW_STRICT 0 /* end edges strictly before/after the middle (Def. 5) */
#define TC_WINDOW_CLOSED 1 /* closed windows [t-delta,t], [t,t+delta] (Claim 1)  */

/*
 * Temporal motif M = (H, pi, delta) without delta (Def. 1).  Edge i of H runs
 * from vertex label src[i] to dst[i] (labels 0..3, no self-loops) and has
 * time rank i: the permutation pi is the identity on the listed order.
 *
 * Four labels used (3..16 edges): the anchor is a 3-path.  anchor = {e1,
 * middle, e3} motif edge indices forces it (it must contain edge 0);
 * {-1,-1,-1} selects it by the rule of Alg. 5: among the 3-paths over the
 * four vertices that contain edge 0, the one whose sorted triple of ranks is
 * lexicographically smallest.
 *
 * Three labels used (2..16 edges): the anchor is a wedge (wedge sampling for
 * 3-vertex motifs): the base is edge 0, sampled with weight equal to the
 * number of possible second edges, and the second edge is the motif edge j
 * that shares one vertex s with the base, drawn uniformly from s's out-list
 * (if edge j leaves s; for s the base's source this is the paper's <+,>>
 * wedge) or in-list within (t, t + delta] of the base (closed: [t, t +
 * delta]).  {-1,-1,-1} takes the smallest such j; {j, 0, -1} (s the base's
 * source) or {-1, 0, j} (s its destination) forces one.
 */
typedef struct {
  int32_t num_edges;                 /* 2 or 3 .. TC_MAX_MOTIF_EDGES */
  int8_t src[TC_MAX_MOTIF_EDGES];
  int8_t dst[TC_MAX_MOTIF_EDGES];
  int32_t anchor[3];
  int32_t window;                    /* TC_WINDOW_STRICT or TC_WINDOW_CLOSED */
} tc_motif;

/* Result of a sampling run (Alg. 5). */
typedef struct {
  uint64_t W;          /* total path weight W_delta (Def. 6) */
  uint64_t k;          /* samples drawn */
  uint64_t sum_x;      /* sum over samples of X = CheckMotif(P) */
  uint64_t sum_x2_lo;  /* sum of X^2, low 64 bits */
  uint64_t sum_x2_hi;  /* sum of X^2, high 64 bits */
  uint64_t hits;       /* samples with X > 0 */
  uint64_t checked;    /* samples whose path (wedge) spans four (three) vertices with
                          the anchor's time order and span <= delta (reached the
                          list lookups) */
  double estimate;     /* C_hat = sum_x * W / k (exact integer division, then FP64) */
  double std_err;      /* W * sqrt(s^2 / k), s^2 the unbiased sample variance of X */
} tc_estimate;

typedef struct {
  int64_t n, m;        /* vertices, edges */
  int64_t num_pairs;   /* distinct (src, dst) pairs */
  int64_t t_min, t_max;
} tc_graph_info;

/* Arrays of a graph that tc_graph_copy can export (for inspection and tests). */
typedef enum {
  TC_ARRAY_OUT_OFF = 0,   /* uint32[n+1]   out-list offsets per vertex            */
  TC_ARRAY_OUT_EDGES = 1, /* {int32 src, int32 dst, int64 t}[m], canonical order  */
  TC_ARRAY_EDGE_PERM = 2, /* uint32[m]     canonical position -> input index      */
  TC_ARRAY_IN_OFF = 3,    /* uint32[n+1]   in-list offsets per vertex             */
  TC_ARRAY_IN_EDGES = 4,  /* {int32 src, int32 dst, int64 t}[m], in-list order      */
  TC_ARRAY_PAIR_OFF = 5,  /* uint32[n+1]   first pair index per source vertex      */
  TC_ARRAY_PAIR_DST = 6,  /* int32[P]      destination of each pair, by (src, dst) */
  TC_ARRAY_PAIR_EOFF = 7, /* uint32[P+1]   first pair-list position per pair       */
  TC_ARRAY_PAIR_T = 8,    /* int64[m]      times in pair order                     */
  TC_ARRAY_PAIR_EID = 9,  /* uint32[m]     pair position -> canonical position     */
  TC_ARRAY_IN_EID = 10    /* uint32[m]     in-list position -> canonical position  */
} tc_array;

/*
 * Build the time-sorted out-, in- and pair-lists of a temporal graph
 * (Sec. III: adjacency lists sorted by timestamp; Sec. III-B: the lists
 * L_{u,v} of all u->v edges).
 *   n          number of vertices; ids must lie in [0, n)
 *   m          number of edges (0 allowed)
 *   d_src, d_dst, d_t  device arrays of m entries in input order (borrowed)
 *   *out       receives the new graph; destroy it with tc_graph_destroy
 * Errors: TC_ERR_INVALID_ARG (sizes, null pointers, an id outside [0, n)),
 * TC_ERR_OOM, TC_ERR_CUDA.  Synchronises the stream.
 */
tc_status tc_build_temporal_csr(int64_t n, int64_t m, const int32_t* d_src, const int32_t* d_dst,
                                const int64_t* d_t, void* stream, tc_graph** out);

/* Free a graph (enqueued on the stream it was built on).  NULL is ignored. */
tc_status tc_graph_destroy(tc_graph* g);

/* Sizes and time range of a graph (host struct). */
tc_status tc_graph_info_get(const tc_graph* g, tc_graph_info* h_info);

/* Copy one internal array (tc_array) into caller device memory d_dst, whose
 * size must be at least the array's (listed above).  Enqueued on stream. */
tc_status tc_graph_copy(const tc_graph* g, int32_t which, void* d_dst, void* stream);

/*
 * Canonical edge order (Sec. III: out-lists sorted by time): d_perm[i]
 * receives the input index of the edge at canonical position i, as int64
 * (m entries, caller-owned device memory).  Every per-edge array of this
 * ABI (w, prefix, trace positions) is indexed in this order.  The same
 * permutation as uint32 is TC_ARRAY_EDGE_PERM of tc_graph_copy.
 * Errors: TC_ERR_INVALID_ARG (NULL graph or d_perm with m > 0), TC_ERR_CUDA.
 */
tc_status tc_graph_edge_order(const tc_graph* g, int64_t* d_perm, void* stream);

/*
 * Bytes of device memory a sampling index needs for graph g: a 256-byte
 * header, per canonical edge a 16-byte entry {uint32 lo1, uint32 d1,
 * uint32 lo3, uint32 d3} (both window ranges of Alg. 2: e1 lies at list
 * positions [lo1, lo1 + d1), e3 at [lo3, lo3 + d3)), and a guide table of
 * uint32 that maps equal slices of [0, W) to the first candidate edge of
 * the CDF search.  Independent of the motif and delta.
 */
tc_status tc_sample_index_bytes(const tc_graph* g, size_t* h_bytes);

/*
 * Path weights and their exact prefix sum (Claim 1, Alg. 1).  For every edge
 * e = (u, v, t) in canonical order, with the motif's anchor class
 * <alpha1, alpha3, beta1, beta3> (Def. 5):
 *   w_e = d^{alpha1}_u[window1(t)] * d^{alpha3}_v[window3(t)]
 * where the window is [t - delta, t) for beta = '<' and (t, t + delta] for
 * beta = '>' (closed at t with TC_WINDOW_CLOSED).
 *   d_w       optional uint64[m]; receives w_e (NULL: not returned)
 *   d_prefix  uint64[m+1]; prefix[0] = 0, prefix[i+1] = prefix[i] + w_i
 *   d_index   tc_sample_index_bytes(g) bytes, 256-byte aligned; receives the
 *             sampling index consumed by tc_sample_estimate
 *   h_W       optional; receives W = prefix[m] (synchronises the stream)
 * Errors: TC_ERR_INVALID_ARG, TC_ERR_UNSUPPORTED_MOTIF, TC_ERR_OVERFLOW (W
 * does not fit 64 bits; reported when h_W is requested), TC_ERR_CUDA.
 */
tc_status tc_path_weights(const tc_graph* g, const tc_motif* motif, int64_t delta, uint64_t* d_w,
                          uint64_t* d_prefix, void* d_index, uint64_t* h_W, void* stream);

/*
 * Draw k delta-centered 3-paths and count their motif completions
 * (Alg. 2, 3, 4, 5).  Sample s = sample_offset + i, i < k, uses Philox4x32-10
 * (Salmon et al., SC'11) with key (seed low, seed high) and counter
 * (s low, s high, draw, attempt); draw 0 picks the middle edge as the unique
 * e with prefix[e] <= r < prefix[e+1] for r uniform in [0, W) from words 0-1
 * of its block, and draw 1 picks the end edges uniformly in their windows, e1
 * from words 0-1 and e3 from words 2-3 of its block (Lemire's bounded draw
 * with rejection, each draw at most 64 attempts).  Each path contributes
 * X = prod over gaps of ListCount (Alg. 3, 4).
 *   d_prefix, d_index  as filled by tc_path_weights for the same graph,
 *                      motif and delta (checked on the device)
 *   h_out     receives the sums and the estimate (synchronises the stream)
 * Ranges [offset, offset + k) of one seed can be merged by adding the sums.
 * Errors: TC_ERR_INVALID_ARG, TC_ERR_OVERFLOW, TC_ERR_RNG_EXHAUSTED,
 * TC_ERR_CUDA.
 */
tc_status tc_sample_estimate(const tc_graph* g, const tc_motif* motif, int64_t delta,
                             const uint64_t* d_prefix, const void* d_index, uint64_t k, uint64_t seed,
                             uint64_t sample_offset, tc_estimate* h_out, void* stream);

/*
 * The estimate of Alg. 5 from exact sums: C_hat = sum_x * W / k by exact
 * 128-bit integer division, q + r / k in FP64, and its standard error
 * W * sqrt(s^2 / k) with s^2 = (sum_x2 - sum_x^2 / k) / (k - 1) in FP64
 * (NaN for k = 1; estimate and error 0 for k = 0 or W = 0).  The same
 * arithmetic tc_sample_estimate applies to one run; this entry point forms
 * it for sums added up over runs on disjoint sample-id ranges of one seed
 * (for example one range per GPU).  sum_x2 is 128 bits (lo, hi).  h_out
 * receives W, k and the sums as given, hits = checked = 0, the estimate and
 * its error.  Host only.  Errors: TC_ERR_INVALID_ARG (h_out NULL).
 */
tc_status tc_estimate_from_sums(uint64_t sum_x, uint64_t sum_x2_lo, uint64_t sum_x2_hi, uint64_t k, uint64_t W,
                                tc_estimate* h_out);

/*
 * Same sampling as tc_sample_estimate for `count` samples, writing per sample
 * (canonical middle edge, list position of e1, list position of e3, X) as 4
 * uint64 into d_trace[4*count].  e1 lies in the in-list (alpha1 = '-') or
 * out-list (alpha1 = '+') of the middle edge's source; e3 likewise for its
 * destination.  For inspection and parity tests.
 */
tc_status tc_sample_trace(const tc_graph* g, const tc_motif* motif, int64_t delta,
                          const uint64_t* d_prefix, const void* d_index, uint64_t count,
                          uint64_t seed, uint64_t sample_offset, uint64_t* d_trace, void* stream);

/*
 * Whole method from host arrays: copy the edges to the device, build the
 * lists, weights, prefix and index, draw k samples and return the estimate.
 * Device memory is taken and released inside the call.  h_src, h_dst, h_t
 * are host arrays of m entries (pinned memory makes the copies faster).
 */
tc_status tc_estimate_from_host(int64_t n, int64_t m, const int32_t* h_src, const int32_t* h_dst,
                                const int64_t* h_t, const tc_motif* motif, int64_t delta, uint64_t k,
                                uint64_t seed, tc_estimate* h_out, void* stream);

/*
 * Exact uint64 prefix sum of d_w (the same result as the d_prefix of
 * tc_path_weights for the same weights) that allocates no device memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc or cudaMallocAsync, for example code whose device
 * memory is owned by another allocator that reserved all of it up front, or
 * a process that runs under a hard memory budget in which a new allocation
 * may fail at any time.  The caller passes the weights and the output:
 *   d_w       uint64[m] device input
 *   d_prefix  uint64[m+1] device output, prefix[0] = 0, prefix[m] = W
 *   h_W       optional; receives W and reports overflow (synchronises)
 * Scratch (per-tile sums and an error word) lives in one static device array
 * of about 1 MiB that every GPU loading this library holds until the process
 * exits.  m may be at most TC_NOALLOC_MAX_EDGES; larger m returns
 * TC_ERR_INVALID_ARG.  Every call shares that array: calls whose work
 * overlaps on the GPU (different streams, or several host threads) race and
 * must be serialised by the caller.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) and keeps it for that
 * device's current context; the first call after a device reset (a new
 * context) looks it up again.  Make the first call on a device before any
 * stream capture.  Overflow of W is detected on the device and reported
 * only when h_W is requested.
 */
#define TC_NOALLOC_MAX_EDGES (1ull << 28)
tc_status tc_prefix_sum_noalloc(const uint64_t* d_w, uint64_t m, uint64_t* d_prefix, uint64_t* h_W,
                                void* stream);

/* Fill in the automatic anchor and report its class: h_anchor[3] = (e1,
 * middle, e3), h_class[4] = (alpha1, alpha3, beta1, beta3) with -1 for '-' /
 * '<' and +1 for '+' / '>'.  Host only. */
tc_status tc_motif_plan(const tc_motif* motif, int32_t* h_anchor, int32_t* h_class);

/*
 * Exact count by exhaustive path sum (the proof of Claim 2: every M-match
 * has exactly one anchor path, so the sum over all W delta-centered paths of
 * the anchor's class of CheckMotif equals C).  Path p in [0, W) is the
 * (p - prefix[e])-th pair (e1, e3) of its middle edge e, e1 major.  Cost
 * O(W) CheckMotif calls: exact counting for graphs whose W is at most some
 * 1e11.  h_out: sum_x = C, sum_x2 = sum of squares of the per-path counts
 * (so the exact variance of one sample is sum_x2 / W - (C / W)^2),
 * k = W (paths), hits = paths with a match, estimate = C as FP64, std_err = 0.
 * Synchronises the stream.
 */
tc_status tc_exact_count(const tc_graph* g, const tc_motif* motif, int64_t delta, const uint64_t* d_prefix,
                         const void* d_index, tc_estimate* h_out, void* stream);

/* ------------------------------------------------------------------------
 * Learned proposal.  The paper's estimator draws the middle edge with
 * probability w_e / W (Alg. 2).  Any proposal q_e = w_e h_e with integer
 * h_e >= 1 keeps it unbiased when each path is weighted by Q / h_e, with
 * Q = sum_e q_e (Claim 2's argument path by path).  Here h_e comes from a
 * small network g(e) in (0, 1) trained to predict whether a path through e
 * completes the motif: h_e = max(1, floor(scale (eps + g_e) + 1/2)).
 * The network: 12 features -> 64 -> 64 -> 1 with ReLU and a sigmoid output,
 * bf16 operands and FP32 accumulation; TC_MLP_PARAMS FP32 parameters laid out
 * as W1[64][16] (columns 12..15 unused, kept 0), b1[64], W2[64][64], b2[64],
 * W3[64], b3.
 * ------------------------------------------------------------------------ */
typedef struct tc_mlp tc_mlp;
#define TC_MLP_PARAMS 5313
#define TC_FEATURE_STRIDE 16 /* bf16 values per feature row (12 used) */
#define TC_PROPOSAL_MAX_H 4095

/* New network with weights U(-1/sqrt(fan_in), 1/sqrt(fan_in)) drawn from
 * Philox keyed by seed; device memory on the current device. */
tc_status tc_mlp_create(uint64_t seed, tc_mlp** out);
tc_status tc_mlp_destroy(tc_mlp* mlp);
/* Copy the FP32 parameters to / from host memory (TC_MLP_PARAMS floats);
 * setting them resets the optimizer state. */
tc_status tc_mlp_get_params(const tc_mlp* mlp, float* h_params);
tc_status tc_mlp_set_params(tc_mlp* mlp, const float* h_params);

/*
 * Per canonical edge e = (u, v, t) with w_e > 0, bf16 features (row stride
 * 16; columns 12..15 are set to zero here and filled by tc_sample_features),
 * each log1p of a count: 0 d1, 1 d3, 2 w_e (the anchor's windows, Claim 1),
 * 3..6 in- and out-degree of u, then of v, over [t - delta, t + delta],
 * 7 sigma_{u,v}[t - delta, t + delta], 8 sigma_{v,u}[t - delta, t + delta]
 * (Def. 3), 9 out-degree of u, 10 in-degree of v, 11 in-degree of u.
 * The row of an edge with w_e = 0 is all zero: such an edge is never drawn
 * and never an input of the network (tc_proposal_weights skips it).
 *   d_index  as filled by tc_path_weights for the same graph, motif, delta
 *   d_feat   uint16 (bf16 bits) [m][16] output
 */
tc_status tc_edge_features(const tc_graph* g, const tc_motif* motif, int64_t delta, const void* d_index,
                           uint16_t* d_feat, void* stream);

/*
 * Sample-statistics features, columns 12..15 of every row of d_feat: draws
 * n_samples paths with the plain sampler (sample ids sample_offset ..
 * sample_offset + n_samples - 1 of seed, as tc_sample_trace) and, with the
 * time bucket b(t) = (floor(t / D) - floor(t_min / D)) mod 2^32 for D =
 * max(delta, 1) and t_min the graph's earliest time, the keys K1 = (u, v),
 * K2 = (u, b(t)), K3 = (v, b(t)) of an edge: n_K = the samples whose middle
 * edge has key K, s_K = the sum of their X^2, prior = sum X^2 / n_samples.
 * Columns: log1p((s_K + prior) / (n_K + 1)) for K1, K2, K3, then
 * log1p(n_K1), in bf16, for the rows of edges with w_e > 0 (the other rows
 * and columns are left as they are).  Draw
 * these samples disjoint from those tc_mlp_train uses (another seed or id
 * range), so that no training path sees its own outcome.  d_feat must be
 * 16-byte aligned.  Synchronises the stream.  Errors as tc_sample_estimate.
 */
tc_status tc_sample_features(const tc_graph* g, const tc_motif* motif, int64_t delta, const uint64_t* d_prefix,
                             const void* d_index, uint64_t n_samples, uint64_t seed, uint64_t sample_offset,
                             uint16_t* d_feat, void* stream);

/* Logits z of rows d_rows[i] (or i when d_rows is NULL) of d_feat into
 * d_logits[n] (FP32); g = sigmoid(z).  Synchronises the stream.
 * TC_ERR_TIMEOUT: a bounded wait of the tcgen05 inference kernel for its
 * tensor-core MMAs gave up (the logits are then incomplete). */
tc_status tc_mlp_forward(const tc_mlp* mlp, const uint16_t* d_feat, const uint32_t* d_rows, uint64_t n,
                         float* d_logits, void* stream);

/* Gradient over n rows of the mean closure loss of g = sigmoid(z) against
 * the closure counts d_labels (y >= 0): y softplus(-z) = -y log g for y > 0,
 * softplus(z) = -log(1 - g) for y = 0 -- the binary cross-entropy when every
 * y is 0 or 1, and minimised at g = E[X] / (E[X] + P(X = 0)) -- into
 * d_grad[TC_MLP_PARAMS] (FP32, overwritten); h_loss (optional) receives the
 * mean loss.  Synchronises the stream. */
tc_status tc_mlp_grad(const tc_mlp* mlp, const uint16_t* d_feat, const uint32_t* d_rows, const float* d_labels,
                      uint64_t n, float* d_grad, float* h_loss, void* stream);

/*
 * Train on n_samples paths drawn by the plain sampler (tc_sample_trace with
 * seed, ids 0..n_samples-1): input the 16 features of the middle edge,
 * label the closure count X, loss as tc_mlp_grad.  One pass of Adam (lr,
 * betas 0.9 / 0.999) in batches of `batch`.
 * h_losses (optional) receives the mean loss of the first and last batch.
 * Synchronises the stream.
 */
tc_status tc_mlp_train(tc_mlp* mlp, const tc_graph* g, const tc_motif* motif, int64_t delta,
                       const uint64_t* d_prefix, const void* d_index, const uint16_t* d_feat,
                       uint64_t n_samples, uint64_t seed, uint32_t batch, float lr, float* h_losses,
                       void* stream);

/*
 * Training objectives (the paper has no learned part; the estimator whose
 * variance the second objective targets is that of Claim 2 with the
 * proposal's weights).  TC_OBJECTIVE_CLOSURE: the closure loss above.
 * TC_OBJECTIVE_BCE: the binary cross-entropy of g against the closure
 * outcome 1[X > 0] (the closure loss on labels clipped to 1).
 * TC_OBJECTIVE_VARIANCE: the estimator's own variance -- with h = eps + g
 * for the proposal's eps, a sample drawn from q ~ w h has second moment
 * proportional to Q * sum over paths of X^2 / h, estimated over a batch of
 * plain samples by mean(h) * mean(X^2 / h); minimising it drives h towards
 * sqrt(E[X^2 | e]), the variance-optimal per-edge proposal.
 * tc_mlp_grad_ex / tc_mlp_train_ex: as tc_mlp_grad / tc_mlp_train with the
 * objective and eps (> 0 for the variance objective, else
 * TC_ERR_INVALID_ARG, as is an unknown objective); d_labels (grad) and the
 * sampled paths (train) carry the closure counts X.  For the variance
 * objective h_loss and h_losses receive the objective's value over the
 * rows or batch (not a per-row mean).  Device buffers are borrowed; the
 * calls allocate their scratch from the library's pool on the stream.
 */
#define TC_OBJECTIVE_CLOSURE 0
#define TC_OBJECTIVE_VARIANCE 1
#define TC_OBJECTIVE_BCE 2
tc_status tc_mlp_grad_ex(const tc_mlp* mlp, const uint16_t* d_feat, const uint32_t* d_rows, const float* d_labels,
                         uint64_t n, int32_t objective, float eps, float* d_grad, float* h_loss, void* stream);
tc_status tc_mlp_train_ex(tc_mlp* mlp, const tc_graph* g, const tc_motif* motif, int64_t delta,
                          const uint64_t* d_prefix, const void* d_index, const uint16_t* d_feat,
                          uint64_t n_samples, uint64_t seed, uint32_t batch, float lr, int32_t objective,
                          float eps, float* h_losses, void* stream);

/* Bytes of a proposal index (header and guide table) for graph g. */
tc_status tc_proposal_index_bytes(const tc_graph* g, size_t* h_bytes);

/*
 * Proposal weights: d_h[m] (uint16) = max(1, floor(scale (eps + g_e) + 1/2))
 * for every edge with w_e > 0, and 1 for an edge with w_e = 0 (it is never
 * drawn, so the network is not evaluated on it: only the rows of edges with
 * w_e > 0 of d_feat are read), d_qprefix[m+1] the exact prefix sum of
 * w_e h_e (w_e from d_prefix), and the
 * proposal's sampling index d_qindex (tc_proposal_index_bytes, 256-byte
 * aligned).  scale >= 1, eps >= 0, scale (1 + eps) + 1 <= TC_PROPOSAL_MAX_H.
 * h_Q (optional) receives Q = d_qprefix[m] and reports overflow.
 */
tc_status tc_proposal_weights(const tc_mlp* mlp, const tc_graph* g, const tc_motif* motif, int64_t delta,
                              const uint64_t* d_prefix, const uint16_t* d_feat, float eps, uint32_t scale,
                              uint16_t* d_h, uint64_t* d_qprefix, void* d_qindex, uint64_t* h_Q,
                              void* stream);

/*
 * Sampling with the proposal: sample s draws r uniform in [0, Q) (draw 0)
 * and the middle edge e with qprefix[e] <= r < qprefix[e+1]; e1, e3 and X as
 * in tc_sample_estimate.  The exact per-h sums B_h = sum X and B2_h = sum X^2
 * give C_hat = Q / k * sum over ascending h of B_h / h (FP64 on the host).
 *   d_index   the plain index of the same graph, motif and delta (records)
 *   h_bins    optional host array [3 * (TC_PROPOSAL_MAX_H + 1)]: per h,
 *             B_h, B2_h low 64 bits, B2_h high 64 bits
 *   d_trace   optional [4 * k] as in tc_sample_trace
 * h_out->W receives Q.  Synchronises the stream.
 */
tc_status tc_sample_estimate_q(const tc_graph* g, const tc_motif* motif, int64_t delta, const void* d_index,
                               const uint16_t* d_h, const uint64_t* d_qprefix, const void* d_qindex,
                               uint64_t k, uint64_t seed, uint64_t sample_offset, tc_estimate* h_out,
                               uint64_t* h_bins, uint64_t* d_trace, void* stream);

/*
 * Batched queries.  A batch is a fixed list of queries, each a motif and
 * window on a built graph with k samples (sample ids sample_offset ..
 * sample_offset + k - 1 of seed), answered together: every run recomputes
 * the path weights, prefix and index once per distinct (graph, anchor class,
 * window kind, delta), puts every query's samples in key order, and samples
 * all queries in one persistent launch whose blocks take (query, tile) work
 * items from a counter.  With use_graph, that whole sequence is captured
 * once into a CUDA graph at creation and each run replays it.  The sums of
 * each query are bit-identical to tc_sample_estimate on the same query (the
 * samples are keyed by id and the sums are integers).
 *
 * Graphs are borrowed: they must outlive the batch.  The batch owns device
 * memory for each distinct weights key (prefix and index, 8 (m + 1) plus
 * tc_sample_index_bytes) and 4 k bytes of sample order per query with
 * k >= 65536; k may be at most 2^40.
 */
typedef struct {
  const tc_graph* graph;
  tc_motif motif;
  int64_t delta;
  uint64_t k, seed, sample_offset;
} tc_query;

typedef struct {
  int32_t block_size; /* threads per block of the batch launch: 128, 256 or 512; 0 = autotune */
  uint32_t tile;      /* samples per work item, a multiple of block_size; 0 = autotune */
  int32_t use_graph;  /* nonzero: capture one CUDA graph at creation and replay it */
  int32_t reserved;
} tc_batch_options;

typedef struct tc_batch tc_batch;

/* Validates the queries (as tc_sample_estimate would), allocates the batch's
 * memory and, when block_size or tile is 0, times every candidate
 * (block size 128/256/512 x tile 2048/8192/32768) on one full run and keeps
 * the fastest.  opts may be NULL (autotune, use_graph = 1).  Synchronises
 * stream.  Errors: TC_ERR_INVALID_ARG for a NULL or bad argument,
 * TC_ERR_UNSUPPORTED_MOTIF, TC_ERR_OOM, TC_ERR_CUDA. */
tc_status tc_batch_create(const tc_query* h_queries, int64_t nq, const tc_batch_options* opts, void* stream,
                          tc_batch** out);

/* One run: h_out[nq] receives every query's estimate (as
 * tc_sample_estimate).  Synchronises stream.  A query whose weights
 * overflow or whose samples hit a device error makes the call return that
 * status; h_out is still filled for the others. */
tc_status tc_batch_run(tc_batch* b, tc_estimate* h_out, void* stream);

/* The batch's chosen launch shape, the kernels one run launches, the
 * device bytes the batch holds and its number of distinct weights keys
 * (any pointer may be NULL). */
tc_status tc_batch_info(const tc_batch* b, tc_batch_options* h_opts, uint64_t* h_launches_per_run,
                        uint64_t* h_device_bytes, uint64_t* h_weight_slots);

/* Device time of the last completed run, from CUDA events recorded inside
 * the sequence: the whole run (weights, key sorts, sampling) and the
 * persistent sampling launch alone, in milliseconds.  Call after
 * tc_batch_run has returned. */
tc_status tc_batch_timing(const tc_batch* b, float* h_run_ms, float* h_sampling_ms);

tc_status tc_batch_destroy(tc_batch* b);

/* Number of kernels this library has launched in this process so far
 * (a diagnostic for counting launches around a region). */
uint64_t tc_kernel_launches(void);

/* Diagnostic timing on this thread: while enabled, tc_sample_estimate,
 * tc_sample_trace and tc_sample_estimate_q record CUDA events around their
 * sampling launches (the key-order sort excluded), and tc_last_sampler_ms
 * returns the device time of those launches in the last such call, in
 * milliseconds (0 when timing was off). */
tc_status tc_set_timing(int32_t enabled);
float tc_last_sampler_ms(void);

/* Device time, in milliseconds, of one phase of the last call on this
 * thread that ran it while timing was enabled (tc_set_timing): the sum over
 * CUDA events recorded around the phase's launches on the call's stream (0
 * when timing was off or the phase did not run).  Phases: the path weights
 * and their exact prefix sum (Claim 1, Alg. 1) of tc_path_weights; the
 * guide table of its sampling index (or of tc_proposal_weights' index); the
 * key-order sort of the sample ids of a sampling call; its sampling
 * launches (Alg. 2-4, the same as tc_last_sampler_ms); the network, h, q
 * and q-prefix of tc_proposal_weights. */
#define TC_PHASE_WEIGHTS 0
#define TC_PHASE_INDEX 1
#define TC_PHASE_ORDER 2
#define TC_PHASE_SAMPLE 3
#define TC_PHASE_PROPOSAL 4
float tc_last_phase_ms(int32_t phase);

/* Which kernel runs the network's inference (tc_mlp_forward, the logits of
 * the variance objective, tc_proposal_weights), for the whole process:
 * kind 0 = warp-level mma.sync tiles with register-resident weights,
 * 1 = tcgen05 MMAs into TMEM accumulators issued by one thread per block;
 * kind < 0 only queries.  Both compute the same network in the same
 * precisions (bf16 operands, FP32 accumulation); sums may differ in
 * rounding order.  The default is the build's TC_MLP_TCGEN05 (1: tcgen05),
 * overridden by the environment variable of the same name ("0" or "1").  Returns the kind
 * in effect after the call; -1 for an unknown kind (nothing changes). */
int32_t tc_mlp_kernel(int32_t kind);

/* Message of the last failed call on this thread ("" if none). */
const char* tc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TC_H */
