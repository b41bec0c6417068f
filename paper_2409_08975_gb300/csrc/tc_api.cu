// C ABI of the library (include/tc.h): argument checks, the motif compiler,
// object lifetime, error reporting and the host arithmetic of the estimate.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "tc_internal.cuh"

namespace tc {

static thread_local std::string t_err;
static std::atomic<uint64_t> g_launches{0};

void note_launches(unsigned count) { g_launches.fetch_add(count, std::memory_order_relaxed); }

cudaError_t pool_malloc(void** p, size_t bytes, cudaStream_t st) {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaMallocAsync(p, bytes, st);
  cudaMemPool_t pool;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
      cudaMemPoolProps props;
      std::memset(&props, 0, sizeof(props));
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      e = cudaMemPoolCreate(&pools[dev], &props);
      if (e != cudaSuccess) {
        pools[dev] = nullptr;
        return e;
      }
      uint64_t keep = UINT64_MAX;
      cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
    }
    pool = pools[dev];
  }
  return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

tc_status set_error(tc_status st, const std::string& msg) {
  t_err = msg;
  return st;
}

tc_status cuda_status(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return set_error(TC_ERR_OOM, std::string(what) + ": " + cudaGetErrorString(e));
  }
  return set_error(TC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

tc_status device_status(uint32_t bits, const char* what) {
  std::string w(what);
  if (bits & kErrIndexMismatch)
    return set_error(TC_ERR_INVALID_ARG, w + ": sampling index was built for another graph, motif or delta");
  if (bits & kErrBadId) return set_error(TC_ERR_INVALID_ARG, w + ": vertex id outside [0, n)");
  if (bits & kErrOverflow) return set_error(TC_ERR_OVERFLOW, w + ": a 64-bit count overflowed");
  if (bits & kErrRng) return set_error(TC_ERR_RNG_EXHAUSTED, w + ": 64 rejected draws in a row");
  if (bits & kErrBounds) return set_error(TC_ERR_BOUNDS, w + ": device index check failed");
  if (bits & kErrTimeout) return set_error(TC_ERR_TIMEOUT, w + ": a bounded device wait gave up");
  return TC_OK;
}

// Anchor rule (Alg. 5): the 3-path over the four vertices that contains
// edge 0 and whose sorted ranks are lexicographically smallest; its class
// <alpha1, alpha3, beta1, beta3> (Def. 5); the non-anchor edges per gap.
// Wedge anchor of a 3-vertex motif: base = edge 0, second edge = the
// smallest j sharing exactly one vertex with it (or the forced one).
static tc_status compile_wedge(const tc_motif* M, Plan* P, std::string* why) {
  const int r = M->num_edges;
  const bool forced = !(M->anchor[0] == -1 && M->anchor[1] == -1 && M->anchor[2] == -1);
  const int A = M->src[0], B = M->dst[0];
  int best = -1;
  for (int j = 1; j < r && best < 0; j++) {
    const int x = M->src[j], y = M->dst[j];
    const int shared = (x == A || y == A) + (x == B || y == B);
    if (shared != 1) continue;
    const bool at_src = x == A || y == A;
    if (forced && !(at_src ? (M->anchor[0] == j && M->anchor[1] == 0 && M->anchor[2] == -1)
                           : (M->anchor[0] == -1 && M->anchor[1] == 0 && M->anchor[2] == j)))
      continue;
    best = j;
  }
  if (best < 0) {
    *why = forced ? "forced anchor is not a wedge on edge 0" : "motif has no wedge that contains edge 0";
    return TC_ERR_UNSUPPORTED_MOTIF;
  }
  const int x = M->src[best], y = M->dst[best];
  const bool at_src = x == A || y == A;
  const int s = at_src ? A : B;
  const int third = x == s ? y : x;
  const int alpha = x == s ? +1 : -1;  // the second edge leaves s: out-list
  std::memset(P, 0, sizeof(*P));
  P->r = r;
  P->mid = 0;
  P->closed = M->window == TC_WINDOW_CLOSED;
  P->wedge = at_src ? 1 : 2;
  P->lab[1] = A;
  P->lab[2] = B;
  if (at_src) {
    P->e1 = best;
    P->e3 = -1;
    P->alpha1 = alpha;
    P->beta1 = +1;
    P->lab[0] = third;
    P->lab[3] = -1;
  } else {
    P->e1 = -1;
    P->e3 = best;
    P->alpha3 = alpha;
    P->beta3 = +1;
    P->lab[0] = -1;
    P->lab[3] = third;
  }
  P->rk[0] = 0;
  P->rk[1] = best;
  P->rk[2] = r;
  int role[4] = {-1, -1, -1, -1};  // label -> position in (u', u, v, v')
  role[A] = 1;
  role[B] = 2;
  role[third] = at_src ? 0 : 3;
  for (int gp = 0; gp < 2; gp++) {
    const int lo = gp == 0 ? 0 : best, hi = gp == 0 ? best : r;
    for (int f = lo + 1; f < hi; f++) {
      P->gx[gp][P->ngap[gp]] = (int8_t)role[M->src[f]];
      P->gy[gp][P->ngap[gp]] = (int8_t)role[M->dst[f]];
      P->ngap[gp]++;
    }
  }
  return TC_OK;
}

tc_status compile_plan(const tc_motif* M, Plan* P, std::string* why) {
  const int r = M->num_edges;
  if (r < 2 || r > TC_MAX_MOTIF_EDGES) {
    *why = "motif needs 2..16 edges (3..16 on four vertices)";
    return TC_ERR_INVALID_ARG;
  }
  if (M->window != TC_WINDOW_STRICT && M->window != TC_WINDOW_CLOSED) {
    *why = "window must be TC_WINDOW_STRICT or TC_WINDOW_CLOSED";
    return TC_ERR_INVALID_ARG;
  }
  int used = 0;
  for (int i = 0; i < r; i++) {
    const int x = M->src[i], y = M->dst[i];
    if (x < 0 || x > 3 || y < 0 || y > 3 || x == y) {
      *why = "motif edges must join two distinct labels in 0..3";
      return TC_ERR_INVALID_ARG;
    }
    used |= (1 << x) | (1 << y);
  }
  const int nlab = __builtin_popcount((unsigned)used);
  if (nlab == 3) return compile_wedge(M, P, why);
  if (nlab != 4 || r < 3) {
    *why = "motif must use three vertex labels (2..16 edges) or four (3..16 edges)";
    return TC_ERR_INVALID_ARG;
  }
  const bool forced = !(M->anchor[0] == -1 && M->anchor[1] == -1 && M->anchor[2] == -1);
  bool found = false;
  int best_e1 = -1, best_mid = -1, best_e3 = -1, best_lab[4] = {0, 0, 0, 0};
  // triples {0, j, k} in lexicographic order: the first valid one is the anchor
  for (int j = 1; j < r && !found; j++)
    for (int k = j + 1; k < r && !found; k++) {
      const int trip[3] = {0, j, k};
      for (int mi = 0; mi < 3 && !found; mi++) {
        const int mid = trip[mi];
        const int oa = trip[(mi + 1) % 3], ob = trip[(mi + 2) % 3];
        const int U = M->src[mid], V = M->dst[mid];
        for (int swap = 0; swap < 2 && !found; swap++) {
          const int e1 = swap ? ob : oa, e3 = swap ? oa : ob;
          const int a0 = M->src[e1], a1 = M->dst[e1], c0 = M->src[e3], c1 = M->dst[e3];
          const bool e1_at_u = (a0 == U || a1 == U) && a0 != V && a1 != V;
          const bool e3_at_v = (c0 == V || c1 == V) && c0 != U && c1 != U;
          if (!e1_at_u || !e3_at_v) continue;
          const int Up = a1 == U ? a0 : a1, Vp = c0 == V ? c1 : c0;
          if (Up == Vp) continue;
          if (forced && !(M->anchor[0] == e1 && M->anchor[1] == mid && M->anchor[2] == e3)) continue;
          found = true;
          best_e1 = e1;
          best_mid = mid;
          best_e3 = e3;
          best_lab[0] = Up;
          best_lab[1] = U;
          best_lab[2] = V;
          best_lab[3] = Vp;
        }
      }
    }
  if (!found) {
    *why = forced ? "forced anchor is not a 3-path over four vertices containing edge 0"
                  : "motif has no 3-path over its four vertices that contains edge 0";
    return TC_ERR_UNSUPPORTED_MOTIF;
  }
  std::memset(P, 0, sizeof(*P));
  P->r = r;
  P->e1 = best_e1;
  P->mid = best_mid;
  P->e3 = best_e3;
  const int U = M->src[best_mid], V = M->dst[best_mid];
  P->alpha1 = M->dst[best_e1] == U ? -1 : +1;  // e1 enters u: in-list
  P->alpha3 = M->src[best_e3] == V ? +1 : -1;  // e3 leaves v: out-list
  P->beta1 = best_e1 < best_mid ? -1 : +1;
  P->beta3 = best_e3 < best_mid ? -1 : +1;
  P->closed = M->window == TC_WINDOW_CLOSED;
  for (int i = 0; i < 4; i++) P->lab[i] = best_lab[i];
  int rk[3] = {best_e1, best_mid, best_e3};
  for (int a = 0; a < 3; a++)
    for (int b = a + 1; b < 3; b++)
      if (rk[b] < rk[a]) { int x = rk[a]; rk[a] = rk[b]; rk[b] = x; }
  for (int a = 0; a < 3; a++) P->rk[a] = rk[a];
  int role[4];  // label -> position in (u', u, v, v')
  for (int i = 0; i < 4; i++) role[best_lab[i]] = i;
  for (int gp = 0; gp < 3; gp++) {
    const int lo = rk[gp], hi = gp < 2 ? rk[gp + 1] : r;
    for (int f = lo + 1; f < hi; f++) {
      P->gx[gp][P->ngap[gp]] = (int8_t)role[M->src[f]];
      P->gy[gp][P->ngap[gp]] = (int8_t)role[M->dst[f]];
      P->ngap[gp]++;
    }
  }
  return TC_OK;
}

static std::atomic<uint64_t> g_next_graph_id{1};

static cudaStream_t S(void* stream) { return (cudaStream_t)stream; }

static tc_status check_graph(const tc_graph* g) {
  if (!g) return set_error(TC_ERR_INVALID_ARG, "graph is NULL");
  return TC_OK;
}

static tc_status plan_of(const tc_motif* motif, Plan* p) {
  if (!motif) return set_error(TC_ERR_INVALID_ARG, "motif is NULL");
  std::string why;
  tc_status s = compile_plan(motif, p, &why);
  if (s != TC_OK) return set_error(s, why);
  return TC_OK;
}

tc_status compile_plan_checked(const tc_motif* motif, Plan* p) { return plan_of(motif, p); }

static void free_graph_arrays(tc_graph* g) {
  void* ps[] = {g->out_off, g->out_e,  g->perm,     g->in_off,  g->in_e,    g->in_eid,  g->pair_off, g->pair_dst,
                g->pair_eoff, g->pair_t, g->pair_eid, g->pair_hash, g->out_t32, g->in_t32, g->pair_t32, g->x_in,
                g->x_out, g->out2in, g->r_in, g->r_out, g->r_o2i, g->r_self};
  for (void* p : ps)
    if (p) cudaFree(p);
}

// Host form of C_hat = sum_x * W / k (Alg. 5): exact 128-bit product and
// division, then q + r / k in FP64; standard error W * sqrt(s^2 / k).
void finish_estimate(tc_estimate* o) {
  o->estimate = 0.0;
  o->std_err = 0.0;
  if (o->k == 0 || o->W == 0) return;
  const unsigned __int128 num = (unsigned __int128)o->sum_x * o->W;
  const unsigned __int128 q = num / o->k, r = num % o->k;
  o->estimate = (double)q + (double)(uint64_t)r / (double)o->k;
  if (o->k < 2) {
    o->std_err = NAN;
    return;
  }
  const unsigned __int128 x2 = ((unsigned __int128)o->sum_x2_hi << 64) | o->sum_x2_lo;
  const double sx = (double)o->sum_x, sx2 = (double)x2, kf = (double)o->k;
  double s2 = (sx2 - sx * sx / kf) / (kf - 1.0);
  if (s2 < 0.0) s2 = 0.0;
  o->std_err = (double)o->W * std::sqrt(s2 / kf);
}

}  // namespace tc

using namespace tc;

extern "C" {

const char* tc_last_error(void) { return t_err.c_str(); }

uint64_t tc_kernel_launches(void) { return g_launches.load(); }

tc_status tc_set_timing(int32_t enabled) {
  set_timing(enabled != 0);
  return TC_OK;
}

float tc_last_sampler_ms(void) { return last_sampler_ms(); }

float tc_last_phase_ms(int32_t phase) { return last_phase_ms(phase); }

int32_t tc_mlp_kernel(int32_t kind) { return mlp_kernel(kind); }

tc_status tc_motif_plan(const tc_motif* motif, int32_t* h_anchor, int32_t* h_class) {
  Plan p;
  TC_TRY(plan_of(motif, &p));
  if (h_anchor) {
    h_anchor[0] = p.e1;
    h_anchor[1] = p.mid;
    h_anchor[2] = p.e3;
  }
  if (h_class) {
    h_class[0] = p.alpha1;
    h_class[1] = p.alpha3;
    h_class[2] = p.beta1;
    h_class[3] = p.beta3;
  }
  return TC_OK;
}

tc_status tc_build_temporal_csr(int64_t n, int64_t m, const int32_t* d_src, const int32_t* d_dst,
                                const int64_t* d_t, void* stream, tc_graph** out) {
  if (!out) return set_error(TC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n < 1 || n >= (1ll << 31)) return set_error(TC_ERR_INVALID_ARG, "n must lie in [1, 2^31)");
  if (m < 0 || m >= (int64_t)0xFFFFFFFFll) return set_error(TC_ERR_INVALID_ARG, "m must lie in [0, 2^32 - 1)");
  if (m > 0 && (!d_src || !d_dst || !d_t)) return set_error(TC_ERR_INVALID_ARG, "edge arrays are NULL");
  tc_graph* g = new (std::nothrow) tc_graph;
  if (!g) return set_error(TC_ERR_OOM, "host allocation failed");
  std::memset(g, 0, sizeof(*g));
  cudaGetDevice(&g->device);
  g->id = g_next_graph_id.fetch_add(1);
  tc_status s = build_graph(n, m, d_src, d_dst, d_t, S(stream), g);
  if (s != TC_OK) {
    cudaStreamSynchronize(S(stream));
    free_graph_arrays(g);
    delete g;
    return s;
  }
  *out = g;
  return TC_OK;
}

tc_status tc_graph_destroy(tc_graph* g) {
  if (!g) return TC_OK;
  free_graph_arrays(g);  // cudaFree waits for work still using the arrays
  delete g;
  return TC_OK;
}

tc_status tc_graph_info_get(const tc_graph* g, tc_graph_info* h_info) {
  TC_TRY(check_graph(g));
  if (!h_info) return set_error(TC_ERR_INVALID_ARG, "info is NULL");
  h_info->n = g->n;
  h_info->m = g->m;
  h_info->num_pairs = g->P;
  h_info->t_min = g->tmin;
  h_info->t_max = g->tmax;
  return TC_OK;
}

tc_status tc_graph_copy(const tc_graph* g, int32_t which, void* d_dst, void* stream) {
  TC_TRY(check_graph(g));
  if (!d_dst) return set_error(TC_ERR_INVALID_ARG, "destination is NULL");
  const void* src = nullptr;
  size_t bytes = 0;
  const size_t n1 = (size_t)g->n + 1, m = (size_t)g->m, P = (size_t)g->P;
  switch (which) {
    case TC_ARRAY_OUT_OFF: src = g->out_off; bytes = 4 * n1; break;
    case TC_ARRAY_OUT_EDGES: src = g->out_e; bytes = 16 * m; break;
    case TC_ARRAY_EDGE_PERM: src = g->perm; bytes = 4 * m; break;
    case TC_ARRAY_IN_OFF: src = g->in_off; bytes = 4 * n1; break;
    case TC_ARRAY_IN_EDGES: src = g->in_e; bytes = 16 * m; break;
    case TC_ARRAY_IN_EID: src = g->in_eid; bytes = 4 * m; break;
    case TC_ARRAY_PAIR_OFF: src = g->pair_off; bytes = 4 * n1; break;
    case TC_ARRAY_PAIR_DST: src = g->pair_dst; bytes = 4 * P; break;
    case TC_ARRAY_PAIR_EOFF: src = g->pair_eoff; bytes = 4 * (P + 1); break;
    case TC_ARRAY_PAIR_T: src = g->pair_t; bytes = 8 * m; break;
    case TC_ARRAY_PAIR_EID: src = g->pair_eid; bytes = 4 * m; break;
    default: return set_error(TC_ERR_INVALID_ARG, "unknown array");
  }
  if (bytes) TC_CUDA(cudaMemcpyAsync(d_dst, src, bytes, cudaMemcpyDeviceToDevice, S(stream)));
  return TC_OK;
}

tc_status tc_graph_edge_order(const tc_graph* g, int64_t* d_perm, void* stream) {
  TC_TRY(check_graph(g));
  if (!d_perm && g->m > 0) return set_error(TC_ERR_INVALID_ARG, "d_perm is NULL");
  return launch_widen_u32(g->perm, (uint64_t)g->m, d_perm, S(stream));
}

tc_status tc_estimate_from_sums(uint64_t sum_x, uint64_t sum_x2_lo, uint64_t sum_x2_hi, uint64_t k, uint64_t W,
                                tc_estimate* h_out) {
  if (!h_out) return set_error(TC_ERR_INVALID_ARG, "out is NULL");
  std::memset(h_out, 0, sizeof(*h_out));
  h_out->W = W;
  h_out->k = k;
  h_out->sum_x = sum_x;
  h_out->sum_x2_lo = sum_x2_lo;
  h_out->sum_x2_hi = sum_x2_hi;
  finish_estimate(h_out);
  return TC_OK;
}

tc_status tc_sample_index_bytes(const tc_graph* g, size_t* h_bytes) {
  TC_TRY(check_graph(g));
  if (!h_bytes) return set_error(TC_ERR_INVALID_ARG, "bytes is NULL");
  *h_bytes = index_bytes((uint64_t)g->m);
  return TC_OK;
}

tc_status tc_path_weights(const tc_graph* g, const tc_motif* motif, int64_t delta, uint64_t* d_w,
                          uint64_t* d_prefix, void* d_index, uint64_t* h_W, void* stream) {
  TC_TRY(check_graph(g));
  Plan plan;
  TC_TRY(plan_of(motif, &plan));
  if (delta < 0) return set_error(TC_ERR_INVALID_ARG, "delta must be >= 0");
  if (!d_prefix || !d_index) return set_error(TC_ERR_INVALID_ARG, "prefix or index is NULL");
  if (((uintptr_t)d_index & 255) != 0) return set_error(TC_ERR_INVALID_ARG, "index must be 256-byte aligned");
  cudaStream_t st = S(stream);
  const uint64_t m = (uint64_t)g->m;
  char* scratch = nullptr;  // error word, then the scan's tile states
  tc_status s = TC_OK;
  cudaError_t e = pool_malloc(&scratch, 256 + weights_scan_scratch_bytes(m), st);
  if (e != cudaSuccess) return cuda_status(e, "pool_malloc(weights scratch)");
  uint32_t* err = (uint32_t*)scratch;
  e = cudaMemsetAsync(err, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) s = cuda_status(e, "cudaMemsetAsync");
  char* idx = (char*)d_index;
  EdgeWin* win = (EdgeWin*)(idx + kIndexHeaderBytes);
  PhaseTimer wt(TC_PHASE_WEIGHTS, st), it(TC_PHASE_INDEX, st);
  wt.start();
  if (s == TC_OK) s = launch_weights_scan(g, plan, delta, win, d_prefix, d_w, scratch + 256, err, st);
  wt.stop();
  it.start();
  if (s == TC_OK) s = launch_guide(g, plan, delta, d_prefix, d_index, err, st);
  it.stop();
  uint32_t h_err = 0;
  if (s == TC_OK && h_W) {
    e = cudaMemcpyAsync(h_W, d_prefix + m, sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_status(e, "tc_path_weights");
  }
  cudaFreeAsync(scratch, st);
  if (s == TC_OK && h_err) s = device_status(h_err, "tc_path_weights");
  return s;
}

static tc_status sample_common(const tc_graph* g, const tc_motif* motif, int64_t delta, const uint64_t* d_prefix,
                               const void* d_index, uint64_t k, uint64_t seed, uint64_t offset, uint64_t* d_trace,
                               tc_estimate* h_out, void* stream, const char* what) {
  TC_TRY(check_graph(g));
  Plan plan;
  TC_TRY(plan_of(motif, &plan));
  if (delta < 0) return set_error(TC_ERR_INVALID_ARG, "delta must be >= 0");
  if (!d_prefix || !d_index) return set_error(TC_ERR_INVALID_ARG, "prefix or index is NULL");
  if (((uintptr_t)d_index & 255) != 0) return set_error(TC_ERR_INVALID_ARG, "index must be 256-byte aligned");
  cudaStream_t st = S(stream);
  SampleSums* sums = nullptr;
  TC_CUDA(pool_malloc(&sums, sizeof(SampleSums), st));
  tc_status s = TC_OK;
  cudaError_t e = cudaMemsetAsync(sums, 0, sizeof(SampleSums), st);
  if (e != cudaSuccess) s = cuda_status(e, "cudaMemsetAsync");
  if (s == TC_OK) s = launch_sampler(g, plan, delta, d_prefix, d_index, k, seed, offset, d_trace, sums, st);
  SampleSums h;
  std::memset(&h, 0, sizeof(h));
  if (s == TC_OK) {
    e = cudaMemcpyAsync(&h, sums, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_status(e, what);
  }
  cudaFreeAsync(sums, st);
  if (s == TC_OK && h.err) s = device_status(h.err, what);
  if (s == TC_OK && h_out) {
    h_out->W = h.W;
    h_out->k = k;
    h_out->sum_x = h.sum_x;
    h_out->sum_x2_lo = h.sum_x2_lo;
    h_out->sum_x2_hi = h.sum_x2_hi;
    h_out->hits = h.hits;
    h_out->checked = h.checked;
    finish_estimate(h_out);
  }
  return s;
}

tc_status tc_sample_estimate(const tc_graph* g, const tc_motif* motif, int64_t delta, const uint64_t* d_prefix,
                             const void* d_index, uint64_t k, uint64_t seed, uint64_t sample_offset,
                             tc_estimate* h_out, void* stream) {
  if (!h_out) return set_error(TC_ERR_INVALID_ARG, "out is NULL");
  return sample_common(g, motif, delta, d_prefix, d_index, k, seed, sample_offset, nullptr, h_out, stream,
                       "tc_sample_estimate");
}

tc_status tc_sample_trace(const tc_graph* g, const tc_motif* motif, int64_t delta, const uint64_t* d_prefix,
                          const void* d_index, uint64_t count, uint64_t seed, uint64_t sample_offset,
                          uint64_t* d_trace, void* stream) {
  if (!d_trace && count) return set_error(TC_ERR_INVALID_ARG, "trace is NULL");
  return sample_common(g, motif, delta, d_prefix, d_index, count, seed, sample_offset, d_trace, nullptr, stream,
                       "tc_sample_trace");
}

tc_status tc_estimate_from_host(int64_t n, int64_t m, const int32_t* h_src, const int32_t* h_dst,
                                const int64_t* h_t, const tc_motif* motif, int64_t delta, uint64_t k,
                                uint64_t seed, tc_estimate* h_out, void* stream) {
  if (!h_out) return set_error(TC_ERR_INVALID_ARG, "out is NULL");
  if (m < 0 || m >= (int64_t)0xFFFFFFFFll) return set_error(TC_ERR_INVALID_ARG, "m must lie in [0, 2^32 - 1)");
  if (m > 0 && (!h_src || !h_dst || !h_t)) return set_error(TC_ERR_INVALID_ARG, "edge arrays are NULL");
  Plan plan;
  TC_TRY(plan_of(motif, &plan));
  cudaStream_t st = S(stream);
  const size_t M = (size_t)(m ? m : 1);
  int32_t *d_src = nullptr, *d_dst = nullptr;
  int64_t* d_t = nullptr;
  uint64_t* d_prefix = nullptr;
  void* d_index = nullptr;
  tc_graph* g = nullptr;
  tc_status s = TC_OK;
  cudaError_t e = pool_malloc(&d_src, 4 * M, st);
  if (e == cudaSuccess) e = pool_malloc(&d_dst, 4 * M, st);
  if (e == cudaSuccess) e = pool_malloc(&d_t, 8 * M, st);
  if (e == cudaSuccess && m) e = cudaMemcpyAsync(d_src, h_src, 4 * (size_t)m, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && m) e = cudaMemcpyAsync(d_dst, h_dst, 4 * (size_t)m, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && m) e = cudaMemcpyAsync(d_t, h_t, 8 * (size_t)m, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) s = cuda_status(e, "tc_estimate_from_host");
  if (s == TC_OK) s = tc_build_temporal_csr(n, m, d_src, d_dst, d_t, stream, &g);
  if (d_src) cudaFreeAsync(d_src, st);
  if (d_dst) cudaFreeAsync(d_dst, st);
  if (d_t) cudaFreeAsync(d_t, st);
  size_t ib = 0;
  if (s == TC_OK) s = tc_sample_index_bytes(g, &ib);
  if (s == TC_OK) {
    e = pool_malloc(&d_prefix, 8 * ((size_t)m + 1), st);
    if (e == cudaSuccess) e = pool_malloc(&d_index, ib, st);
    if (e != cudaSuccess) s = cuda_status(e, "cudaMallocAsync");
  }
  uint64_t W = 0;
  if (s == TC_OK) s = tc_path_weights(g, motif, delta, nullptr, d_prefix, d_index, &W, stream);
  if (s == TC_OK) s = tc_sample_estimate(g, motif, delta, d_prefix, d_index, k, seed, 0, h_out, stream);
  if (d_prefix) cudaFreeAsync(d_prefix, st);
  if (d_index) cudaFreeAsync(d_index, st);
  cudaStreamSynchronize(st);
  if (g) tc_graph_destroy(g);
  return s;
}

tc_status tc_exact_count(const tc_graph* g, const tc_motif* motif, int64_t delta, const uint64_t* d_prefix,
                         const void* d_index, tc_estimate* h_out, void* stream) {
  TC_TRY(check_graph(g));
  Plan plan;
  TC_TRY(plan_of(motif, &plan));
  if (delta < 0) return set_error(TC_ERR_INVALID_ARG, "delta must be >= 0");
  if (!d_prefix || !d_index || !h_out) return set_error(TC_ERR_INVALID_ARG, "NULL argument");
  if (((uintptr_t)d_index & 255) != 0) return set_error(TC_ERR_INVALID_ARG, "index must be 256-byte aligned");
  cudaStream_t st = S(stream);
  uint64_t W = 0;
  TC_CUDA(cudaMemcpyAsync(&W, d_prefix + g->m, sizeof(W), cudaMemcpyDeviceToHost, st));
  TC_CUDA(cudaStreamSynchronize(st));
  SampleSums* sums = nullptr;
  TC_CUDA(pool_malloc(&sums, sizeof(SampleSums), st));
  tc_status s = TC_OK;
  cudaError_t e = cudaMemsetAsync(sums, 0, sizeof(SampleSums), st);
  if (e != cudaSuccess) s = cuda_status(e, "memset");
  if (s == TC_OK && W) s = launch_path_sum(g, plan, delta, d_prefix, d_index, W, sums, st);
  SampleSums h;
  std::memset(&h, 0, sizeof(h));
  if (s == TC_OK) {
    e = cudaMemcpyAsync(&h, sums, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_status(e, "tc_exact_count");
  }
  cudaFreeAsync(sums, st);
  if (s == TC_OK && h.err) s = device_status(h.err, "tc_exact_count");
  if (s != TC_OK) return s;
  h_out->W = W;
  h_out->k = W;
  h_out->sum_x = h.sum_x;
  h_out->sum_x2_lo = h.sum_x2_lo;
  h_out->sum_x2_hi = h.sum_x2_hi;
  h_out->hits = h.hits;
  h_out->checked = h.checked;
  h_out->estimate = (double)h.sum_x;
  h_out->std_err = 0.0;
  return TC_OK;
}

// ---------------------------------------------------------------------------
// Learned proposal.

static tc_status check_index_header(const tc_graph* g, const Plan& plan, int64_t delta, const void* d_index,
                                    cudaStream_t st) {
  IndexHeader h;
  TC_CUDA(cudaMemcpyAsync(&h, d_index, sizeof(h), cudaMemcpyDeviceToHost, st));
  TC_CUDA(cudaStreamSynchronize(st));
  const bool ok = h.magic == kIndexMagic && h.graph_id == g->id && h.delta == delta && h.cls[0] == plan.alpha1 &&
                  h.cls[1] == plan.alpha3 && h.cls[2] == plan.beta1 && h.cls[3] == plan.beta3 &&
                  h.closed == plan.closed && h.anchor[0] == plan.e1 && h.anchor[1] == plan.mid &&
                  h.anchor[2] == plan.e3;
  if (!ok) return set_error(TC_ERR_INVALID_ARG, "index was built for another graph, motif or delta");
  if (h.status) return device_status(h.status, "index");
  return TC_OK;
}

tc_status tc_mlp_create(uint64_t seed, tc_mlp** out) {
  if (!out) return set_error(TC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  return mlp_create(seed, out);
}

tc_status tc_mlp_destroy(tc_mlp* mlp) {
  if (mlp) mlp_destroy(mlp);
  return TC_OK;
}

tc_status tc_mlp_get_params(const tc_mlp* mlp, float* h_params) {
  if (!mlp || !h_params) return set_error(TC_ERR_INVALID_ARG, "mlp or params is NULL");
  return mlp_get_params(mlp, h_params);
}

tc_status tc_mlp_set_params(tc_mlp* mlp, const float* h_params) {
  if (!mlp || !h_params) return set_error(TC_ERR_INVALID_ARG, "mlp or params is NULL");
  return mlp_set_params(mlp, h_params);
}

tc_status tc_edge_features(const tc_graph* g, const tc_motif* motif, int64_t delta, const void* d_index,
                           uint16_t* d_feat, void* stream) {
  TC_TRY(check_graph(g));
  Plan plan;
  TC_TRY(plan_of(motif, &plan));
  if (delta < 0) return set_error(TC_ERR_INVALID_ARG, "delta must be >= 0");
  if (!d_index || !d_feat) return set_error(TC_ERR_INVALID_ARG, "index or features is NULL");
  cudaStream_t st = S(stream);
  TC_TRY(check_index_header(g, plan, delta, d_index, st));
  const EdgeWin* win = (const EdgeWin*)((const char*)d_index + kIndexHeaderBytes);
  return launch_features(g, win, delta, d_feat, st);
}

tc_status tc_sample_features(const tc_graph* g, const tc_motif* motif, int64_t delta, const uint64_t* d_prefix,
                             const void* d_index, uint64_t n_samples, uint64_t seed, uint64_t sample_offset,
                             uint16_t* d_feat, void* stream) {
  TC_TRY(check_graph(g));
  Plan plan;
  TC_TRY(plan_of(motif, &plan));
  if (delta < 0) return set_error(TC_ERR_INVALID_ARG, "delta must be >= 0");
  if (!d_prefix || !d_index || !d_feat) return set_error(TC_ERR_INVALID_ARG, "NULL argument");
  if (((uintptr_t)d_feat & 15) != 0) return set_error(TC_ERR_INVALID_ARG, "features must be 16-byte aligned");
  cudaStream_t st = S(stream);
  uint64_t* trace = nullptr;
  SampleSums* sums = nullptr;
  uint32_t* err = nullptr;
  tc_status s = TC_OK;
  cudaError_t e = pool_malloc(&trace, 32 * (n_samples ? n_samples : 1), st);
  if (e == cudaSuccess) e = pool_malloc(&sums, sizeof(SampleSums) + 16, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(sums, 0, sizeof(SampleSums) + 16, st);
  if (e != cudaSuccess) s = cuda_status(e, "tc_sample_features allocation");
  if (s == TC_OK) err = (uint32_t*)(sums + 1);
  if (s == TC_OK && n_samples)
    s = launch_sampler(g, plan, delta, d_prefix, d_index, n_samples, seed, sample_offset, trace, sums, st);
  if (s == TC_OK) s = launch_sample_features(g, d_prefix, trace, n_samples, delta, d_feat, err, st);
  SampleSums hs;
  uint32_t herr = 0;
  std::memset(&hs, 0, sizeof(hs));
  if (s == TC_OK) {
    e = cudaMemcpyAsync(&hs, sums, sizeof(hs), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_status(e, "tc_sample_features");
  }
  if (trace) cudaFreeAsync(trace, st);
  if (sums) cudaFreeAsync(sums, st);
  if (s == TC_OK && (hs.err | herr)) s = device_status(hs.err | herr, "tc_sample_features");
  return s;
}

tc_status tc_mlp_forward(const tc_mlp* mlp, const uint16_t* d_feat, const uint32_t* d_rows, uint64_t n,
                         float* d_logits, void* stream) {
  if (!mlp || (n && (!d_feat || !d_logits))) return set_error(TC_ERR_INVALID_ARG, "NULL argument");
  TC_TRY(launch_mlp_forward(mlp, d_feat, d_rows, n, d_logits, S(stream)));
  return mlp_check_error(mlp, S(stream), "tc_mlp_forward");
}

tc_status tc_mlp_grad(const tc_mlp* mlp, const uint16_t* d_feat, const uint32_t* d_rows, const float* d_labels,
                      uint64_t n, float* d_grad, float* h_loss, void* stream) {
  return tc_mlp_grad_ex(mlp, d_feat, d_rows, d_labels, n, TC_OBJECTIVE_CLOSURE, 0.f, d_grad, h_loss, stream);
}

tc_status tc_mlp_grad_ex(const tc_mlp* mlp, const uint16_t* d_feat, const uint32_t* d_rows, const float* d_labels,
                         uint64_t n, int32_t objective, float eps, float* d_grad, float* h_loss, void* stream) {
  if (!mlp || !d_grad || (n && (!d_feat || !d_labels))) return set_error(TC_ERR_INVALID_ARG, "NULL argument");
  if (objective != TC_OBJECTIVE_CLOSURE && objective != TC_OBJECTIVE_VARIANCE && objective != TC_OBJECTIVE_BCE)
    return set_error(TC_ERR_INVALID_ARG, "unknown training objective");
  if (objective == TC_OBJECTIVE_VARIANCE && !(eps > 0.f)) return set_error(TC_ERR_INVALID_ARG, "eps must be > 0");
  const bool var = objective == TC_OBJECTIVE_VARIANCE, bce = objective == TC_OBJECTIVE_BCE;
  cudaStream_t st = S(stream);
  // loss, spare float, then (variance) logits and dloss/dz or (BCE) the clipped labels
  float* buf = nullptr;
  TC_CUDA(pool_malloc(&buf, sizeof(float) * (2 + (var ? 2 * (n ? n : 1) : (bce ? (n ? n : 1) : 0))), st));
  float* loss = buf;
  tc_status s = TC_OK;
  cudaError_t e = cudaMemsetAsync(d_grad, 0, sizeof(float) * TC_MLP_PARAMS, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, sizeof(float) * 2, st);
  if (e != cudaSuccess) s = cuda_status(e, "memset");
  if (s == TC_OK) {
    if (var) {
      s = launch_variance_grad(mlp, d_feat, d_rows, d_labels, n, eps, d_grad, loss, buf + 2, buf + 2 + n, buf + 1, st);
    } else if (bce) {
      s = launch_clip_labels(d_labels, n, buf + 2, st);
      if (s == TC_OK) s = launch_mlp_grad(mlp, d_feat, d_rows, buf + 2, n, d_grad, loss, st);
    } else {
      s = launch_mlp_grad(mlp, d_feat, d_rows, d_labels, n, d_grad, loss, st);
    }
  }
  float hl = 0.f;
  if (s == TC_OK) {
    e = cudaMemcpyAsync(&hl, loss, sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_status(e, "tc_mlp_grad");
  }
  cudaFreeAsync(buf, st);
  if (s == TC_OK && var) s = mlp_check_error(mlp, st, "tc_mlp_grad_ex");
  if (s == TC_OK && h_loss) *h_loss = var ? hl : (n ? hl / (float)n : 0.f);
  return s;
}

tc_status tc_mlp_train(tc_mlp* mlp, const tc_graph* g, const tc_motif* motif, int64_t delta,
                       const uint64_t* d_prefix, const void* d_index, const uint16_t* d_feat,
                       uint64_t n_samples, uint64_t seed, uint32_t batch, float lr, float* h_losses,
                       void* stream) {
  return tc_mlp_train_ex(mlp, g, motif, delta, d_prefix, d_index, d_feat, n_samples, seed, batch, lr,
                         TC_OBJECTIVE_CLOSURE, 0.f, h_losses, stream);
}

tc_status tc_mlp_train_ex(tc_mlp* mlp, const tc_graph* g, const tc_motif* motif, int64_t delta,
                          const uint64_t* d_prefix, const void* d_index, const uint16_t* d_feat,
                          uint64_t n_samples, uint64_t seed, uint32_t batch, float lr, int32_t objective,
                          float eps, float* h_losses, void* stream) {
  if (objective != TC_OBJECTIVE_CLOSURE && objective != TC_OBJECTIVE_VARIANCE && objective != TC_OBJECTIVE_BCE)
    return set_error(TC_ERR_INVALID_ARG, "unknown training objective");
  if (objective == TC_OBJECTIVE_VARIANCE && !(eps > 0.f)) return set_error(TC_ERR_INVALID_ARG, "eps must be > 0");
  TC_TRY(check_graph(g));
  Plan plan;
  TC_TRY(plan_of(motif, &plan));
  if (!mlp || !d_prefix || !d_index || !d_feat) return set_error(TC_ERR_INVALID_ARG, "NULL argument");
  if (batch == 0 || !(lr > 0.f)) return set_error(TC_ERR_INVALID_ARG, "batch must be > 0 and lr > 0");
  if (n_samples == 0) return TC_OK;
  cudaStream_t st = S(stream);
  const uint64_t steps = (n_samples + batch - 1) / batch;
  uint64_t* trace = nullptr;
  uint32_t* rows = nullptr;
  float* labels = nullptr;
  float* losses = nullptr;
  float* zbuf = nullptr;  // variance objective: logits, dloss/dz and a spare float of a batch
  SampleSums* sums = nullptr;
  tc_status s = TC_OK;
  const bool var = objective == TC_OBJECTIVE_VARIANCE;
  const uint64_t bmax = batch < n_samples ? batch : n_samples;
  cudaError_t e = pool_malloc(&trace, 32 * n_samples, st);
  if (e == cudaSuccess && var) e = pool_malloc(&zbuf, sizeof(float) * (2 * bmax + 1), st);
  if (e == cudaSuccess) e = pool_malloc(&rows, 4 * n_samples, st);
  if (e == cudaSuccess) e = pool_malloc(&labels, 4 * n_samples, st);
  if (e == cudaSuccess) e = pool_malloc(&losses, sizeof(float) * steps, st);
  if (e == cudaSuccess) e = pool_malloc(&sums, sizeof(SampleSums), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(sums, 0, sizeof(SampleSums), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(losses, 0, sizeof(float) * steps, st);
  if (e != cudaSuccess) s = cuda_status(e, "tc_mlp_train allocation");
  // training paths from the plain sampler: rows = middle edges, labels = closure counts X
  if (s == TC_OK) s = launch_sampler(g, plan, delta, d_prefix, d_index, n_samples, seed, 0, trace, sums, st);
  if (s == TC_OK) s = launch_trace_to_rows(trace, n_samples, rows, labels, st, objective == TC_OBJECTIVE_BCE);
  for (uint64_t b = 0; b < steps && s == TC_OK; b++) {
    const uint64_t lo = b * batch, nb = (n_samples - lo) < batch ? (n_samples - lo) : batch;
    if (var)
      s = launch_variance_grad(mlp, d_feat, rows + lo, labels + lo, nb, eps, mlp_grad_buffer(mlp), losses + b, zbuf,
                               zbuf + bmax, zbuf + 2 * bmax, st);
    else
      s = launch_mlp_grad(mlp, d_feat, rows + lo, labels + lo, nb, mlp_grad_buffer(mlp), losses + b, st);
    if (s == TC_OK) s = mlp_adam(mlp, lr, st);
  }
  SampleSums hs;
  float first = 0.f, last = 0.f;
  if (s == TC_OK) {
    e = cudaMemcpyAsync(&hs, sums, sizeof(hs), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&first, losses, sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&last, losses + steps - 1, sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_status(e, "tc_mlp_train");
  }
  for (void* p : {(void*)trace, (void*)rows, (void*)labels, (void*)losses, (void*)sums, (void*)zbuf})
    if (p) cudaFreeAsync(p, st);
  if (s == TC_OK && hs.err) s = device_status(hs.err, "tc_mlp_train");
  if (s == TC_OK && var) s = mlp_check_error(mlp, st, "tc_mlp_train");
  if (s == TC_OK && h_losses) {
    const uint64_t last_n = n_samples - (steps - 1) * (uint64_t)batch;
    h_losses[0] = var ? first : first / (float)(batch < n_samples ? batch : n_samples);
    h_losses[1] = var ? last : last / (float)last_n;
  }
  return s;
}

tc_status tc_proposal_index_bytes(const tc_graph* g, size_t* h_bytes) {
  TC_TRY(check_graph(g));
  if (!h_bytes) return set_error(TC_ERR_INVALID_ARG, "bytes is NULL");
  *h_bytes = proposal_index_bytes((uint64_t)g->m);
  return TC_OK;
}

tc_status tc_proposal_weights(const tc_mlp* mlp, const tc_graph* g, const tc_motif* motif, int64_t delta,
                              const uint64_t* d_prefix, const uint16_t* d_feat, float eps, uint32_t scale,
                              uint16_t* d_h, uint64_t* d_qprefix, void* d_qindex, uint64_t* h_Q,
                              void* stream) {
  TC_TRY(check_graph(g));
  Plan plan;
  TC_TRY(plan_of(motif, &plan));
  if (!mlp || !d_prefix || !d_feat || !d_h || !d_qprefix || !d_qindex)
    return set_error(TC_ERR_INVALID_ARG, "NULL argument");
  if (((uintptr_t)d_qindex & 255) != 0) return set_error(TC_ERR_INVALID_ARG, "index must be 256-byte aligned");
  if (scale < 1 || !(eps >= 0.f) || (double)scale * (1.0 + eps) + 1.0 > TC_PROPOSAL_MAX_H)
    return set_error(TC_ERR_INVALID_ARG, "need scale >= 1, eps >= 0 and scale (1 + eps) + 1 <= 4095");
  cudaStream_t st = S(stream);
  const uint64_t m = (uint64_t)g->m;
  char* scratch = nullptr;  // error word, then the scan's tile states
  tc_status s = TC_OK;
  cudaError_t e = pool_malloc(&scratch, 256 + proposal_scan_scratch_bytes(m), st);
  if (e != cudaSuccess) return cuda_status(e, "tc_proposal_weights allocation");
  uint32_t* err = (uint32_t*)scratch;
  e = cudaMemsetAsync(err, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) s = cuda_status(e, "tc_proposal_weights allocation");
  PhaseTimer pt(TC_PHASE_PROPOSAL, st), it(TC_PHASE_INDEX, st);
  pt.start();
  if (s == TC_OK)
    s = launch_proposal_scan(mlp, d_feat, d_prefix, m, eps, (float)scale, d_h, d_qprefix,
                             (uint32_t*)((char*)d_qindex + kProposalRangeOffset), scratch + 256, err, st);
  pt.stop();
  it.start();
  if (s == TC_OK)
    s = launch_guide_at(g, plan, delta, d_qprefix, (IndexHeader*)d_qindex,
                        (uint32_t*)((char*)d_qindex + kIndexHeaderBytes), err, st);
  it.stop();
  uint32_t h_err = 0;
  if (s == TC_OK && h_Q) {
    e = cudaMemcpyAsync(h_Q, d_qprefix + m, sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_status(e, "tc_proposal_weights");
  }
  cudaFreeAsync(scratch, st);
  if (s == TC_OK && h_err) s = device_status(h_err, "tc_proposal_weights");
  return s;
}

tc_status tc_sample_estimate_q(const tc_graph* g, const tc_motif* motif, int64_t delta, const void* d_index,
                               const uint16_t* d_h, const uint64_t* d_qprefix, const void* d_qindex,
                               uint64_t k, uint64_t seed, uint64_t sample_offset, tc_estimate* h_out,
                               uint64_t* h_bins, uint64_t* d_trace, void* stream) {
  TC_TRY(check_graph(g));
  Plan plan;
  TC_TRY(plan_of(motif, &plan));
  if (!d_index || !d_h || !d_qprefix || !d_qindex || !h_out) return set_error(TC_ERR_INVALID_ARG, "NULL argument");
  if ((((uintptr_t)d_index) | ((uintptr_t)d_qindex)) & 255)
    return set_error(TC_ERR_INVALID_ARG, "indexes must be 256-byte aligned");
  cudaStream_t st = S(stream);
  const size_t nbins = 3 * (size_t)(TC_PROPOSAL_MAX_H + 1);
  unsigned long long* bins = nullptr;
  SampleSums* sums = nullptr;
  tc_status s = TC_OK;
  cudaError_t e = pool_malloc(&bins, 8 * nbins, st);
  if (e == cudaSuccess) e = pool_malloc(&sums, sizeof(SampleSums), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(bins, 0, 8 * nbins, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(sums, 0, sizeof(SampleSums), st);
  if (e != cudaSuccess) s = cuda_status(e, "tc_sample_estimate_q allocation");
  if (s == TC_OK)
    s = launch_sampler(g, plan, delta, d_qprefix, d_index, k, seed, sample_offset, d_trace, sums, st, d_qindex, d_h,
                       bins);
  std::vector<uint64_t> hb(nbins);
  SampleSums hs;
  std::memset(&hs, 0, sizeof(hs));
  if (s == TC_OK) {
    e = cudaMemcpyAsync(hb.data(), bins, 8 * nbins, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, sums, sizeof(hs), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_status(e, "tc_sample_estimate_q");
  }
  if (bins) cudaFreeAsync(bins, st);
  if (sums) cudaFreeAsync(sums, st);
  if (s == TC_OK && hs.err) s = device_status(hs.err, "tc_sample_estimate_q");
  if (s != TC_OK) return s;
  const uint64_t Q = hs.W;
  h_out->W = Q;
  h_out->k = k;
  h_out->sum_x = hs.sum_x;
  h_out->sum_x2_lo = hs.sum_x2_lo;
  h_out->sum_x2_hi = hs.sum_x2_hi;
  h_out->hits = hs.hits;
  h_out->checked = hs.checked;
  // C_hat = Q / k * sum over ascending h of B_h / h; SE from sum Y and sum Y^2
  double s1 = 0.0, s2 = 0.0;
  for (int hv = 1; hv <= TC_PROPOSAL_MAX_H; hv++) {
    const uint64_t b = hb[3 * hv];
    const unsigned __int128 b2 = ((unsigned __int128)hb[3 * hv + 2] << 64) | hb[3 * hv + 1];
    if (!b && !b2) continue;
    const double h = (double)hv;
    s1 += (double)b / h;
    s2 += (double)b2 / (h * h);
  }
  h_out->estimate = 0.0;
  h_out->std_err = 0.0;
  if (k && Q) {
    const double Qf = (double)Q, kf = (double)k;
    h_out->estimate = Qf / kf * s1;
    if (k >= 2) {
      const double sy = Qf * s1, sy2 = Qf * Qf * s2;
      double var = (sy2 - sy * sy / kf) / (kf - 1.0);
      if (var < 0.0) var = 0.0;
      h_out->std_err = std::sqrt(var / kf);
    } else {
      h_out->std_err = NAN;
    }
  }
  if (h_bins) std::memcpy(h_bins, hb.data(), 8 * nbins);
  return TC_OK;
}

}  // extern "C"
