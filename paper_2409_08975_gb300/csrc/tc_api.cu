// C ABI of the library (include/tc.h): argument checks, the motif compiler,
// object lifetime, error reporting and the host arithmetic of the estimate.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "tc_internal.cuh"

namespace tc {

static thread_local std::string t_err;
static std::atomic<uint64_t> g_launches{0};

void note_launches(unsigned count) { g_launches.fetch_add(count, std::memory_order_relaxed); }

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
  return TC_OK;
}

// Anchor rule (Alg. 5): the 3-path over the four vertices that contains
// edge 0 and whose sorted ranks are lexicographically smallest; its class
// <alpha1, alpha3, beta1, beta3> (Def. 5); the non-anchor edges per gap.
tc_status compile_plan(const tc_motif* M, Plan* P, std::string* why) {
  const int r = M->num_edges;
  if (r < 3 || r > TC_MAX_MOTIF_EDGES) {
    *why = "motif needs 3..16 edges";
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
  if (used != 0xF) {
    *why = "motif must use all four vertex labels";
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

static void free_graph_arrays(tc_graph* g) {
  void* ps[] = {g->out_off, g->out_e, g->perm, g->in_off, g->in_e, g->in_eid, g->pair_off,
                g->pair_dst, g->pair_eoff, g->pair_t, g->pair_eid, g->pair_hash};
  for (void* p : ps)
    if (p) cudaFree(p);
}

// Host form of C_hat = sum_x * W / k (Alg. 5): exact 128-bit product and
// division, then q + r / k in FP64; standard error W * sqrt(s^2 / k).
static void finish_estimate(tc_estimate* o) {
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
  uint64_t* w = d_w;
  uint32_t* err = nullptr;
  tc_status s = TC_OK;
  if (!w) {
    cudaError_t e = cudaMallocAsync(&w, sizeof(uint64_t) * (m ? m : 1), st);
    if (e != cudaSuccess) return cuda_status(e, "cudaMallocAsync(w)");
  }
  cudaError_t e = cudaMallocAsync(&err, sizeof(uint32_t), st);
  if (e != cudaSuccess) s = cuda_status(e, "cudaMallocAsync(err)");
  if (s == TC_OK) {
    e = cudaMemsetAsync(err, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) s = cuda_status(e, "cudaMemsetAsync");
  }
  char* idx = (char*)d_index;
  EdgeRec* rec = (EdgeRec*)(idx + kIndexHeaderBytes);
  if (s == TC_OK) s = launch_weights(g, plan, delta, rec, w, st);
  if (s == TC_OK) s = scan_u64(w, d_prefix, m, err, st);
  if (s == TC_OK) s = launch_guide(g, plan, delta, d_prefix, d_index, err, st);
  uint32_t h_err = 0;
  if (s == TC_OK && h_W) {
    e = cudaMemcpyAsync(h_W, d_prefix + m, sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_status(e, "tc_path_weights");
  }
  if (err) cudaFreeAsync(err, st);
  if (!d_w && w) cudaFreeAsync(w, st);
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
  TC_CUDA(cudaMallocAsync(&sums, sizeof(SampleSums), st));
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
                             const void* d_index, const uint16_t* d_h, uint64_t k, uint64_t seed,
                             uint64_t sample_offset, tc_estimate* h_out, void* stream) {
  if (d_h) return set_error(TC_ERR_INVALID_ARG, "d_h is reserved; pass NULL");
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
  cudaError_t e = cudaMallocAsync(&d_src, 4 * M, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&d_dst, 4 * M, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&d_t, 8 * M, st);
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
    e = cudaMallocAsync(&d_prefix, 8 * ((size_t)m + 1), st);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_index, ib, st);
    if (e != cudaSuccess) s = cuda_status(e, "cudaMallocAsync");
  }
  uint64_t W = 0;
  if (s == TC_OK) s = tc_path_weights(g, motif, delta, nullptr, d_prefix, d_index, &W, stream);
  if (s == TC_OK) s = tc_sample_estimate(g, motif, delta, d_prefix, d_index, nullptr, k, seed, 0, h_out, stream);
  if (d_prefix) cudaFreeAsync(d_prefix, st);
  if (d_index) cudaFreeAsync(d_index, st);
  cudaStreamSynchronize(st);
  if (g) tc_graph_destroy(g);
  return s;
}

}  // extern "C"
