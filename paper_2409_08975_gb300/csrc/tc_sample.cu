// Path weights (Claim 1, Alg. 1), the guide table of the CDF search, and the
// sampler with CheckMotif / ListCount and the reduction of X (Alg. 2-5).
#include <cuda_runtime.h>

#include "tc_internal.cuh"

namespace tc {

// ---------------------------------------------------------------------------
// Weights: one thread per canonical edge e = (u, v, t).  The window of u's
// alpha1 list and of v's alpha3 list are found by binary search on time
// (Alg. 1: four searches per edge); w_e = d1 * d3 (Claim 1).

__global__ void __launch_bounds__(256) k_weights(const OutEdge* __restrict__ out_e,
                                                 const uint32_t* __restrict__ out_off,
                                                 const InEdge* __restrict__ in_e,
                                                 const uint32_t* __restrict__ in_off, uint32_t m, Plan plan,
                                                 int64_t delta, EdgeRec* __restrict__ rec,
                                                 uint64_t* __restrict__ w) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    const OutEdge e = out_e[i];
    uint32_t lo1, hi1, lo3, hi3;
    window_range(out_e, out_off, in_e, in_off, plan.alpha1, plan.beta1, plan.closed, e.src, e.t, delta, &lo1,
                 &hi1);
    window_range(out_e, out_off, in_e, in_off, plan.alpha3, plan.beta3, plan.closed, e.dst, e.t, delta, &lo3,
                 &hi3);
    EdgeRec r;
    r.u = e.src;
    r.v = e.dst;
    r.t = e.t;
    r.lo1 = lo1;
    r.d1 = hi1 - lo1;
    r.lo3 = lo3;
    r.d3 = hi3 - lo3;
    rec[i] = r;
    w[i] = (uint64_t)r.d1 * (uint64_t)r.d3;
  }
}

tc_status launch_weights(const tc_graph* g, const Plan& plan, int64_t delta, EdgeRec* rec, uint64_t* w,
                         cudaStream_t st) {
  const uint32_t m = (uint32_t)g->m;
  if (m == 0) return TC_OK;
  unsigned blocks = (m + 255) / 256;
  k_weights<<<blocks, 256, 0, st>>>(g->out_e, g->out_off, g->in_e, g->in_off, m, plan, delta, rec, w);
  TC_LAUNCHED(1);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

// ---------------------------------------------------------------------------
// Index layout: [header 256 B][EdgeRec m][guide uint32 (2^gbits + 1)].

int guide_bits(uint64_t m) {
  int b = 0;
  while (b < 32 && (1ull << b) < m) b++;
  return b;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t index_bytes(uint64_t m) {
  return kIndexHeaderBytes + align256(sizeof(EdgeRec) * m) + sizeof(uint32_t) * ((1ull << guide_bits(m)) + 1);
}

struct IndexView {
  IndexHeader* hdr;
  EdgeRec* rec;
  uint32_t* guide;
};

static IndexView index_view(void* index, uint64_t m) {
  char* p = (char*)index;
  IndexView v;
  v.hdr = (IndexHeader*)p;
  v.rec = (EdgeRec*)(p + kIndexHeaderBytes);
  v.guide = (uint32_t*)(p + kIndexHeaderBytes + align256(sizeof(EdgeRec) * m));
  return v;
}

// Guide table: bucket b covers r in [b << shift, (b + 1) << shift); guide[b]
// is the largest i < m with prefix[i] <= b << shift, the first candidate of
// the CDF search for any r in the bucket; guide[nb] = m - 1.  Each block
// first bounds its buckets' answers, then each thread searches that range.
__global__ void __launch_bounds__(256) k_guide(const uint64_t* __restrict__ prefix, uint32_t m, int gbits,
                                               uint32_t* __restrict__ guide, IndexHeader* hdr, Plan plan,
                                               int64_t delta, uint64_t graph_id, const uint32_t* err) {
  const uint64_t W = prefix[m];
  const int wbits = W ? 64 - __clzll(W - 1) : 0;
  const uint32_t shift = wbits > gbits ? (uint32_t)(wbits - gbits) : 0u;
  const uint32_t nb = W ? (uint32_t)(((W - 1) >> shift) + 1) : 0u;
  auto largest_le = [&](uint64_t x, uint32_t lo, uint32_t hi) {  // in [lo, hi], prefix[lo] <= x
    while (lo < hi) {
      const uint32_t mid = lo + ((hi - lo + 1) >> 1);
      if (prefix[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
  };
  __shared__ uint32_t s_lo, s_hi;
  const uint64_t b0 = (uint64_t)blockIdx.x * blockDim.x;
  if (b0 >= nb) {
    if (b0 == nb && threadIdx.x == 0 && m) guide[nb] = m - 1;
  } else {
    if (threadIdx.x == 0) {
      const uint64_t blast = min((uint64_t)nb - 1, b0 + blockDim.x - 1);
      s_lo = largest_le(b0 << shift, 0, m - 1);
      s_hi = largest_le(blast << shift, s_lo, m - 1);
    }
    __syncthreads();
    const uint64_t b = b0 + threadIdx.x;
    if (b < nb) guide[b] = largest_le(b << shift, s_lo, s_hi);
    if (b == nb && m) guide[nb] = m - 1;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    IndexHeader h;
    h.magic = kIndexMagic;
    h.W = W;
    h.m = m;
    h.shift = shift;
    h.nb = nb;
    h.cls[0] = plan.alpha1;
    h.cls[1] = plan.alpha3;
    h.cls[2] = plan.beta1;
    h.cls[3] = plan.beta3;
    h.closed = plan.closed;
    h.anchor[0] = plan.e1;
    h.anchor[1] = plan.mid;
    h.anchor[2] = plan.e3;
    h.delta = delta;
    h.graph_id = graph_id;
    h.status = err ? *err : 0u;
    *hdr = h;
  }
}

tc_status launch_guide(const tc_graph* g, const Plan& plan, int64_t delta, const uint64_t* prefix, void* index,
                       uint32_t* d_err, cudaStream_t st) {
  const uint64_t m = (uint64_t)g->m;
  IndexView v = index_view(index, m);
  const int gb = guide_bits(m);
  const uint64_t slots = (1ull << gb) + 1;  // nb <= 2^gb, plus guide[nb]
  const unsigned blocks = (unsigned)((slots + 255) / 256);
  k_guide<<<blocks, 256, 0, st>>>(prefix, (uint32_t)m, gb, v.guide, v.hdr, plan, delta, g->id, d_err);
  TC_LAUNCHED(1);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

// ---------------------------------------------------------------------------
// Sampler.

struct SamplerArgs {
  const OutEdge* out_e;
  const InEdge* in_e;
  const uint32_t* pair_off;
  const int32_t* pair_dst;
  const uint32_t* pair_eoff;
  const int64_t* pair_t;
  const uint64_t* prefix;
  const IndexHeader* hdr;
  const EdgeRec* rec;
  const uint32_t* guide;
  uint64_t k, seed, offset;
  uint32_t m;
  int64_t delta;
  uint64_t graph_id;
  uint64_t* trace;
  SampleSums* sums;
};

// Positions [a, b) of the pair list L_{x,y} with time in (tlo, thi) or
// (tlo, thi] (hi_incl).  Returns false when x never sends to y.
__device__ __forceinline__ bool pair_window(const SamplerArgs& A, int32_t x, int32_t y, int64_t tlo, int64_t thi,
                                            bool hi_incl, uint32_t* a, uint32_t* b) {
  uint32_t lo = __ldg(A.pair_off + x), hi = __ldg(A.pair_off + x + 1);
  while (lo < hi) {
    const uint32_t mid = lo + ((hi - lo) >> 1);
    if (__ldg(A.pair_dst + mid) < y) lo = mid + 1; else hi = mid;
  }
  if (lo >= __ldg(A.pair_off + x + 1) || __ldg(A.pair_dst + lo) != y) return false;
  const uint32_t s = __ldg(A.pair_eoff + lo), e = __ldg(A.pair_eoff + lo + 1);
  auto tt = [&](uint32_t p) { return __ldg(A.pair_t + p); };
  *a = search_time<false>(s, e, tlo, tt);
  *b = hi_incl ? search_time<false>(*a, e, thi, tt) : search_time<true>(*a, e, thi, tt);
  return true;
}

// ListCount (Alg. 4) over l lists by one merged pass in time order: an
// element of list r extends every increasing tuple of lists 1..r-1 that ends
// strictly earlier, so with acc[r] = number of tuples over lists 1..r seen
// so far, each element of list r adds acc[r-1] (acc[0] = 1).  Elements with
// equal time are handled lists-last-first so that ties never chain.
__device__ uint64_t list_count_merge(const int64_t* __restrict__ pt, const uint32_t* a, const uint32_t* b, int l,
                                     uint32_t* err) {
  uint64_t acc[17];
  uint32_t head[16];
  acc[0] = 1;
  for (int r = 0; r < l; r++) {
    acc[r + 1] = 0;
    head[r] = a[r];
  }
  for (;;) {
    int64_t tau = INT64_MAX;
    bool any = false;
    for (int r = 0; r < l; r++)
      if (head[r] < b[r]) {
        const int64_t x = __ldg(pt + head[r]);
        if (!any || x < tau) tau = x;
        any = true;
      }
    if (!any) break;
    for (int r = l - 1; r >= 0; r--)
      while (head[r] < b[r] && __ldg(pt + head[r]) == tau) {
        const uint64_t s = acc[r + 1] + acc[r];
        if (s < acc[r + 1]) atomicOr(err, kErrOverflow);
        acc[r + 1] = s;
        head[r]++;
      }
  }
  return acc[l];
}

// CheckMotif (Alg. 3) of the path (u' -e1- u -e2- v -e3- v').
__device__ __forceinline__ uint64_t check_motif(const SamplerArgs& A, const Plan& P, int32_t up, int32_t u,
                                                int32_t v, int32_t vp, int64_t t1, int64_t t2, int64_t t3,
                                                uint32_t* err, uint64_t* checked) {
  if (up == u || up == v || up == vp || u == v || u == vp || v == vp) return 0;
  // anchor edges ordered by rank must have strictly increasing times
  int64_t ta[3];  // times of anchor ranks rk[0] < rk[1] < rk[2]
#pragma unroll
  for (int j = 0; j < 3; j++) {
    const int r = P.rk[j];
    ta[j] = r == P.e1 ? t1 : (r == P.mid ? t2 : t3);
  }
  if (!(ta[0] < ta[1] && ta[1] < ta[2])) return 0;
  if ((uint64_t)ta[2] - (uint64_t)ta[0] > (uint64_t)A.delta) return 0;
  ++*checked;
  int32_t phi[4];
  phi[P.lab[0]] = up;
  phi[P.lab[1]] = u;
  phi[P.lab[2]] = v;
  phi[P.lab[3]] = vp;
  uint64_t X = 1;
  for (int gp = 0; gp < 3; gp++) {
    const int l = P.ngap[gp];
    if (l == 0) continue;
    const int64_t tlo = ta[gp];
    const int64_t thi = gp < 2 ? ta[gp + 1] : sat_add(ta[0], A.delta);
    const bool incl = gp == 2;
    uint32_t a[16], b[16];
    for (int j = 0; j < l; j++) {
      if (!pair_window(A, phi[P.gx[gp][j]], phi[P.gy[gp][j]], tlo, thi, incl, &a[j], &b[j])) return 0;
      if (a[j] == b[j]) return 0;
    }
    uint64_t c;
    if (l == 1) c = b[0] - a[0];
    else c = list_count_merge(A.pair_t, a, b, l, err);
    if (c == 0) return 0;
    const uint64_t hi = __umul64hi(X, c);
    if (hi) atomicOr(err, kErrOverflow);
    X *= c;
  }
  return X;
}

template <bool Trace>
__global__ void __launch_bounds__(256) k_sample(SamplerArgs A, Plan P) {
  const IndexHeader* H = A.hdr;
  const uint64_t W = H->W;
  const uint32_t shift = H->shift;
  __shared__ uint32_t s_err;
  __shared__ unsigned long long s_x, s_x2lo, s_x2hi, s_hits, s_checked;
  if (threadIdx.x == 0) {
    s_err = 0;
    s_x = s_x2lo = s_x2hi = s_hits = s_checked = 0;
  }
  __syncthreads();
  if (H->magic == kIndexMagic && H->status) {  // the weights pass overflowed
    if (threadIdx.x == 0) atomicOr(&A.sums->err, H->status);
    return;
  }
  bool header_ok = H->magic == kIndexMagic && H->cls[0] == P.alpha1 && H->cls[1] == P.alpha3 &&
                   H->cls[2] == P.beta1 && H->cls[3] == P.beta3 && H->closed == P.closed &&
                   H->anchor[0] == P.e1 && H->anchor[1] == P.mid && H->anchor[2] == P.e3 &&
                   H->delta == A.delta && H->graph_id == A.graph_id;
  if (!header_ok) {
    if (threadIdx.x == 0) atomicOr(&A.sums->err, kErrIndexMismatch);
    return;
  }
  uint64_t sx = 0, hits = 0, checked = 0;
  unsigned __int128 sx2 = 0;
  uint32_t err = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.k && W; i += stride) {
    const uint64_t s = A.offset + i;
    uint64_t r2, r1, r3;
    if (!bounded_draw(A.seed, s, 0, W, &r2)) { err |= kErrRng; continue; }
    // middle edge: the unique e with prefix[e] <= r2 < prefix[e + 1]
    const uint32_t b = (uint32_t)(r2 >> shift);
    uint32_t lo = __ldg(A.guide + b), hi = __ldg(A.guide + b + 1);
    while (lo < hi) {
      const uint32_t mid = lo + ((hi - lo + 1) >> 1);
      if (__ldg(A.prefix + mid) <= r2) lo = mid; else hi = mid - 1;
    }
    const EdgeRec e = A.rec[lo];
    if (e.d1 == 0 || e.d3 == 0) { err |= kErrBounds; continue; }  // index not built from this prefix
    if (!bounded_draw(A.seed, s, 1, e.d1, &r1) || !bounded_draw(A.seed, s, 2, e.d3, &r3)) {
      err |= kErrRng;
      continue;
    }
    const uint32_t p1 = e.lo1 + (uint32_t)r1, p3 = e.lo3 + (uint32_t)r3;
    if (lo >= A.m || p1 >= A.m || p3 >= A.m) { err |= kErrBounds; continue; }
    int32_t up, vp;
    int64_t t1, t3;
    if (P.alpha1 < 0) {
      const InEdge x = A.in_e[p1];
      up = x.src;
      t1 = x.t;
    } else {
      const OutEdge x = A.out_e[p1];
      up = x.dst;
      t1 = x.t;
    }
    if (P.alpha3 < 0) {
      const InEdge x = A.in_e[p3];
      vp = x.src;
      t3 = x.t;
    } else {
      const OutEdge x = A.out_e[p3];
      vp = x.dst;
      t3 = x.t;
    }
    const uint64_t X = check_motif(A, P, up, e.u, e.v, vp, t1, e.t, t3, &s_err, &checked);
    if (Trace) {
      A.trace[4 * i + 0] = lo;
      A.trace[4 * i + 1] = p1;
      A.trace[4 * i + 2] = p3;
      A.trace[4 * i + 3] = X;
    }
    const uint64_t nx = sx + X;
    if (nx < sx) err |= kErrOverflow;
    sx = nx;
    sx2 += (unsigned __int128)X * X;
    hits += X != 0;
  }
  // warp reduction, then one atomic per warp into shared, one per block global
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t ox = __shfl_down_sync(0xffffffffu, sx, o);
    const uint64_t olo = __shfl_down_sync(0xffffffffu, (uint64_t)sx2, o);
    const uint64_t ohi = __shfl_down_sync(0xffffffffu, (uint64_t)(sx2 >> 64), o);
    const uint64_t oh = __shfl_down_sync(0xffffffffu, hits, o);
    const uint64_t oc = __shfl_down_sync(0xffffffffu, checked, o);
    const uint32_t oe = __shfl_down_sync(0xffffffffu, err, o);
    const uint64_t nx = sx + ox;
    if (nx < sx) err |= kErrOverflow;
    sx = nx;
    sx2 += ((unsigned __int128)ohi << 64) | olo;
    hits += oh;
    checked += oc;
    err |= oe;
  }
  if ((threadIdx.x & 31) == 0) {
    const unsigned long long old = atomicAdd(&s_x, (unsigned long long)sx);
    if (old + sx < old) err |= kErrOverflow;
    const unsigned long long lo = (uint64_t)sx2;
    const unsigned long long ol = atomicAdd(&s_x2lo, lo);
    unsigned long long carry = (ol + lo < ol) ? 1ull : 0ull;
    atomicAdd(&s_x2hi, (unsigned long long)(sx2 >> 64) + carry);
    atomicAdd(&s_hits, (unsigned long long)hits);
    atomicAdd(&s_checked, (unsigned long long)checked);
    if (err) atomicOr(&s_err, err);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    SampleSums* G = A.sums;
    uint32_t e2 = s_err;
    const unsigned long long old = atomicAdd(&G->sum_x, s_x);
    if (old + s_x < old) e2 |= kErrOverflow;
    const unsigned long long ol = atomicAdd(&G->sum_x2_lo, s_x2lo);
    atomicAdd(&G->sum_x2_hi, s_x2hi + ((ol + s_x2lo < ol) ? 1ull : 0ull));
    atomicAdd(&G->hits, s_hits);
    atomicAdd(&G->checked, s_checked);
    if (blockIdx.x == 0) G->W = W;
    if (e2) atomicOr(&G->err, e2);
  }
}

tc_status launch_sampler(const tc_graph* g, const Plan& plan, int64_t delta, const uint64_t* prefix,
                         const void* index, uint64_t k, uint64_t seed, uint64_t offset, uint64_t* trace,
                         SampleSums* d_sums, cudaStream_t st) {
  const uint64_t m = (uint64_t)g->m;
  IndexView v = index_view(const_cast<void*>(index), m);
  SamplerArgs A;
  A.out_e = g->out_e;
  A.in_e = g->in_e;
  A.pair_off = g->pair_off;
  A.pair_dst = g->pair_dst;
  A.pair_eoff = g->pair_eoff;
  A.pair_t = g->pair_t;
  A.prefix = prefix;
  A.hdr = v.hdr;
  A.rec = v.rec;
  A.guide = v.guide;
  A.k = k;
  A.m = (uint32_t)m;
  A.seed = seed;
  A.offset = offset;
  A.delta = delta;
  A.graph_id = g->id;
  A.trace = trace;
  A.sums = d_sums;
  static int blocks_per_sm[2] = {0, 0};
  const int ti = trace ? 1 : 0;
  if (!blocks_per_sm[ti]) {
    int b = 0;
    if (trace)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_sample<true>, 256, 0);
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_sample<false>, 256, 0);
    blocks_per_sm[ti] = b > 0 ? b : 1;
  }
  uint64_t blocks = (uint64_t)num_sms() * blocks_per_sm[ti];
  const uint64_t need = (k + 255) / 256;
  if (need < blocks) blocks = need ? need : 1;
  if (trace)
    k_sample<true><<<(unsigned)blocks, 256, 0, st>>>(A, plan);
  else
    k_sample<false><<<(unsigned)blocks, 256, 0, st>>>(A, plan);
  TC_LAUNCHED(1);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

}  // namespace tc
