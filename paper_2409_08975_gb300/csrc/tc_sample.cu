// Path weights (Claim 1, Alg. 1), the guide table of the CDF search, and the
// sampler with CheckMotif / ListCount and the reduction of X (Alg. 2-5).
#include <cuda_runtime.h>

#include <cstring>
#include <utility>
#include <vector>

#include "tc_internal.cuh"

namespace tc {

// ---------------------------------------------------------------------------
// Weights (Claim 1, Alg. 1): w_e = d1 * d3 for every canonical edge
// e = (u, v, t), the sizes of the window of u's alpha1 list and of v's alpha3
// list, and their exact prefix sum.
//
// The four binary searches per edge of Alg. 1 start from anchors built with
// the lists (tc_graph::x_in, x_out, out2in; independent of delta): each
// window bound is found by a galloping search (doubling steps, then
// bisection) from a position where the list reaches time t, so a window of
// d entries costs O(log d) probes near the anchor instead of O(log deg)
// probes over the whole list.  The anchors' range words give the list's
// bounds (no random load of the destination's offsets), and an exact anchor
// (the list's lower bound of t) is itself the window's bound at t in strict
// mode.  The u side of consecutive edges (one source vertex in time order)
// searches the same list at increasing positions.
//
// The weights pass also sums w over each tile of kWTile edges, the first
// level of the reduce-then-scan that writes the prefix (so w is read once
// more, not twice).
//
// A wedge anchor (3-vertex motif) has one window, at u or at v; the other
// side is the dummy [0, 1), so w_e is the size of that window.

// Window searches on the 32-bit time arrays when the graph has them.
#ifndef TC_COMPACT_TIMES
#define TC_COMPACT_TIMES 1
#endif

// Pair-list searches of the sampler on the 32-bit times when the graph has them.
#ifndef TC_COMPACT_PAIRS
#define TC_COMPACT_PAIRS 1
#endif

// Resident blocks per SM the weights kernel is compiled for (caps its registers).
#ifndef TC_WEIGHTS_MIN_BLOCKS
#define TC_WEIGHTS_MIN_BLOCKS 8
#endif

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr int kWThreads = 256;
constexpr int kWItems = 8;
constexpr int kWTile = kWThreads * kWItems;  // edges per tile: the scan's tile

// First position p in [s, f) whose time is >= x (Gt: > x), searched from a
// position a in [s, f]: doubling steps away from a until the answer is
// bracketed, then bisection.  At most 2 log2(f - s) + 2 probes.
template <bool Gt, class TimeAt>
__device__ __forceinline__ uint32_t gallop(uint32_t s, uint32_t f, uint32_t a, int64_t x, TimeAt tt) {
  auto pred = [&](uint32_t p) {
    const int64_t v = tt(p);
    return Gt ? v > x : v >= x;
  };
  uint32_t lo, hi;  // the answer lies in [lo, hi]; pred(hi) holds or hi == f
  if (a < f && !pred(a)) {
    lo = a + 1;
    hi = f;
    uint32_t step = 1;
    while (lo < hi) {
      const uint32_t p = (hi - lo > step - 1) ? lo + (step - 1) : hi - 1;
      if (pred(p)) {
        hi = p;
        break;
      }
      lo = p + 1;
      step <<= 1;
    }
  } else {
    lo = s;
    hi = a;
    uint32_t step = 1;
    while (hi > lo) {
      const uint32_t p = (hi - lo > step) ? hi - step : lo;
      if (!pred(p)) {
        lo = p + 1;
        break;
      }
      hi = p;
      step <<= 1;
    }
  }
  while (lo < hi) {
    const uint32_t mid = lo + ((hi - lo) >> 1);
    if (pred(mid)) hi = mid; else lo = mid + 1;
  }
  return lo;
}

// The window of list [s, f) around time t (beta < 0: before, else after;
// strict or closed at t) as positions [*lo, *hi), searched from an anchor a
// with lower_bound(t) <= a <= upper_bound(t).
template <class TimeAt>
__device__ __forceinline__ void window_from(uint32_t s, uint32_t f, uint32_t a, int beta, int closed, int64_t t,
                                            int64_t delta, TimeAt tt, uint32_t* lo, uint32_t* hi) {
  if (beta < 0) {
    *hi = closed ? gallop<true>(s, f, a, t, tt) : gallop<false>(s, f, a, t, tt);
    *lo = gallop<false>(s, f, *hi, sat_sub(t, delta), tt);
  } else {
    *lo = closed ? gallop<false>(s, f, a, t, tt) : gallop<true>(s, f, a, t, tt);
    *hi = gallop<true>(s, f, *lo, sat_add(t, delta), tt);
  }
}

struct WeightsArgs {
  const OutEdge* out_e;
  const InEdge* in_e;
  const uint32_t* out_off;
  const uint32_t* in_off;
  const uint32_t* out_t32;
  const uint32_t* in_t32;
  const uint32_t* x_in;
  const uint32_t* x_out;
  const uint32_t* out2in;
  const uint32_t* r_in;    // range words of x_in, x_out, out2in and of the edge in u's out-list
  const uint32_t* r_out;
  const uint32_t* r_o2i;
  const uint32_t* r_self;
  int64_t tmin;
  uint64_t m;
  int64_t delta;
  int alpha1, alpha3, beta1, beta3, closed;
  EdgeWin* win;
  uint64_t* w;
  uint64_t* tile_sums;  // sum of w over each tile
  uint32_t* err;
};

// Window of side alpha (< 0: the vertex's in-list, > 0: its out-list) of
// canonical edge i = (x, ., t), searched from anchor a.
template <bool Compact>
__device__ __forceinline__ void side_window(const WeightsArgs& A, int alpha, int beta, int32_t x, uint32_t a,
                                            int64_t t, uint32_t* lo, uint32_t* hi) {
  if (alpha < 0) {
    auto tt = [&](uint32_t p) -> int64_t { return Compact ? (int64_t)__ldg(A.in_t32 + p) + A.tmin : A.in_e[p].t; };
    window_from(__ldg(A.in_off + x), __ldg(A.in_off + x + 1), a, beta, A.closed, t, A.delta, tt, lo, hi);
  } else {
    auto tt = [&](uint32_t p) -> int64_t { return Compact ? (int64_t)__ldg(A.out_t32 + p) + A.tmin : A.out_e[p].t; };
    window_from(__ldg(A.out_off + x), __ldg(A.out_off + x + 1), a, beta, A.closed, t, A.delta, tt, lo, hi);
  }
}

// Block b takes tile b: the windows and w of its kWTile edges (coalesced:
// edge b kWTile + j 256 + thread), and the tile's sum of w.
template <bool Compact>
__global__ void __launch_bounds__(kWThreads, TC_WEIGHTS_MIN_BLOCKS) k_weights(const __grid_constant__ WeightsArgs A) {
  __shared__ unsigned long long s_warp[kWThreads / 32];
  __shared__ uint32_t s_ovf;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) s_ovf = 0;
  const uint64_t base = (uint64_t)blockIdx.x * kWTile;
  unsigned long long sum = 0;
  bool ovf = false;
#pragma unroll 1
  for (int j = 0; j < kWItems; j++) {
    const uint64_t i = base + (uint64_t)j * kWThreads + tid;
    if (i >= A.m) break;
    const OutEdge e = A.out_e[i];
    uint32_t lo1 = 0, hi1 = 1, lo3 = 0, hi3 = 1;  // a wedge's unused side is [0, 1)
    // anchors: u's in-list (x_in) or the edge itself in u's out-list; the
    // edge itself in v's in-list (out2in) or v's out-list (x_out)
    if (A.alpha1 != 0)
      side_window<Compact>(A, A.alpha1, A.beta1, e.src, A.alpha1 < 0 ? __ldg(A.x_in + i) : (uint32_t)i, e.t, &lo1,
                           &hi1);
    if (A.alpha3 != 0)
      side_window<Compact>(A, A.alpha3, A.beta3, e.dst, A.alpha3 < 0 ? __ldg(A.out2in + i) : __ldg(A.x_out + i), e.t,
                           &lo3, &hi3);
    EdgeWin r;
    r.lo1 = lo1;
    r.d1 = hi1 - lo1;
    r.lo3 = lo3;
    r.d3 = hi3 - lo3;
    A.win[i] = r;
    const unsigned long long wv = (unsigned long long)r.d1 * (unsigned long long)r.d3;
    A.w[i] = wv;
    if (sum + wv < sum) ovf = true;
    sum += wv;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, sum, o);
    if (sum + y < sum) ovf = true;
    sum += y;
  }
  if (lane == 0) s_warp[wid] = sum;
  if (ovf) s_ovf = 1;
  __syncthreads();
  if (tid == 0) {
    unsigned long long t = 0;
    bool o2 = s_ovf != 0;
    for (int v = 0; v < kWThreads / 32; v++) {
      if (t + s_warp[v] < t) o2 = true;
      t += s_warp[v];
    }
    A.tile_sums[blockIdx.x] = t;
    if (o2) atomicOr(A.err, kErrOverflow);
  }
}

// Window of one side on the 32-bit list times, searched from anchor a: the
// list [s, f) from the anchor's range word rw (the offsets of x's list are
// read only where a field is saturated).  exact: a is the list's lower bound
// of t (x_in, x_out), so "time >= t" needs no probe.
// The vertex x (the edge's source, or its destination when dst_side) is
// read from the edge record only then.
__device__ __forceinline__ void side_window_rw(const WeightsArgs& A, int alpha, int beta, uint64_t i, bool dst_side,
                                               uint32_t a, uint32_t rw, bool exact, int64_t t, uint32_t* lo,
                                               uint32_t* hi) {
  const uint32_t* off = alpha < 0 ? A.in_off : A.out_off;
  uint32_t s = a - (rw >> 16), f = a + (rw & 0xFFFFu);
  if ((rw >> 16) == kRangeCap || (rw & 0xFFFFu) == kRangeCap) {
    const int2 sd = __ldg(reinterpret_cast<const int2*>(A.out_e + i));  // (src, dst)
    const int32_t x = dst_side ? sd.y : sd.x;
    if ((rw >> 16) == kRangeCap) s = __ldg(off + x);
    if ((rw & 0xFFFFu) == kRangeCap) f = __ldg(off + x + 1);
  }
  const uint32_t* t32 = alpha < 0 ? A.in_t32 : A.out_t32;
  auto tt = [&](uint32_t p) -> int64_t { return (int64_t)__ldg(t32 + p) + A.tmin; };
  if (beta < 0) {
    *hi = (exact && !A.closed) ? a : (A.closed ? gallop<true>(s, f, a, t, tt) : gallop<false>(s, f, a, t, tt));
    *lo = gallop<false>(s, f, *hi, sat_sub(t, A.delta), tt);
  } else {
    *lo = (exact && A.closed) ? a : (A.closed ? gallop<false>(s, f, a, t, tt) : gallop<true>(s, f, a, t, tt));
    *hi = gallop<true>(s, f, *lo, sat_add(t, A.delta), tt);
  }
}

// Block b takes tile b (coalesced: edge b kWTile + j 256 + thread) on the
// 32-bit list times: the edge's time from the 32-bit out-list times, the
// list bounds from the anchors' range words (the edge record and the
// offsets are read only where a word is saturated), an exact anchor's
// bound without a probe, the windows and w written with streaming stores,
// and the tile's sum of w.
__global__ void __launch_bounds__(kWThreads, TC_WEIGHTS_MIN_BLOCKS)
    k_weights_rw(const __grid_constant__ WeightsArgs A) {
  __shared__ unsigned long long s_warp[kWThreads / 32];
  __shared__ uint32_t s_ovf;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) s_ovf = 0;
  const uint64_t base = (uint64_t)blockIdx.x * kWTile;
  unsigned long long sum = 0;
  bool ovf = false;
#pragma unroll 1
  for (int j = 0; j < kWItems; j++) {
    const uint64_t i = base + (uint64_t)j * kWThreads + tid;
    if (i >= A.m) break;
    const int64_t t = (int64_t)__ldg(A.out_t32 + i) + A.tmin;  // the edge's time (4 bytes, not the record)
    uint32_t lo1 = 0, hi1 = 1, lo3 = 0, hi3 = 1;
    // anchors: u's in-list (x_in, exact) or the edge itself in u's out-list;
    // the edge itself in v's in-list (out2in) or v's out-list (x_out, exact)
    if (A.alpha1 < 0)
      side_window_rw(A, -1, A.beta1, i, false, __ldg(A.x_in + i), __ldg(A.r_in + i), true, t, &lo1, &hi1);
    else if (A.alpha1 > 0)
      side_window_rw(A, 1, A.beta1, i, false, (uint32_t)i, __ldg(A.r_self + i), false, t, &lo1, &hi1);
    if (A.alpha3 < 0)
      side_window_rw(A, -1, A.beta3, i, true, __ldg(A.out2in + i), __ldg(A.r_o2i + i), false, t, &lo3, &hi3);
    else if (A.alpha3 > 0)
      side_window_rw(A, 1, A.beta3, i, true, __ldg(A.x_out + i), __ldg(A.r_out + i), true, t, &lo3, &hi3);
    __stcs(reinterpret_cast<uint4*>(A.win + i), make_uint4(lo1, hi1 - lo1, lo3, hi3 - lo3));
    const unsigned long long wv = (unsigned long long)(hi1 - lo1) * (unsigned long long)(hi3 - lo3);
    __stcs(reinterpret_cast<unsigned long long*>(A.w + i), wv);
    if (sum + wv < sum) ovf = true;
    sum += wv;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, sum, o);
    if (sum + y < sum) ovf = true;
    sum += y;
  }
  if (lane == 0) s_warp[wid] = sum;
  if (ovf) s_ovf = 1;
  __syncthreads();
  if (tid == 0) {
    unsigned long long t = 0;
    bool o2 = s_ovf != 0;
    for (int v = 0; v < kWThreads / 32; v++) {
      if (t + s_warp[v] < t) o2 = true;
      t += s_warp[v];
    }
    A.tile_sums[blockIdx.x] = t;
    if (o2) atomicOr(A.err, kErrOverflow);
  }
}

static uint64_t weights_tiles(uint64_t m) { return (m + kWTile - 1) / kWTile; }

// Scratch of launch_weights_scan: w (unless the caller keeps it), the tile
// sums, and the tile sums' own scan levels.
size_t weights_scan_scratch_bytes(uint64_t m) {
  const uint64_t T = weights_tiles(m) ? weights_tiles(m) : 1;
  return align256(8 * (m ? m : 1)) + align256(8 * T) + align256(8 * (scan_u64_scratch_words(T) + 1));
}

tc_status launch_weights_scan(const tc_graph* g, const Plan& plan, int64_t delta, EdgeWin* win, uint64_t* prefix,
                              uint64_t* w, void* scratch, uint32_t* d_err, cudaStream_t st) {
  static_assert(kWTile == 2048, "the weights tiles are the scan's tiles");
  const uint64_t m = (uint64_t)g->m;
  if (m == 0) {
    TC_CUDA(cudaMemsetAsync(prefix, 0, sizeof(uint64_t), st));
    return TC_OK;
  }
  if (scan_tile_size() != (uint64_t)kWTile) return set_error(TC_ERR_INVALID_ARG, "scan tile mismatch");
  const uint64_t T = weights_tiles(m);
  if (T > 0x7FFFFFFFull) return set_error(TC_ERR_INVALID_ARG, "too many edges for the weights pass");
  char* p = (char*)scratch;
  uint64_t* wbuf = w ? w : (uint64_t*)p;
  uint64_t* sums = (uint64_t*)(p + align256(8 * m));
  uint64_t* scan_scratch = (uint64_t*)(p + align256(8 * m) + align256(8 * T));
  WeightsArgs A;
  A.out_e = g->out_e;
  A.in_e = g->in_e;
  A.out_off = g->out_off;
  A.in_off = g->in_off;
  A.out_t32 = g->out_t32;
  A.in_t32 = g->in_t32;
  A.x_in = g->x_in;
  A.x_out = g->x_out;
  A.out2in = g->out2in;
  A.r_in = g->r_in;
  A.r_out = g->r_out;
  A.r_o2i = g->r_o2i;
  A.r_self = g->r_self;
  A.tmin = g->tmin;
  A.m = m;
  A.delta = delta;
  A.alpha1 = plan.alpha1;
  A.alpha3 = plan.alpha3;
  A.beta1 = plan.beta1;
  A.beta3 = plan.beta3;
  A.closed = plan.closed;
  A.win = win;
  A.w = wbuf;
  A.tile_sums = sums;
  A.err = d_err;
  const bool compact = TC_COMPACT_TIMES && g->out_t32 && g->in_t32;
  if (compact)
    k_weights_rw<<<(unsigned)T, kWThreads, 0, st>>>(A);
  else
    k_weights<false><<<(unsigned)T, kWThreads, 0, st>>>(A);
  TC_LAUNCHED(1);
  TC_CUDA(cudaGetLastError());
  return scan_u64_from_tile_sums(wbuf, prefix, m, sums, d_err, scan_scratch, scan_u64_scratch_words(T) + 1, st);
}

// ---------------------------------------------------------------------------
// Index layout: [header 256 B][EdgeWin m][guide uint32 (2^gbits + 1)].

int guide_bits(uint64_t m) {
  int b = 0;
  while (b < 32 && (1ull << b) < m) b++;
  return b;
}


size_t index_bytes(uint64_t m) {
  return kIndexHeaderBytes + align256(sizeof(EdgeWin) * m) + sizeof(uint32_t) * ((1ull << guide_bits(m)) + 1);
}

struct IndexView {
  IndexHeader* hdr;
  EdgeWin* win;
  uint32_t* guide;
};

static IndexView index_view(void* index, uint64_t m) {
  char* p = (char*)index;
  IndexView v;
  v.hdr = (IndexHeader*)p;
  v.win = (EdgeWin*)(p + kIndexHeaderBytes);
  v.guide = (uint32_t*)(p + kIndexHeaderBytes + align256(sizeof(EdgeWin) * m));
  return v;
}

// Guide table: bucket b covers r in [b << shift, (b + 1) << shift); guide[b]
// is the edge whose range [prefix[i], prefix[i+1]) holds b << shift (the
// largest i with prefix[i] <= b << shift), the first candidate of the CDF
// search for any r in the bucket; guide[nb] = m - 1.  Filled edge-parallel:
// edge i owns the buckets b with b << shift in its range; a warp shares the
// writes of its 32 edges evenly, so that heavy edges do not serialise.
__global__ void __launch_bounds__(256) k_guide(const uint64_t* __restrict__ prefix, uint32_t m, int gbits,
                                               uint32_t* __restrict__ guide, IndexHeader* hdr, Plan plan,
                                               int64_t delta, uint64_t graph_id, const uint32_t* err) {
  const uint64_t W = prefix[m];
  const int wbits = W ? 64 - __clzll(W - 1) : 0;
  const uint32_t shift = wbits > gbits ? (uint32_t)(wbits - gbits) : 0u;
  const uint32_t nb = W ? (uint32_t)(((W - 1) >> shift) + 1) : 0u;
  const uint64_t low = (1ull << shift) - 1ull;
  auto first_bucket = [&](uint64_t x) { return (uint32_t)((x >> shift) + ((x & low) != 0)); };  // ceil(x / 2^shift)
  const int lane = threadIdx.x & 31;
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t wb = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; wb * 32 < m; wb += warps) {
    const uint64_t i = wb * 32 + lane;
    uint32_t b0 = 0, n = 0;
    if (i < m) {
      b0 = first_bucket(prefix[i]);
      n = first_bucket(prefix[i + 1]) - b0;
    }
    uint32_t incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const uint32_t excl = incl - n;
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    for (uint32_t q0 = 0; q0 < total; q0 += 32) {
      const uint32_t q = q0 + lane;
      // owner: the last lane whose exclusive offset is <= q
      int lo = 0, hi = 31;
#pragma unroll
      for (int step = 0; step < 5; step++) {
        const int mid = (lo + hi + 1) >> 1;
        const uint32_t ex = __shfl_sync(0xffffffffu, excl, mid);
        if (ex <= q) lo = mid; else hi = mid - 1;
      }
      const uint32_t ob0 = __shfl_sync(0xffffffffu, b0, lo);
      const uint32_t oex = __shfl_sync(0xffffffffu, excl, lo);
      if (q < total) guide[ob0 + (q - oex)] = (uint32_t)(wb * 32 + lo);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (m) guide[nb] = m - 1;
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
  IndexView v = index_view(index, (uint64_t)g->m);
  return launch_guide_at(g, plan, delta, prefix, v.hdr, v.guide, d_err, st);
}

size_t proposal_index_bytes(uint64_t m) {
  return kIndexHeaderBytes + sizeof(uint32_t) * ((1ull << guide_bits(m)) + 1);
}

tc_status launch_guide_at(const tc_graph* g, const Plan& plan, int64_t delta, const uint64_t* prefix,
                          IndexHeader* hdr, uint32_t* guide, uint32_t* d_err, cudaStream_t st) {
  const uint64_t m = (uint64_t)g->m;
  IndexView v;
  v.hdr = hdr;
  v.guide = guide;
  const int gb = guide_bits(m);
  uint64_t blocks = (m + 255) / 256;
  const uint64_t cap = (uint64_t)num_sms() * 16;
  if (blocks > cap) blocks = cap;
  if (blocks == 0) blocks = 1;
  k_guide<<<(unsigned)blocks, 256, 0, st>>>(prefix, (uint32_t)m, gb, v.guide, v.hdr, plan, delta, g->id, d_err);
  TC_LAUNCHED(1);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

// ---------------------------------------------------------------------------
// Sampler.

struct SamplerArgs {
  const OutEdge* out_e;
  const InEdge* in_e;
  const PairSlot* pair_hash;
  uint64_t hash_mask;
  const int64_t* pair_t;
  const uint32_t* pair_t32;  // pair-list times as t - tmin, or NULL
  int64_t tmin;
  const uint64_t* prefix;
  const IndexHeader* hdr;
  const EdgeWin* win;
  const uint32_t* guide;
  uint64_t k, seed, offset;
  const uint32_t* order;  // processing order of the chunk's samples (NULL: in id order)
  uint64_t chunk_base;    // index of the chunk's first sample within the call
  uint64_t count;         // samples in the chunk
  uint32_t m;
  int64_t delta;
  uint64_t graph_id;
  uint64_t* trace;
  SampleSums* sums;
  // proposal mode (h != NULL): the middle edge is drawn from the proposal's
  // prefix and guide (hdr, prefix, guide), the records come from the plain
  // index (win, rec_hdr), and each hit adds X and X^2 to bins[3 h + 0..2]
  const uint16_t* h;
  unsigned long long* bins;
  const uint32_t* hrange;  // proposal: smallest and largest h (in the proposal index header)
  const IndexHeader* rec_hdr;
};

// Two bisections of [s, e) at once: *a = the first position with time > xa,
// *b = the first with time > xb (incl) or >= xb; one probe of each per step.
template <class TimeAt>
__device__ __forceinline__ void search_time2(uint32_t s, uint32_t e, int64_t xa, int64_t xb, bool incl, TimeAt tt,
                                             uint32_t* a, uint32_t* b) {
  uint32_t la = s, ha = e, lb = s, hb = e;
  while (la < ha || lb < hb) {
    const uint32_t ma = la + ((ha - la) >> 1), mb = lb + ((hb - lb) >> 1);
    const bool ra = la < ha, rb = lb < hb;
    const int64_t va = ra ? tt(ma) : 0, vb = rb ? tt(mb) : 0;
    if (ra) {
      if (va <= xa) la = ma + 1; else ha = ma;
    }
    if (rb) {
      if (incl ? vb <= xb : vb < xb) lb = mb + 1; else hb = mb;
    }
  }
  *a = la;
  *b = lb;
}

// Positions [a, b) of the pair list L_{x,y} with time in (tlo, thi) or
// (tlo, thi] (hi_incl).  The list's range comes from the pair hash table (one
// 16-byte slot per probe).  Returns false when x never sends to y.
__device__ __forceinline__ bool pair_window(const SamplerArgs& A, int32_t x, int32_t y, int64_t tlo, int64_t thi,
                                            bool hi_incl, uint32_t* a, uint32_t* b) {
  const uint64_t key = pair_key((uint32_t)x, (uint32_t)y);
  uint64_t h = mix64(key) & A.hash_mask;
  uint32_t s = 0, e = 0;
  bool found = false;
  for (uint64_t probe = 0; probe <= A.hash_mask; probe++) {
    const uint4 slot = __ldg(reinterpret_cast<const uint4*>(A.pair_hash + h));
    if (slot.x == (uint32_t)x && slot.y == (uint32_t)y) {
      s = slot.z;
      e = slot.w;
      found = true;
      break;
    }
    if (slot.x == 0xFFFFFFFFu) break;
    h = (h + 1) & A.hash_mask;
  }
  if (!found) return false;
  // both bounds bisect [s, e) in lockstep, so that their probes are in flight together
  if (A.pair_t32) {  // 4-byte entries, eight per sector
    auto tt = [&](uint32_t p) { return (int64_t)__ldg(A.pair_t32 + p) + A.tmin; };
    search_time2(s, e, tlo, thi, hi_incl, tt, a, b);
  } else {
    auto tt = [&](uint32_t p) { return __ldg(A.pair_t + p); };
    search_time2(s, e, tlo, thi, hi_incl, tt, a, b);
  }
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

// ListCount of a gap with two or more lists (kept out of line so that its
// arrays do not weigh on the single-list path).
__device__ __noinline__ uint64_t gap_count_multi(const SamplerArgs& A, const Plan& P, int gp, int32_t up, int32_t u,
                                                int32_t v, int32_t vp, int64_t tlo, int64_t thi, bool incl,
                                                uint32_t* err) {
  auto phi = [&](int role) { return role == 0 ? up : (role == 1 ? u : (role == 2 ? v : vp)); };
  const int l = P.ngap[gp];
  uint32_t a[16], b[16];
  for (int j = 0; j < l; j++) {
    if (!pair_window(A, phi(P.gx[gp][j]), phi(P.gy[gp][j]), tlo, thi, incl, &a[j], &b[j])) return 0;
    if (a[j] == b[j]) return 0;
  }
  return list_count_merge(A.pair_t, a, b, l, err);
}

// Product over the gaps of their ListCounts (Alg. 3, 4): gap gp holds the
// non-anchor motif edges of ranks between anchor ranks NG gp and gp + 1, with
// times in (ta[gp], ta[gp + 1]); the last gap runs up to ta[0] + delta
// inclusive.  phi maps path roles (u', u, v, v') to graph vertices.
template <int NG>
__device__ __forceinline__ uint64_t gaps_product(const SamplerArgs& A, const Plan& P, const int64_t* ta, int32_t up,
                                                 int32_t u, int32_t v, int32_t vp, uint32_t* err) {
  auto phi = [&](int role) { return role == 0 ? up : (role == 1 ? u : (role == 2 ? v : vp)); };
  uint64_t X = 1;
#pragma unroll
  for (int gp = 0; gp < NG; gp++) {
    const int l = P.ngap[gp];
    if (l == 0) continue;
    const int64_t tlo = ta[gp];
    const int64_t thi = gp < NG - 1 ? ta[gp + 1] : sat_add(ta[0], A.delta);
    const bool incl = gp == NG - 1;
    uint64_t c;
    if (l == 1) {  // one list: its length in the window
      uint32_t a0, b0;
      if (!pair_window(A, phi(P.gx[gp][0]), phi(P.gy[gp][0]), tlo, thi, incl, &a0, &b0)) return 0;
      c = b0 - a0;
    } else {
      c = gap_count_multi(A, P, gp, up, u, v, vp, tlo, thi, incl, err);
    }
    if (c == 0) return 0;
    const uint64_t hi = __umul64hi(X, c);
    if (hi) atomicOr(err, kErrOverflow);
    X *= c;
  }
  return X;
}

// CheckMotif of a wedge (3-vertex motif): base (u, v, t0) and second edge
// to or from y at time tj; the three vertices distinct, t0 < tj <= t0 + delta.
__device__ __forceinline__ uint64_t check_wedge(const SamplerArgs& A, const Plan& P, int32_t y, int32_t u, int32_t v,
                                                int64_t t0, int64_t tj, uint32_t* err, uint32_t* checked) {
  if (u == v || y == u || y == v) return 0;
  if (!(t0 < tj) || (uint64_t)tj - (uint64_t)t0 > (uint64_t)A.delta) return 0;
  ++*checked;
  const int64_t ta[2] = {t0, tj};
  return gaps_product<2>(A, P, ta, y, u, v, y, err);
}

// CheckMotif (Alg. 3) of the path (u' -e1- u -e2- v -e3- v'), or of the
// wedge (u' -e1- u -e2- v) / (u -e2- v -e3- v') of a wedge anchor.
__device__ __forceinline__ uint64_t check_motif(const SamplerArgs& A, const Plan& P, int32_t up, int32_t u,
                                                int32_t v, int32_t vp, int64_t t1, int64_t t2, int64_t t3,
                                                uint32_t* err, uint32_t* checked) {
  if (P.wedge)
    return P.wedge == 1 ? check_wedge(A, P, up, u, v, t2, t1, err, checked)
                        : check_wedge(A, P, vp, u, v, t2, t3, err, checked);
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
  return gaps_product<3>(A, P, ta, up, u, v, vp, err);
}

// The far vertex and time of the end edge at list position p of an alpha
// list (alpha = 0: a wedge's dummy end, vertex -1).
__device__ __forceinline__ void end_edge(const SamplerArgs& A, int alpha, uint32_t p, int32_t* x, int64_t* t) {
  if (alpha < 0) {
    const InEdge e = A.in_e[p];
    *x = e.src;
    *t = e.t;
  } else if (alpha > 0) {
    const OutEdge e = A.out_e[p];
    *x = e.dst;
    *t = e.t;
  } else {
    *x = -1;
    *t = 0;
  }
}

// Per-thread running sums of a sampling kernel.
struct ThreadSums {
  uint64_t sx = 0, hits = 0;
  uint32_t checked = 0;
  unsigned __int128 sx2 = 0;
  uint32_t err = 0;
};

// The index must have been built for this graph, anchor class and delta
// (the weights depend on nothing else); a proposal's records come from the
// plain index.  Returns 0 or the error bits to report.
__device__ __forceinline__ uint32_t index_check(const SamplerArgs& A, const Plan& P) {
  const IndexHeader* H = A.hdr;
  if (H->magic == kIndexMagic && H->status) return H->status;  // the weights pass overflowed
  auto matches = [&](const IndexHeader* X) {
    return X->magic == kIndexMagic && X->cls[0] == P.alpha1 && X->cls[1] == P.alpha3 && X->cls[2] == P.beta1 &&
           X->cls[3] == P.beta3 && X->closed == P.closed && X->delta == A.delta && X->graph_id == A.graph_id;
  };
  return (matches(H) && (A.rec_hdr == nullptr || matches(A.rec_hdr))) ? 0u : kErrIndexMismatch;
}

// Resident blocks per SM the sampler is compiled for (caps its registers).
#ifndef TC_SAMPLE_MIN_BLOCKS
#define TC_SAMPLE_MIN_BLOCKS 4
#endif
#define TC_SAMPLE_MIN_BLOCKS_DECL TC_SAMPLE_MIN_BLOCKS

// Warp-shuffle reduction of the per-thread sums, one shared atomic per warp
// and one global atomic per block; 128-bit sum of squares with carries,
// overflow of the 64-bit sum flagged.
__device__ __forceinline__ void block_commit(SampleSums* G, uint64_t W, uint64_t sx, unsigned __int128 sx2,
                                             uint64_t hits, uint64_t checked, uint32_t err, uint32_t& s_err,
                                             unsigned long long& s_x, unsigned long long& s_x2lo,
                                             unsigned long long& s_x2hi, unsigned long long& s_hits,
                                             unsigned long long& s_checked) {
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
    const unsigned long long carry = (ol + lo < ol) ? 1ull : 0ull;
    atomicAdd(&s_x2hi, (unsigned long long)(sx2 >> 64) + carry);
    atomicAdd(&s_hits, (unsigned long long)hits);
    atomicAdd(&s_checked, (unsigned long long)checked);
    if (err) atomicOr(&s_err, err);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t e2 = s_err;
    const unsigned long long old = atomicAdd(&G->sum_x, s_x);
    if (old + s_x < old) e2 |= kErrOverflow;
    const unsigned long long ol = atomicAdd(&G->sum_x2_lo, s_x2lo);
    atomicAdd(&G->sum_x2_hi, s_x2hi + ((ol + s_x2lo < ol) ? 1ull : 0ull));
    atomicAdd(&G->hits, s_hits);
    atomicAdd(&G->checked, s_checked);
    G->W = W;
    if (e2) atomicOr(&G->err, e2);
  }
}

// Exhaustive path sum (the proof of Claim 2): path p in [0, W) is the
// (p - prefix[e])-th pair (p1, p3) of middle edge e, p1 major; the sum of
// CheckMotif over all paths is the exact count C, the sum of squares gives
// the exact variance of one sample.  Paths [first, first + count).
__global__ void __launch_bounds__(256, TC_SAMPLE_MIN_BLOCKS_DECL) k_path_sum(const __grid_constant__ SamplerArgs A,
                                                                            const __grid_constant__ Plan P,
                                                                            uint64_t first, uint64_t count) {
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
  const uint32_t bad = index_check(A, P);
  if (bad) {
    if (threadIdx.x == 0) atomicOr(&A.sums->err, bad);
    return;
  }
  uint64_t sx = 0, hits = 0;
  uint32_t checked = 0;
  unsigned __int128 sx2 = 0;
  uint32_t err = 0;
  const uint64_t end = first + count < W ? first + count : W;
  for (uint64_t p = first + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < end;
       p += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t b = (uint32_t)(p >> shift);
    uint32_t lo = __ldg(A.guide + b), hi = __ldg(A.guide + b + 1);
    while (lo < hi) {
      const uint32_t mid = lo + ((hi - lo + 1) >> 1);
      if (__ldg(A.prefix + mid) <= p) lo = mid; else hi = mid - 1;
    }
    if (lo >= A.m) { err |= kErrBounds; continue; }
    const EdgeWin wn = A.win[lo];
    const OutEdge e = A.out_e[lo];
    if (wn.d1 == 0 || wn.d3 == 0) { err |= kErrBounds; continue; }
    const uint64_t j = p - __ldg(A.prefix + lo);
    const uint32_t p1 = wn.lo1 + (uint32_t)(j / wn.d3), p3 = wn.lo3 + (uint32_t)(j % wn.d3);
    if (p1 >= A.m || p3 >= A.m) { err |= kErrBounds; continue; }
    int32_t up, vp;
    int64_t t1, t3;
    end_edge(A, P.alpha1, p1, &up, &t1);
    end_edge(A, P.alpha3, p3, &vp, &t3);
    const uint64_t X = check_motif(A, P, up, e.src, e.dst, vp, t1, e.t, t3, &s_err, &checked);
    const uint64_t nx = sx + X;
    if (nx < sx) err |= kErrOverflow;
    sx = nx;
    sx2 += (unsigned __int128)X * X;
    hits += X != 0;
  }
  block_commit(A.sums, W, sx, sx2, hits, checked, err, s_err, s_x, s_x2lo, s_x2hi, s_hits, s_checked);
}

// The rejection loops: the first attempt is tested in the sampler itself and
// these run only when it is rejected (probability below range / 2^64),
// starting again from attempt 0.
__device__ __forceinline__ bool bounded_draw_slow(uint64_t seed, uint64_t s, uint32_t draw, bool upper, uint64_t range,
                                               uint64_t* out) {
  return bounded_draw_words(seed, s, draw, upper, range, out);
}

// One sample (Alg. 2, 3): sample index i within the call (id offset + i).
constexpr uint32_t kSmemBins = 1088;  // per-block bins of the proposal sampler (see k_sample): the 1,025 h of S = 1024
constexpr size_t kSmemBinBytes = 3 * sizeof(unsigned long long) * kSmemBins;

// Adds X and X^2 to bin h: three 64-bit words (sum X, sum X^2 low, high).
__device__ __forceinline__ void bin_add(unsigned long long* bin, uint64_t X) {
  atomicAdd(bin, (unsigned long long)X);
  const unsigned __int128 x2 = (unsigned __int128)X * X;
  const unsigned long long l2 = (uint64_t)x2;
  const unsigned long long old = atomicAdd(bin + 1, l2);
  const unsigned long long carry = (old + l2 < old) ? 1ull : 0ull;
  if ((x2 >> 64) || carry) atomicAdd(bin + 2, (unsigned long long)(x2 >> 64) + carry);
}

template <bool Trace>
__device__ __forceinline__ void sample_one(const SamplerArgs& A, const Plan& P, uint64_t W, uint32_t shift,
                                           uint64_t i, ThreadSums& T, uint32_t* s_err,
                                           unsigned long long* sbins = nullptr, uint32_t hmin = 0) {
  const uint64_t s = A.offset + i;
  uint64_t r2, r1, r3;
  const uint2 key = make_uint2((uint32_t)A.seed, (uint32_t)(A.seed >> 32));
  {
    const uint4 o = philox4x32_10(make_uint4((uint32_t)s, (uint32_t)(s >> 32), 0u, 0u), key);
    if (!lemire_accept((uint64_t)o.x | ((uint64_t)o.y << 32), W, &r2) &&
        !bounded_draw_slow(A.seed, s, 0, false, W, &r2)) {
      T.err |= kErrRng;
      return;
    }
  }
  // middle edge: the unique e with prefix[e] <= r2 < prefix[e + 1]
  const uint32_t b = (uint32_t)(r2 >> shift);
  uint32_t lo = __ldg(A.guide + b), hi = __ldg(A.guide + b + 1);
  while (lo < hi) {
    const uint32_t mid = lo + ((hi - lo + 1) >> 1);
    if (__ldg(A.prefix + mid) <= r2) lo = mid; else hi = mid - 1;
  }
  if (lo >= A.m) { T.err |= kErrBounds; return; }
  const EdgeWin e = A.win[lo];
  const OutEdge me = A.out_e[lo];  // the middle edge (u, v, t)
  if (e.d1 == 0 || e.d3 == 0) { T.err |= kErrBounds; return; }  // index not built from this prefix
  // e1 and e3 from the two halves of block 1; a draw over one position is 0
  // without drawing (a wedge's dummy end, or a window of one edge)
  r1 = r3 = 0;
  if (e.d1 > 1 || e.d3 > 1) {
    const uint4 o = philox4x32_10(make_uint4((uint32_t)s, (uint32_t)(s >> 32), 1u, 0u), key);
    if ((e.d1 > 1 && !lemire_accept((uint64_t)o.x | ((uint64_t)o.y << 32), e.d1, &r1) &&
         !bounded_draw_slow(A.seed, s, 1, false, e.d1, &r1)) ||
        (e.d3 > 1 && !lemire_accept((uint64_t)o.z | ((uint64_t)o.w << 32), e.d3, &r3) &&
         !bounded_draw_slow(A.seed, s, 1, true, e.d3, &r3))) {
      T.err |= kErrRng;
      return;
    }
  }
  const uint32_t p1 = e.lo1 + (uint32_t)r1, p3 = e.lo3 + (uint32_t)r3;
  if (p1 >= A.m || p3 >= A.m) { T.err |= kErrBounds; return; }
  int32_t up, vp;
  int64_t t1, t3;
  end_edge(A, P.alpha1, p1, &up, &t1);
  end_edge(A, P.alpha3, p3, &vp, &t3);
  const uint64_t X = check_motif(A, P, up, me.src, me.dst, vp, t1, me.t, t3, s_err, &T.checked);
  if (A.h && X) {  // exact per-h bins of the proposal estimator (the block's own when it has them)
    const uint32_t hv = __ldg(A.h + lo);
    const bool local = sbins && hv - hmin < kSmemBins;  // an h outside the recorded range goes to global
    bin_add(local ? sbins + 3 * (uint64_t)(hv - hmin) : A.bins + 3 * (uint64_t)hv, X);
  }
  if (Trace) {
    A.trace[4 * i + 0] = lo;
    A.trace[4 * i + 1] = p1;
    A.trace[4 * i + 2] = p3;
    A.trace[4 * i + 3] = X;
  }
  const uint64_t nx = T.sx + X;
  if (nx < T.sx) T.err |= kErrOverflow;
  T.sx = nx;
  T.sx2 += (unsigned __int128)X * X;
  T.hits += X != 0;
}

// Proposal mode: a block accumulates the per-h bins of its samples in
// shared memory (kSmemBins consecutive h values from the proposal's
// smallest h) and adds them to the global bins once at its end, instead of
// one global atomic per hit on a few hot bins.
template <bool Trace>
__global__ void __launch_bounds__(256, TC_SAMPLE_MIN_BLOCKS) k_sample(const __grid_constant__ SamplerArgs A,
                                                const __grid_constant__ Plan P) {
  extern __shared__ unsigned long long s_bins[];  // kSmemBinBytes in proposal mode, else none
  const IndexHeader* H = A.hdr;
  const uint64_t W = H->W;
  const uint32_t shift = H->shift;
  __shared__ uint32_t s_err;
  __shared__ unsigned long long s_x, s_x2lo, s_x2hi, s_hits, s_checked;
  if (threadIdx.x == 0) {
    s_err = 0;
    s_x = s_x2lo = s_x2hi = s_hits = s_checked = 0;
  }
  uint32_t hmin = 0;
  bool local_bins = false;
  if (A.h && A.hrange) {
    hmin = A.hrange[0];
    local_bins = A.hrange[1] >= hmin;  // h beyond hmin + kSmemBins - 1 (a wider range) goes to the global bins
    if (local_bins)
      for (uint32_t b = threadIdx.x; b < 3 * kSmemBins; b += blockDim.x) s_bins[b] = 0;
  }
  __syncthreads();
  const uint32_t bad = index_check(A, P);
  if (bad) {
    if (threadIdx.x == 0) atomicOr(&A.sums->err, bad);
    return;
  }
  ThreadSums T;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < A.count && W; j += stride) {
    const uint64_t i = A.chunk_base + (A.order ? __ldg(A.order + j) : j);  // sample index within the call
    sample_one<Trace>(A, P, W, shift, i, T, &s_err, local_bins ? s_bins : nullptr, hmin);
  }
  if (local_bins) {
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < kSmemBins; b += blockDim.x) {
      const unsigned long long x = s_bins[3 * b], lo = s_bins[3 * b + 1], hi = s_bins[3 * b + 2];
      if (!x && !lo && !hi) continue;
      unsigned long long* g = A.bins + 3 * (uint64_t)(hmin + b);
      atomicAdd(g, x);
      const unsigned long long old = atomicAdd(g + 1, lo);
      const unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
      if (hi || carry) atomicAdd(g + 2, hi + carry);
    }
  }
  block_commit(A.sums, W, T.sx, T.sx2, T.hits, T.checked, T.err, s_err, s_x, s_x2lo, s_x2hi, s_hits, s_checked);
}

// Processing order of the samples.  Samples whose middle-edge draws r are
// close share records, windows and pair lists, so each chunk of samples is
// put in order of the top 16 bits of r by a two-pass most-significant-digit
// counting sort: pass A partitions the samples by the high byte of the key
// into 256 segments, pass B orders each segment by the low byte.  The order
// of samples with equal keys is free, so ranks inside a tile come from
// shared-memory atomics; tiles are staged in shared memory in digit order so
// that global writes form contiguous runs.  The first pass draws r once per
// sample and stores its 16-bit key.  Integer sums do not depend on the order.
constexpr int kBuckets = 256;
constexpr int kBucketItems = 16;
constexpr int kBucketTile = 256 * kBucketItems;

struct SegInfo {          // pass-B tiling of the 256 segments of pass A
  uint32_t start[kBuckets + 1];      // first element of each segment
  uint32_t ntiles[kBuckets];         // tiles of each segment
  uint32_t tile_base[kBuckets + 1];  // first tile of each segment
};

// Pass A histogram: draws the keys (writing them in id order) and counts
// their high bytes; hist[d * tiles + tile].
__global__ void __launch_bounds__(256) k_key_hist(const IndexHeader* __restrict__ H, uint64_t seed, uint64_t first,
                                                  uint64_t count, uint16_t* __restrict__ keys,
                                                  uint32_t* __restrict__ hist, uint32_t tiles) {
  __shared__ uint32_t cnt[kBuckets];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const uint64_t W = H->W;
  const int wbits = W > 1 ? 64 - __clzll(W - 1) : 0;
  const int drop = wbits > 16 ? wbits - 16 : 0;
  const uint64_t base = (uint64_t)blockIdx.x * kBucketTile;
#pragma unroll 4
  for (int it = 0; it < kBucketItems; it++) {
    const uint64_t j = base + (uint64_t)it * 256 + threadIdx.x;
    if (j < count) {
      uint64_t r = 0;
      if (W) bounded_draw(seed, first + j, 0, W, &r);  // a failed draw is flagged by the sampler
      const uint32_t key = (uint32_t)(r >> drop);
      keys[j] = (uint16_t)key;
      atomicAdd(&cnt[key >> 8], 1u);
    }
  }
  __syncthreads();
  hist[(uint64_t)threadIdx.x * tiles + blockIdx.x] = cnt[threadIdx.x];
}

// Scatter the elements [lo, hi) of one tile by digit (key >> shift) & 255 to
// out_base[d] + rank, staging the tile in shared memory in digit order.
// ids_in == NULL means the element's own position.
__device__ __forceinline__ void tile_scatter(uint32_t lo, uint32_t hi, const uint16_t* __restrict__ keys_in,
                                             const uint32_t* __restrict__ ids_in, int shift,
                                             const uint32_t* s_out_base, uint16_t* __restrict__ keys_out,
                                             uint32_t* __restrict__ ids_out, uint32_t* cnt, uint32_t* start,
                                             uint32_t* warp_tot, uint32_t* stage, uint16_t* stage_k) {
  cnt[threadIdx.x] = 0;
  __syncthreads();
  // key (16 bits) and rank within the tile (< kBucketTile) packed in one
  // register per item; the ids are loaded up front with the keys
  uint32_t kr[kBucketItems], id[kBucketItems];
#pragma unroll
  for (int it = 0; it < kBucketItems; it++) {
    const uint32_t j = lo + (uint32_t)it * 256 + threadIdx.x;
    kr[it] = 0xFFFFFFFFu;
    if (j < hi) {
      kr[it] = (uint32_t)__ldg(keys_in + j) << 16;
      id[it] = ids_in ? __ldg(ids_in + j) : j;
    }
  }
#pragma unroll
  for (int it = 0; it < kBucketItems; it++)
    if (kr[it] != 0xFFFFFFFFu) kr[it] |= atomicAdd(&cnt[((kr[it] >> 16) >> shift) & 255u], 1u);
  __syncthreads();
  {  // exclusive scan of the tile's digit counts
    const uint32_t v = cnt[threadIdx.x];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < wid; w++) before += warp_tot[w];
    start[threadIdx.x] = before + inc - v;
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < kBucketItems; it++) {
    if (kr[it] != 0xFFFFFFFFu) {
      const uint32_t key = kr[it] >> 16;
      const uint32_t p = start[(key >> shift) & 255u] + (kr[it] & 0xFFFFu);
      stage[p] = id[it];
      stage_k[p] = (uint16_t)key;
    }
  }
  __syncthreads();
  const uint32_t n = hi - lo;
  for (uint32_t i = threadIdx.x; i < n; i += 256) {
    const uint32_t kk = stage_k[i];
    const uint32_t d = (kk >> shift) & 255u;
    const uint32_t g = s_out_base[d] + (i - start[d]);
    ids_out[g] = stage[i];
    if (keys_out) keys_out[g] = (uint16_t)kk;
  }
}

// Pass A scatter: tile t of the chunk, by the high byte.
__global__ void __launch_bounds__(256, 6) k_key_scatter_a(uint64_t count, const uint16_t* __restrict__ keys,
                                                       const uint32_t* __restrict__ offs, uint32_t tiles,
                                                       uint16_t* __restrict__ keys_out,
                                                       uint32_t* __restrict__ ids_out) {
  __shared__ uint32_t cnt[kBuckets], start[kBuckets], base_s[kBuckets], warp_tot[8];
  __shared__ uint32_t stage[kBucketTile];
  __shared__ uint16_t stage_k[kBucketTile];
  base_s[threadIdx.x] = offs[(uint64_t)threadIdx.x * tiles + blockIdx.x];
  const uint64_t lo = (uint64_t)blockIdx.x * kBucketTile;
  const uint64_t hi = lo + kBucketTile < count ? lo + kBucketTile : count;
  tile_scatter((uint32_t)lo, (uint32_t)hi, keys, nullptr, 8, base_s, keys_out, ids_out, cnt, start, warp_tot, stage,
               stage_k);
}

// Segment sizes from the scanned pass-A histogram and the pass-B tiling.
__global__ void k_seg_info(const uint32_t* __restrict__ offs, uint32_t tiles, uint64_t count, SegInfo* info) {
  __shared__ uint32_t nt[kBuckets + 1];
  const int d = threadIdx.x;
  const uint32_t s0 = offs[(uint64_t)d * tiles];
  const uint32_t s1 = d + 1 < kBuckets ? offs[(uint64_t)(d + 1) * tiles] : (uint32_t)count;
  info->start[d] = s0;
  if (d == kBuckets - 1) info->start[kBuckets] = (uint32_t)count;
  nt[d] = (s1 - s0 + kBucketTile - 1) / kBucketTile;
  info->ntiles[d] = nt[d];
  __syncthreads();
  if (d == 0) {
    uint32_t run = 0;
    for (int i = 0; i < kBuckets; i++) {
      info->tile_base[i] = run;
      run += nt[i];
    }
    info->tile_base[kBuckets] = run;
  }
}

// Segment and tile of pass-B block b (false past the last tile).
__device__ __forceinline__ bool seg_tile(const SegInfo* info, uint32_t b, uint32_t* seg, uint32_t* t) {
  if (b >= info->tile_base[kBuckets]) return false;
  uint32_t lo = 0, hi = kBuckets - 1;  // last segment with tile_base <= b
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (info->tile_base[mid] <= b) lo = mid; else hi = mid - 1;
  }
  *seg = lo;
  *t = b - info->tile_base[lo];
  return true;
}

// Pass B: histogram of the low byte per (segment, digit, tile) at
// tile_base[s] * 256 + d * ntiles[s] + t, so that one flat exclusive scan
// gives every element's final position.
__global__ void __launch_bounds__(256) k_key_hist_b(const uint16_t* __restrict__ keys, const SegInfo* __restrict__ info,
                                                    uint32_t* __restrict__ hist) {
  __shared__ uint32_t cnt[kBuckets];
  uint32_t seg, t;
  if (!seg_tile(info, blockIdx.x, &seg, &t)) return;
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t lo = info->start[seg] + t * kBucketTile;
  const uint32_t end = info->start[seg + 1];
  const uint32_t hi = lo + kBucketTile < end ? lo + kBucketTile : end;
  for (uint32_t j = lo + threadIdx.x; j < hi; j += 256) atomicAdd(&cnt[__ldg(keys + j) & 255u], 1u);
  __syncthreads();
  hist[(uint64_t)info->tile_base[seg] * kBuckets + (uint64_t)threadIdx.x * info->ntiles[seg] + t] = cnt[threadIdx.x];
}

__global__ void __launch_bounds__(256, 5) k_key_scatter_b(const uint16_t* __restrict__ keys,
                                                       const uint32_t* __restrict__ ids,
                                                       const SegInfo* __restrict__ info,
                                                       const uint32_t* __restrict__ offs,
                                                       uint32_t* __restrict__ ids_out) {
  __shared__ uint32_t cnt[kBuckets], start[kBuckets], base_s[kBuckets], warp_tot[8];
  __shared__ uint32_t stage[kBucketTile];
  __shared__ uint16_t stage_k[kBucketTile];
  uint32_t seg, t;
  if (!seg_tile(info, blockIdx.x, &seg, &t)) return;
  base_s[threadIdx.x] = offs[(uint64_t)info->tile_base[seg] * kBuckets + (uint64_t)threadIdx.x * info->ntiles[seg] + t];
  const uint32_t lo = info->start[seg] + t * kBucketTile;
  const uint32_t end = info->start[seg + 1];
  const uint32_t hi = lo + kBucketTile < end ? lo + kBucketTile : end;
  tile_scatter(lo, hi, keys, ids, 0, base_s, nullptr, ids_out, cnt, start, warp_tot, stage, stage_k);
}

// Scratch layout of sort_sample_ids for count samples: ids after pass A,
// keys in id order and after pass A, the digit histogram, the segment tiling
// and the histogram scan's tile sums.
struct SortScratch {
  uint32_t tiles, tiles_b;
  size_t ids_a, keys_0, keys_a, hist, info, scan, bytes;  // byte offsets; total
  uint64_t scan_words;
};

static SortScratch sort_scratch(uint64_t count) {
  SortScratch L;
  L.tiles = (uint32_t)((count + kBucketTile - 1) / kBucketTile);
  L.tiles_b = L.tiles + kBuckets;
  const uint64_t cap = (uint64_t)L.tiles * kBucketTile;
  L.scan_words = scan_u64_scratch_words((uint64_t)kBuckets * L.tiles_b) + 1;
  size_t p = 0;
  L.ids_a = p;
  p += align256(4 * cap);
  L.keys_0 = p;
  p += align256(2 * cap);
  L.keys_a = p;
  p += align256(2 * cap);
  L.hist = p;
  p += align256(4 * ((uint64_t)kBuckets * L.tiles_b + 1));
  L.info = p;
  p += align256(sizeof(SegInfo));
  L.scan = p;
  p += align256(4 * L.scan_words);
  L.bytes = p;
  return L;
}

size_t sort_scratch_bytes(uint64_t count) { return sort_scratch(count).bytes; }

// Writes the indices 0..count-1 of samples first..first+count-1 into order
// in key order (top 16 bits of each sample's middle-edge draw), using only
// the given scratch of sort_scratch_bytes(count) bytes (no allocation).
tc_status sort_sample_ids(const IndexHeader* hdr, uint64_t seed, uint64_t first, uint64_t count, void* scratch,
                          uint32_t* order, cudaStream_t st) {
  const SortScratch L = sort_scratch(count);
  const uint32_t tiles = L.tiles, tiles_b = L.tiles_b;
  char* base = (char*)scratch;
  uint32_t* ids_a = (uint32_t*)(base + L.ids_a);
  uint16_t* keys_0 = (uint16_t*)(base + L.keys_0);
  uint16_t* keys_a = (uint16_t*)(base + L.keys_a);
  uint32_t* hist = (uint32_t*)(base + L.hist);
  SegInfo* info = (SegInfo*)(base + L.info);
  uint32_t* scan_scratch = (uint32_t*)(base + L.scan);
  const uint64_t scan_words = L.scan_words;
  tc_status s = TC_OK;
  auto ok = [&](const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) s = cuda_status(e, what);
    return s == TC_OK;
  };
  k_key_hist<<<tiles, 256, 0, st>>>(hdr, seed, first, count, keys_0, hist, tiles);
  TC_LAUNCHED(1);
  if (!ok("k_key_hist")) return s;
  TC_TRY(scan_u32_in_scratch(hist, hist, (uint64_t)kBuckets * tiles, scan_scratch, scan_words, st));
  k_key_scatter_a<<<tiles, 256, 0, st>>>(count, keys_0, hist, tiles, keys_a, ids_a);
  TC_LAUNCHED(1);
  if (!ok("k_key_scatter_a")) return s;
  k_seg_info<<<1, kBuckets, 0, st>>>(hist, tiles, count, info);
  TC_LAUNCHED(1);
  if (!ok("k_seg_info")) return s;
  TC_CUDA(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * (size_t)kBuckets * tiles_b, st));
  k_key_hist_b<<<tiles_b, 256, 0, st>>>(keys_a, info, hist);
  TC_LAUNCHED(1);
  if (!ok("k_key_hist_b")) return s;
  TC_TRY(scan_u32_in_scratch(hist, hist, (uint64_t)kBuckets * tiles_b, scan_scratch, scan_words, st));
  k_key_scatter_b<<<tiles_b, 256, 0, st>>>(keys_a, ids_a, info, hist, order);
  TC_LAUNCHED(1);
  ok("k_key_scatter_b");
  return s;
}

// Diagnostic timing by phase (tc_set_timing): event pairs around the
// launches of a phase, recorded on the launching stream and summed when the
// caller asks.  A call that runs a phase first drops that phase's events of
// the previous call.
static thread_local bool t_timing = false;
static thread_local std::vector<std::pair<cudaEvent_t, cudaEvent_t>> t_events[kNumPhases];

PhaseTimer::PhaseTimer(int phase, cudaStream_t s) : ph(phase), st(s) {
  if (!t_timing) return;
  for (auto& e : t_events[ph]) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  t_events[ph].clear();
}

void PhaseTimer::start() {
  if (!t_timing) return;
  std::pair<cudaEvent_t, cudaEvent_t> e{nullptr, nullptr};
  if (cudaEventCreate(&e.first) != cudaSuccess) return;
  if (cudaEventCreate(&e.second) != cudaSuccess) {
    cudaEventDestroy(e.first);
    return;
  }
  cudaEventRecord(e.first, st);
  t_events[ph].push_back(e);
}

void PhaseTimer::stop() {
  if (t_timing && !t_events[ph].empty()) cudaEventRecord(t_events[ph].back().second, st);
}

void set_timing(bool on) { t_timing = on; }

float last_phase_ms(int phase) {
  if (phase < 0 || phase >= kNumPhases) return 0.f;
  float total = 0.f;
  for (auto& e : t_events[phase]) {
    float ms = 0.f;
    if (cudaEventSynchronize(e.second) == cudaSuccess && cudaEventElapsedTime(&ms, e.first, e.second) == cudaSuccess)
      total += ms;
  }
  return total;
}

float last_sampler_ms() { return last_phase_ms(TC_PHASE_SAMPLE); }

tc_status launch_sampler(const tc_graph* g, const Plan& plan, int64_t delta, const uint64_t* prefix,
                         const void* index, uint64_t k, uint64_t seed, uint64_t offset, uint64_t* trace,
                         SampleSums* d_sums, cudaStream_t st, const void* qindex, const uint16_t* h,
                         unsigned long long* bins) {
  const uint64_t m = (uint64_t)g->m;
  IndexView v = index_view(const_cast<void*>(index), m);
  const IndexHeader* rec_hdr = nullptr;
  if (h) {  // the proposal's header and guide replace the plain ones
    rec_hdr = v.hdr;
    v.hdr = (IndexHeader*)qindex;
    v.guide = (uint32_t*)((char*)const_cast<void*>(qindex) + kIndexHeaderBytes);
  }
  SamplerArgs A;
  A.out_e = g->out_e;
  A.in_e = g->in_e;
  A.pair_hash = g->pair_hash;
  A.hash_mask = g->hash_mask;
  A.pair_t = g->pair_t;
  A.pair_t32 = TC_COMPACT_PAIRS ? g->pair_t32 : nullptr;
  A.tmin = g->tmin;
  A.prefix = prefix;
  A.hdr = v.hdr;
  A.win = v.win;
  A.guide = v.guide;
  A.k = k;
  A.order = nullptr;
  A.chunk_base = 0;
  A.count = k;
  A.m = (uint32_t)m;
  A.seed = seed;
  A.offset = offset;
  A.delta = delta;
  A.graph_id = g->id;
  A.trace = trace;
  A.sums = d_sums;
  A.h = h;
  A.bins = bins;
  A.hrange = h ? (const uint32_t*)((const char*)qindex + kProposalRangeOffset) : nullptr;
  A.rec_hdr = rec_hdr;
  static int blocks_per_sm[2] = {0, 0};
  const int ti = trace ? 1 : 0;
  if (!blocks_per_sm[ti]) {
    int b = 0;
    if (trace)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_sample<true>, 256, kSmemBinBytes);
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_sample<false>, 256, kSmemBinBytes);
    blocks_per_sm[ti] = b > 0 ? b : 1;
  }
  const uint64_t max_blocks = (uint64_t)num_sms() * blocks_per_sm[ti];
  auto run = [&](const uint32_t* order, uint64_t base, uint64_t count) -> tc_status {
    A.order = order;
    A.chunk_base = base;
    A.count = count;
    uint64_t blocks = max_blocks;
    const uint64_t need = (count + 255) / 256;
    if (need < blocks) blocks = need ? need : 1;
    const size_t dyn = h ? kSmemBinBytes : 0;
    if (trace)
      k_sample<true><<<(unsigned)blocks, 256, dyn, st>>>(A, plan);
    else
      k_sample<false><<<(unsigned)blocks, 256, dyn, st>>>(A, plan);
    TC_LAUNCHED(1);
    TC_CUDA(cudaGetLastError());
    return TC_OK;
  };
  PhaseTimer timer(TC_PHASE_SAMPLE, st), sort_timer(TC_PHASE_ORDER, st);
  if (k < kSortedMinSamples) {
    timer.start();
    tc_status s = run(nullptr, 0, k);
    timer.stop();
    return s;
  }
  // samples in chunks; each chunk is put in key order first
  const uint64_t chunk = k < kChunkSamples ? k : kChunkSamples;
  const size_t sbytes = sort_scratch_bytes(chunk);
  char* buf = nullptr;
  TC_CUDA(pool_malloc(&buf, sbytes + 4 * chunk, st));
  uint32_t* order = (uint32_t*)(buf + sbytes);
  tc_status s = TC_OK;
  for (uint64_t base = 0; base < k && s == TC_OK; base += chunk) {
    const uint64_t count = (k - base) < chunk ? (k - base) : chunk;
    sort_timer.start();
    s = sort_sample_ids(v.hdr, seed, offset + base, count, buf, order, st);
    sort_timer.stop();
    timer.start();
    if (s == TC_OK) s = run(order, base, count);
    timer.stop();
  }
  cudaFreeAsync(buf, st);
  return s;
}

tc_status launch_path_sum(const tc_graph* g, const Plan& plan, int64_t delta, const uint64_t* prefix,
                          const void* index, uint64_t W, SampleSums* d_sums, cudaStream_t st) {
  const uint64_t m = (uint64_t)g->m;
  IndexView v = index_view(const_cast<void*>(index), m);
  SamplerArgs A;
  std::memset(&A, 0, sizeof(A));
  A.out_e = g->out_e;
  A.in_e = g->in_e;
  A.pair_hash = g->pair_hash;
  A.hash_mask = g->hash_mask;
  A.pair_t = g->pair_t;
  A.pair_t32 = TC_COMPACT_PAIRS ? g->pair_t32 : nullptr;
  A.tmin = g->tmin;
  A.prefix = prefix;
  A.hdr = v.hdr;
  A.win = v.win;
  A.guide = v.guide;
  A.m = (uint32_t)m;
  A.delta = delta;
  A.graph_id = g->id;
  A.sums = d_sums;
  int bps = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_path_sum, 256, 0);
  uint64_t blocks = (uint64_t)num_sms() * (bps > 0 ? bps : 1);
  const uint64_t need = (W + 255) / 256;
  if (need < blocks) blocks = need ? need : 1;
  k_path_sum<<<(unsigned)blocks, 256, 0, st>>>(A, plan, 0, W);
  TC_LAUNCHED(1);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

// ---------------------------------------------------------------------------
// Batched sampling: one persistent launch over the tiles of many queries
// (graphs, motifs, windows).  Each block takes the next work item from a
// global counter; items are numbered query after query, so a block sees
// its queries in increasing order, keeps per-thread sums while the query
// stays the same and commits them to that query's sums when it changes.
// A query's samples and sums are those of the same query run alone.

struct alignas(16) BatchQuery {
  SamplerArgs A;
  Plan P;
};
static_assert(sizeof(BatchQuery) <= kBatchQueryBytes, "batch record too large");
static_assert(kBatchQueryBytes % 16 == 0, "batch record must be whole 16-byte words");

void batch_query_record(void* h_rec, const tc_graph* g, const Plan& plan, int64_t delta, const uint64_t* prefix,
                        const void* index, uint64_t k, uint64_t seed, uint64_t offset, const uint32_t* order) {
  std::memset(h_rec, 0, kBatchQueryBytes);
  BatchQuery* Q = (BatchQuery*)h_rec;
  const uint64_t m = (uint64_t)g->m;
  IndexView v = index_view(const_cast<void*>(index), m);
  SamplerArgs& A = Q->A;
  A.out_e = g->out_e;
  A.in_e = g->in_e;
  A.pair_hash = g->pair_hash;
  A.hash_mask = g->hash_mask;
  A.pair_t = g->pair_t;
  A.pair_t32 = TC_COMPACT_PAIRS ? g->pair_t32 : nullptr;
  A.tmin = g->tmin;
  A.prefix = prefix;
  A.hdr = v.hdr;
  A.win = v.win;
  A.guide = v.guide;
  A.k = k;
  A.seed = seed;
  A.offset = offset;
  A.order = order;
  A.chunk_base = 0;
  A.count = k;
  A.m = (uint32_t)m;
  A.delta = delta;
  A.graph_id = g->id;
  Q->P = plan;
}

template <int BS>
__global__ void __launch_bounds__(BS, (256 * TC_SAMPLE_MIN_BLOCKS) / BS)
    k_sample_batch(const char* __restrict__ records, const uint64_t* __restrict__ tile_begin, uint32_t nq,
                   uint32_t tile, unsigned long long* __restrict__ next_item, SampleSums* __restrict__ sums) {
  __shared__ BatchQuery s_q;
  __shared__ unsigned long long s_item;
  __shared__ uint32_t s_query;
  __shared__ uint32_t s_err;
  __shared__ unsigned long long s_x, s_x2lo, s_x2hi, s_hits, s_checked;
  if (threadIdx.x == 0) {
    s_err = 0;
    s_x = s_x2lo = s_x2hi = s_hits = s_checked = 0;
  }
  const uint64_t total = tile_begin[nq];
  uint32_t cur = 0xFFFFFFFFu, bad = 0, shift = 0;
  uint64_t W = 0;
  ThreadSums T;
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned long long item = atomicAdd(next_item, 1ull);
      uint32_t q = nq;
      if (item < total) {  // the last query whose first item is <= item
        uint32_t lo = 0, hi = nq - 1;
        while (lo < hi) {
          const uint32_t mid = (lo + hi + 1) >> 1;
          if (tile_begin[mid] <= item) lo = mid; else hi = mid - 1;
        }
        q = lo;
      }
      s_item = item;
      s_query = q;
    }
    __syncthreads();
    const uint64_t item = s_item;
    const uint32_t q = s_query;
    if (q != cur) {  // block-uniform
      if (cur != 0xFFFFFFFFu && !bad) {
        block_commit(sums + cur, W, T.sx, T.sx2, T.hits, T.checked, T.err, s_err, s_x, s_x2lo, s_x2hi, s_hits,
                     s_checked);
        T = ThreadSums();
        if (threadIdx.x == 0) {
          s_err = 0;
          s_x = s_x2lo = s_x2hi = s_hits = s_checked = 0;
        }
      }
      if (q >= nq) break;
      // the records are kBatchQueryBytes apart
      const uint4* src = reinterpret_cast<const uint4*>(records + (uint64_t)q * kBatchQueryBytes);
      uint4* dst = reinterpret_cast<uint4*>(&s_q);
      for (uint32_t w = threadIdx.x; w < sizeof(BatchQuery) / 16; w += BS) dst[w] = src[w];
      __syncthreads();
      cur = q;
      bad = index_check(s_q.A, s_q.P);
      W = s_q.A.hdr->W;
      shift = s_q.A.hdr->shift;
      if (bad && threadIdx.x == 0) atomicOr(&sums[q].err, bad);
    }
    if (!bad && W) {
      const uint64_t j0 = (item - tile_begin[q]) * tile;
      const uint64_t j1 = j0 + tile < s_q.A.count ? j0 + tile : s_q.A.count;
      const uint32_t* order = s_q.A.order;
      for (uint64_t j = j0 + threadIdx.x; j < j1; j += BS) {
        const uint64_t i = order ? (j & ~(kChunkSamples - 1)) + __ldg(order + j) : j;
        sample_one<false>(s_q.A, s_q.P, W, shift, i, T, &s_err);
      }
    }
    __syncthreads();
  }
}

int sample_batch_blocks_per_sm(int bs) {
  static int cache[3] = {0, 0, 0};
  const int i = bs == 128 ? 0 : bs == 256 ? 1 : bs == 512 ? 2 : -1;
  if (i < 0) return 0;
  if (!cache[i]) {
    int b = 0;
    if (bs == 128) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_sample_batch<128>, 128, 0);
    if (bs == 256) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_sample_batch<256>, 256, 0);
    if (bs == 512) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_sample_batch<512>, 512, 0);
    cache[i] = b > 0 ? b : 1;
  }
  return cache[i];
}

tc_status launch_sample_batch(int bs, uint32_t tile, unsigned blocks, const void* d_records,
                              const uint64_t* d_tile_begin, uint32_t nq, unsigned long long* d_next_item,
                              SampleSums* d_sums, cudaStream_t st) {
  const char* Q = (const char*)d_records;
  if (bs == 128)
    k_sample_batch<128><<<blocks, 128, 0, st>>>(Q, d_tile_begin, nq, tile, d_next_item, d_sums);
  else if (bs == 256)
    k_sample_batch<256><<<blocks, 256, 0, st>>>(Q, d_tile_begin, nq, tile, d_next_item, d_sums);
  else if (bs == 512)
    k_sample_batch<512><<<blocks, 512, 0, st>>>(Q, d_tile_begin, nq, tile, d_next_item, d_sums);
  else
    return set_error(TC_ERR_INVALID_ARG, "batch block size must be 128, 256 or 512");
  TC_LAUNCHED(1);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

}  // namespace tc
