// Internal declarations of the tc library (device layouts, launch helpers).
// Not part of the ABI; include/tc.h is.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/tc.h"

namespace tc {

// ---------------------------------------------------------------------------
// Device layouts.  Edge positions are uint32 (m < 2^32 - 1), vertex ids int32.

struct __align__(16) OutEdge {  // canonical order = out-lists sorted by (src, t, input index)
  int32_t src;
  int32_t dst;
  int64_t t;
};

struct __align__(16) InEdge {  // in-lists sorted by (dst, t, input index)
  int32_t src;
  int32_t dst;
  int64_t t;
};

// Both end-edge windows of a canonical middle edge (Alg. 2), one 16-byte
// entry per edge of the sampling index; the edge itself is out_e.
struct __align__(16) EdgeWin {
  uint32_t lo1, d1;  // window of e1: positions [lo1, lo1 + d1) of u's alpha1 list
  uint32_t lo3, d3;  // window of e3: positions [lo3, lo3 + d3) of v's alpha3 list
};

// Range word of a position a of the list [s, f): (min(a - s, 0xFFFF) << 16)
// | min(f - a, 0xFFFF).  A field below 0xFFFF is the exact distance; 0xFFFF
// means at least that far (the search then reads the list's offsets).
constexpr uint32_t kRangeCap = 0xFFFFu;
__host__ __device__ __forceinline__ uint32_t range_word(uint32_t a, uint32_t s, uint32_t f) {
  const uint32_t ls = a - s < kRangeCap ? a - s : kRangeCap;
  const uint32_t lf = f - a < kRangeCap ? f - a : kRangeCap;
  return (ls << 16) | lf;
}

// Slot of the pair hash table: the pair list L_{x,y} occupies positions
// [begin, end) of pair_t.  Empty slots have x = y = 0xFFFFFFFF.
struct __align__(16) PairSlot {
  uint32_t x, y;
  uint32_t begin, end;
};
constexpr unsigned long long kEmptyPairKey = 0xFFFFFFFFFFFFFFFFull;

// 64-bit finaliser of SplitMix64 (Steele, Lea, Flood, OOPSLA 2014).
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t pair_key(uint32_t x, uint32_t y) {
  return (uint64_t)x | ((uint64_t)y << 32);  // little-endian image of {x, y}
}

constexpr uint64_t kIndexMagic = 0x7463696e64657831ull;  // "tcindex1"
constexpr size_t kIndexHeaderBytes = 256;
// A proposal index keeps its smallest and largest h (uint32 each) at this
// offset of its header, after the IndexHeader fields.
constexpr size_t kProposalRangeOffset = 192;

// Header at the start of a sampling index; written on the device by the guide
// kernel so that sampling needs no host round trip.
struct IndexHeader {
  uint64_t magic;
  uint64_t W;
  uint64_t m;
  uint32_t shift;    // guide bucket b covers [b << shift, (b + 1) << shift)
  uint32_t nb;       // buckets; guide has nb + 1 entries
  int32_t cls[4];    // alpha1, alpha3, beta1, beta3 (+-1)
  int32_t closed;
  int32_t anchor[3];
  int64_t delta;
  uint64_t graph_id;
  uint32_t status;   // device error bits of the weights and prefix pass
};
static_assert(sizeof(IndexHeader) <= 192, "the proposal's h range follows the header fields");

// Device error bits, reduced into a status at the next synchronisation.
enum : uint32_t {
  kErrOverflow = 1u << 0,
  kErrRng = 1u << 1,
  kErrBounds = 1u << 2,
  kErrBadId = 1u << 3,
  kErrIndexMismatch = 1u << 4,
  kErrTimeout = 1u << 5,
};

// ---------------------------------------------------------------------------
// Compiled motif: anchor, class and the non-anchor edges grouped by gap.

// A 3-vertex motif has a wedge anchor (wedge != 0): the base edge (motif
// edge 0) is stored as the middle edge and the second edge as e1 (wedge 1:
// it shares the base's source u) or e3 (wedge 2: it shares the base's
// destination v), with beta = +1; the unused end has index -1, alpha = beta
// = 0 (a dummy window of one position) and label -1.  Gaps: ranks between
// the base and the second edge, and after the second edge.
struct Plan {
  int32_t r;                 // motif edges
  int32_t e1, mid, e3;       // anchor motif edge indices (= time ranks)
  int32_t alpha1, alpha3;    // -1 in-list, +1 out-list, 0 none (wedge)
  int32_t beta1, beta3;      // -1 before the middle edge, +1 after
  int32_t closed;            // 1: closed windows
  int32_t wedge;             // 0: 3-path anchor; 1 or 2: wedge anchor
  int32_t lab[4];            // motif labels of u', u, v, v'
  int32_t rk[3];             // anchor ranks sorted ascending (rk[0] = 0)
  int32_t ngap[3];           // non-anchor lists per gap
  int8_t gx[3][16], gy[3][16];  // path roles (0 u', 1 u, 2 v, 3 v') of the
                                // endpoints of those lists, in rank order
};

tc_status compile_plan(const tc_motif* motif, Plan* plan, std::string* why);

// ---------------------------------------------------------------------------
// Graph object.

}  // namespace tc

struct tc_graph {
  int64_t n, m, P;
  int64_t tmin, tmax;
  int device;
  uint64_t id;
  uint32_t* out_off;
  tc::OutEdge* out_e;
  uint32_t* perm;
  uint32_t* in_off;
  tc::InEdge* in_e;
  uint32_t* in_eid;  // in-list position -> canonical position
  uint32_t* pair_off;
  int32_t* pair_dst;
  uint32_t* pair_eoff;
  int64_t* pair_t;
  uint32_t* pair_eid;
  tc::PairSlot* pair_hash;  // open addressing, linear probing, load <= 1/2
  uint64_t hash_mask;       // capacity - 1 (capacity a power of two)
  // times of the out- and in-lists as t - tmin in 32 bits, when the time
  // span fits (else NULL): the window searches probe 4-byte entries, eight
  // per 32-byte sector
  uint32_t* out_t32;
  uint32_t* in_t32;
  uint32_t* pair_t32;  // pair-list times as t - tmin (same condition)
  // Anchors of the window searches, per canonical edge e = (u, v, t),
  // independent of delta and of the motif: positions in the concatenated
  // lists where u's in-list and v's out-list reach time t (the first entry
  // with time >= t), and e's own position in v's in-list.
  uint32_t* x_in;    // first position p in u's in-list with in_e[p].t >= t
  uint32_t* x_out;   // first position p in v's out-list with out_e[p].t >= t
  uint32_t* out2in;  // canonical position -> in-list position (inverse of in_eid)
  // Range words of the anchors (tc::range_word): how far the anchor lies
  // from the start and the end of its list, so that a window search needs
  // no load of the list's offsets unless it runs beyond 65,534 entries.
  uint32_t* r_in;    // x_in[e] in u's in-list
  uint32_t* r_out;   // x_out[e] in v's out-list
  uint32_t* r_o2i;   // out2in[e] in v's in-list
  uint32_t* r_self;  // e itself in u's out-list
};

namespace tc {

// ---------------------------------------------------------------------------
// Errors (thread-local message, see tc_last_error).

tc_status set_error(tc_status st, const std::string& msg);

// Stream-ordered allocation from a pool owned by the library (one per
// device) that keeps freed memory for reuse instead of returning it to the
// system at every synchronisation.
cudaError_t pool_malloc(void** p, size_t bytes, cudaStream_t st);
template <class T>
inline cudaError_t pool_malloc(T** p, size_t bytes, cudaStream_t st) {
  return pool_malloc(reinterpret_cast<void**>(p), bytes, st);
}
tc_status cuda_status(cudaError_t e, const char* what);
tc_status device_status(uint32_t bits, const char* what);

#define TC_CUDA(call)                                         \
  do {                                                        \
    cudaError_t _e = (call);                                  \
    if (_e != cudaSuccess) return ::tc::cuda_status(_e, #call); \
  } while (0)

#define TC_TRY(call)                    \
  do {                                  \
    tc_status _s = (call);              \
    if (_s != TC_OK) return _s;         \
  } while (0)

inline int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

// Launch counter behind tc_kernel_launches(); every launch site bumps it.
void note_launches(unsigned count);
#define TC_LAUNCHED(n) ::tc::note_launches(n)

inline int bitlen64(uint64_t x) { return x ? 64 - __builtin_clzll(x) : 0; }

// ---------------------------------------------------------------------------
// Device helpers.

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32 -> 64-bit products with multipliers 0xD2511F53, 0xCD9E8D57 and Weyl
// key increments 0x9E3779B9, 0xBB67AE85.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int i = 0; i < 10; i++) {
    const uint32_t p0hi = __umulhi(0xD2511F53u, c.x), p0lo = 0xD2511F53u * c.x;
    const uint32_t p1hi = __umulhi(0xCD9E8D57u, c.z), p1lo = 0xCD9E8D57u * c.z;
    c = make_uint4(p1hi ^ c.y ^ k.x, p1lo, p0hi ^ c.w ^ k.y, p0lo);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// Uniform integer in [0, range), range >= 1 (Lemire, "Fast random integer
// generation in an interval", ACM TOMACS 2019): x * range = hi:lo, accept
// when lo >= 2^64 mod range, answer hi.  Attempt a draws Philox with counter
// (s_lo, s_hi, draw, a).  Returns false after 64 rejected attempts.
// Lemire's test for one 64-bit word x: accepted when x * range mod 2^64 is
// at least 2^64 mod range (always when it is at least range).
__device__ __forceinline__ bool lemire_accept(uint64_t x, uint64_t range, uint64_t* out) {
  const uint64_t lo = x * range;
  if (lo < range && lo < (0ull - range) % range) return false;
  *out = __umul64hi(x, range);
  return true;
}

// x from words 0-1 (upper: words 2-3) of block (s, draw, attempt).
__device__ __forceinline__ bool bounded_draw_words(uint64_t seed, uint64_t s, uint32_t draw, bool upper,
                                                   uint64_t range, uint64_t* out) {
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  for (uint32_t a = 0; a < 64; a++) {
    const uint4 o = philox4x32_10(make_uint4((uint32_t)s, (uint32_t)(s >> 32), draw, a), key);
    const uint64_t x = upper ? ((uint64_t)o.z | ((uint64_t)o.w << 32)) : ((uint64_t)o.x | ((uint64_t)o.y << 32));
    if (lemire_accept(x, range, out)) return true;
  }
  return false;
}

__device__ __forceinline__ bool bounded_draw(uint64_t seed, uint64_t s, uint32_t draw, uint64_t range,
                                             uint64_t* out) {
  return bounded_draw_words(seed, s, draw, false, range, out);
}

__device__ __forceinline__ int64_t sat_add(int64_t a, int64_t d) {
  return (a > INT64_MAX - d) ? INT64_MAX : a + d;
}
__device__ __forceinline__ int64_t sat_sub(int64_t a, int64_t d) {
  return (a < INT64_MIN + d) ? INT64_MIN : a - d;
}

// First position p in [lo, hi) with time(p) >= x (Ge) or > x (!Ge).
template <bool Ge, class TimeAt>
__device__ __forceinline__ uint32_t search_time(uint32_t lo, uint32_t hi, int64_t x, TimeAt time_at) {
  while (lo < hi) {
    const uint32_t mid = lo + ((hi - lo) >> 1);
    const int64_t tm = time_at(mid);
    if (Ge ? (tm < x) : (tm <= x)) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Window of x's list (alpha < 0: in-list, else out-list) around time t
// (beta < 0: before, else after; strict or closed at t) as positions [lo, hi).
// The two bounds are searched independently so that their loads overlap.
// Compact: the list times are read from the 32-bit arrays (t - tmin).
template <bool Compact>
__device__ __forceinline__ void window_range(const OutEdge* __restrict__ out_e,
                                             const uint32_t* __restrict__ out_off,
                                             const InEdge* __restrict__ in_e,
                                             const uint32_t* __restrict__ in_off,
                                             const uint32_t* __restrict__ out_t32,
                                             const uint32_t* __restrict__ in_t32, int64_t tmin, int alpha,
                                             int beta, int closed, int32_t x, int64_t t, int64_t delta,
                                             uint32_t* lo, uint32_t* hi) {
  const bool in = alpha < 0;
  const uint32_t a = __ldg((in ? in_off : out_off) + x), b = __ldg((in ? in_off : out_off) + x + 1);
  const uint32_t* t32 = in ? in_t32 : out_t32;
  auto tt = [&](uint32_t p) -> int64_t {
    if (Compact) return (int64_t)__ldg(t32 + p) + tmin;
    return in ? in_e[p].t : out_e[p].t;
  };
  if (beta < 0) {
    *lo = search_time<true>(a, b, sat_sub(t, delta), tt);
    *hi = closed ? search_time<false>(a, b, t, tt) : search_time<true>(a, b, t, tt);
  } else {
    *lo = closed ? search_time<true>(a, b, t, tt) : search_time<false>(a, b, t, tt);
    *hi = search_time<false>(a, b, sat_add(t, delta), tt);
  }
}

// ---------------------------------------------------------------------------
// Host-side launchers (defined in the .cu files).

// Exclusive scans.  scan_u64 writes out[0..n] (out[n] = total) and sets
// kErrOverflow in *d_err when the total exceeds 64 bits.  in and out must
// not overlap unless in == out.
tc_status scan_u64(const uint64_t* in, uint64_t* out, uint64_t n, uint32_t* d_err, cudaStream_t st);
tc_status scan_u32(const uint32_t* in, uint32_t* out, uint64_t n, cudaStream_t st);
uint64_t scan_u64_scratch_words(uint64_t n);  // also the element count for u32 scans
tc_status scan_u32_in_scratch(const uint32_t* in, uint32_t* out, uint64_t n, uint32_t* scratch,
                              uint64_t scratch_words, cudaStream_t st);
tc_status scan_u64_in_scratch(const uint64_t* in, uint64_t* out, uint64_t n, bool write_total, uint32_t* d_err,
                              uint64_t* scratch, uint64_t scratch_words, cudaStream_t st);
// The same scan when the kernel that wrote `in` also wrote the sums of its
// tiles of scan_tile_size() values into sums[ceil(n / scan_tile_size())]
// (scanned in place; scratch: scan_u64_scratch_words(tiles) words).
uint64_t scan_tile_size();
tc_status scan_u64_from_tile_sums(const uint64_t* in, uint64_t* out, uint64_t n, uint64_t* sums, uint32_t* d_err,
                                  uint64_t* scratch, uint64_t scratch_words, cudaStream_t st);

// Stable LSD radix sort of (key, val) pairs on key bits [bit0, bit1).  The
// sorted data ends in (k0, v0); k1, v1 are scratch of the same size.
tc_status radix_sort_pairs(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, uint64_t n, int bit0,
                           int bit1, cudaStream_t st);

inline size_t scan_align256(size_t x) { return (x + 255) & ~(size_t)255; }

tc_status launch_widen_u32(const uint32_t* in, uint64_t n, int64_t* out, cudaStream_t st);

tc_status build_graph(int64_t n, int64_t m, const int32_t* d_src, const int32_t* d_dst, const int64_t* d_t,
                      cudaStream_t st, tc_graph* g);

// Path weights, their windows and their exact prefix sum: prefix[m + 1],
// win[m], and w[m] when w is not NULL.  scratch:
// weights_scan_scratch_bytes(m) bytes; *d_err collects overflow bits.
size_t weights_scan_scratch_bytes(uint64_t m);
tc_status launch_weights_scan(const tc_graph* g, const Plan& plan, int64_t delta, EdgeWin* win, uint64_t* prefix,
                              uint64_t* w, void* scratch, uint32_t* d_err, cudaStream_t st);
tc_status launch_guide(const tc_graph* g, const Plan& plan, int64_t delta, const uint64_t* prefix,
                       void* index, uint32_t* d_err, cudaStream_t st);
tc_status launch_guide_at(const tc_graph* g, const Plan& plan, int64_t delta, const uint64_t* prefix,
                          IndexHeader* hdr, uint32_t* guide, uint32_t* d_err, cudaStream_t st);
size_t proposal_index_bytes(uint64_t m);  // header + guide of a proposal's CDF

size_t index_bytes(uint64_t m);

// learned proposal (tc_learn.cu)
tc_status mlp_create(uint64_t seed, tc_mlp** out);
void mlp_destroy(tc_mlp* M);
int mlp_num_params();
tc_status mlp_set_params(tc_mlp* M, const float* h);
tc_status mlp_get_params(const tc_mlp* M, float* h);
tc_status launch_features(const tc_graph* g, const EdgeWin* win, int64_t delta, uint16_t* feat, cudaStream_t st);
tc_status launch_mlp_forward(const tc_mlp* M, const uint16_t* feat, const uint32_t* rows, uint64_t n, float* out,
                             cudaStream_t st);
tc_status launch_mlp_grad(const tc_mlp* M, const uint16_t* feat, const uint32_t* rows, const float* labels,
                          uint64_t n, float* grad, float* loss_sum, cudaStream_t st, bool given_dz = false);
// Gradient of the estimator-variance objective (z, dz: n floats of scratch;
// *loss receives the objective, loss_scratch one float the gradient kernel
// may touch).
tc_status launch_variance_grad(const tc_mlp* M, const uint16_t* feat, const uint32_t* rows, const float* X,
                               uint64_t n, float eps, float* grad, float* loss, float* z, float* dz,
                               float* loss_scratch, cudaStream_t st);
tc_status mlp_adam(tc_mlp* M, float lr, cudaStream_t st);
float* mlp_grad_buffer(tc_mlp* M);
int mlp_kernel(int kind);  // tc_mlp_kernel
// Synchronises st, then reports (and clears) the error bits the network's
// inference kernel left in the network's device error word.
tc_status mlp_check_error(const tc_mlp* M, cudaStream_t st, const char* what);
// Columns 12..15 of the rows of edges with w > 0 (prefix: the plain prefix).
tc_status launch_sample_features(const tc_graph* g, const uint64_t* prefix, const uint64_t* trace, uint64_t n,
                                 int64_t delta, uint16_t* feat, uint32_t* d_err, cudaStream_t st);
tc_status launch_trace_to_rows(const uint64_t* trace, uint64_t n, uint32_t* rows, float* labels, cudaStream_t st,
                               bool clip = false);
tc_status launch_clip_labels(const float* labels, uint64_t n, float* out, cudaStream_t st);
// Proposal h, q = w h and the exact prefix of q (scratch:
// proposal_scan_scratch_bytes(m) bytes).
size_t proposal_scan_scratch_bytes(uint64_t m);
tc_status launch_proposal_scan(const tc_mlp* M, const uint16_t* feat, const uint64_t* prefix, uint64_t m, float eps,
                               float scale, uint16_t* h, uint64_t* qprefix, uint32_t* hrange, void* scratch,
                               uint32_t* d_err, cudaStream_t st);
int guide_bits(uint64_t m);

struct SampleSums {  // per-call device accumulator
  unsigned long long sum_x, sum_x2_lo, sum_x2_hi, hits, checked, W;
  unsigned int err;
  unsigned int pad;
};

tc_status launch_path_sum(const tc_graph* g, const Plan& plan, int64_t delta, const uint64_t* prefix,
                          const void* index, uint64_t W, SampleSums* d_sums, cudaStream_t st);
tc_status launch_sampler(const tc_graph* g, const Plan& plan, int64_t delta, const uint64_t* prefix,
                         const void* index, uint64_t k, uint64_t seed, uint64_t offset, uint64_t* trace,
                         SampleSums* d_sums, cudaStream_t st, const void* qindex = nullptr,
                         const uint16_t* h = nullptr, unsigned long long* bins = nullptr);

// Key-ordered sampling: samples are processed in chunks of at most
// kChunkSamples, each put in key order by sort_sample_ids (no allocation;
// scratch of sort_scratch_bytes(count)); calls below kSortedMinSamples
// samples run in id order.
constexpr uint64_t kSortedMinSamples = 1ull << 16;
constexpr uint64_t kChunkSamples = 1ull << 28;
size_t sort_scratch_bytes(uint64_t count);
tc_status sort_sample_ids(const IndexHeader* hdr, uint64_t seed, uint64_t first, uint64_t count, void* scratch,
                          uint32_t* order, cudaStream_t st);

// Batched sampling: each query's arguments are a kBatchQueryBytes-byte
// record in device memory, written on the host by batch_query_record; the
// queries' work items (tiles of `tile` samples) are numbered query after
// query, query q owning items [tile_begin[q], tile_begin[q + 1]).  order is
// the query's key order (chunk after chunk) or NULL for id order.
constexpr size_t kBatchQueryBytes = 512;
void batch_query_record(void* h_rec, const tc_graph* g, const Plan& plan, int64_t delta, const uint64_t* prefix,
                        const void* index, uint64_t k, uint64_t seed, uint64_t offset, const uint32_t* order);
int sample_batch_blocks_per_sm(int block_size);  // 0: unsupported block size
tc_status launch_sample_batch(int block_size, uint32_t tile, unsigned blocks, const void* d_records,
                              const uint64_t* d_tile_begin, uint32_t nq, unsigned long long* d_next_item,
                              SampleSums* d_sums, cudaStream_t st);

// Diagnostic timing by phase (tc_set_timing, tc_last_phase_ms): a
// PhaseTimer records an event pair around each start()/stop() on its stream
// while timing is on; constructing one drops the phase's earlier events.
constexpr int kNumPhases = 5;
struct PhaseTimer {
  int ph;
  cudaStream_t st;
  PhaseTimer(int phase, cudaStream_t s);
  void start();
  void stop();
};
void set_timing(bool on);
float last_phase_ms(int phase);
float last_sampler_ms();

// Host form of the estimate from the sums (tc_api.cu).
void finish_estimate(tc_estimate* o);
tc_status compile_plan_checked(const tc_motif* motif, Plan* p);

}  // namespace tc
