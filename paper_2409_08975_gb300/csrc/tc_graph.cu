// Temporal list construction (Sec. III: adjacency lists sorted by time;
// Sec. III-B: per-pair lists L_{u,v}) on the GPU, with this library's own
// exclusive scans and stable LSD radix sort.
//
// Radix sort: least-significant-digit first, 8-bit digits, one pass =
// per-tile digit histograms, an exclusive scan of the digit-major histogram
// table, and a stable scatter in which each warp ranks its keys with
// __match_any_sync (warp-level multisplit) in input order.
#include <cuda_runtime.h>

#include <algorithm>

#include "tc_internal.cuh"

namespace tc {

// ---------------------------------------------------------------------------
// Exclusive scans (reduce-then-scan).  With an error word, every tile of
// every level checks in 128 bits that its total plus its offset fits 64 bits,
// so a grand total beyond 64 bits is always flagged.

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <class T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* s_warp, T* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_warp[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    T x = lane < (kScanThreads / 32) ? s_warp[lane] : T(0);
    T xi = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, xi, o);
      if (lane >= o) xi += y;
    }
    if (lane < (kScanThreads / 32)) s_warp[lane] = xi - x;
    if (lane == (kScanThreads / 32) - 1) s_warp[kScanThreads / 32] = xi;
  }
  __syncthreads();
  T res = s_warp[wid] + inc - v;
  *total = s_warp[kScanThreads / 32];
  __syncthreads();
  return res;
}

// True in every thread when the sum of the block's `acc` values (plus
// `extra`, added once) does not fit 64 bits; each thread passes its own
// per-thread overflow flag.  128-bit warp sums, one shared flag.
__device__ __forceinline__ bool block_sum_overflows(uint64_t acc, bool thread_ovf, uint64_t extra) {
  __shared__ unsigned int s_flag;
  __shared__ unsigned long long s_part[kScanThreads / 32][2];
  unsigned __int128 a = acc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t lo = __shfl_down_sync(0xffffffffu, (uint64_t)a, o);
    const uint64_t hi = __shfl_down_sync(0xffffffffu, (uint64_t)(a >> 64), o);
    a += ((unsigned __int128)hi << 64) | lo;
  }
  if (threadIdx.x == 0) s_flag = 0;
  if ((threadIdx.x & 31) == 0) {
    s_part[threadIdx.x >> 5][0] = (uint64_t)a;
    s_part[threadIdx.x >> 5][1] = (uint64_t)(a >> 64);
  }
  __syncthreads();
  if (thread_ovf) atomicOr(&s_flag, 1u);
  if (threadIdx.x == 0) {
    unsigned __int128 tot = extra;
    for (int w = 0; w < kScanThreads / 32; w++)
      tot += ((unsigned __int128)s_part[w][1] << 64) | s_part[w][0];
    if (tot >> 64) atomicOr(&s_flag, 1u);
  }
  __syncthreads();
  const bool r = s_flag != 0;
  __syncthreads();
  return r;
}

// Tile sums.  With an error word (uint64 only) a tile total beyond 64 bits
// sets kErrOverflow.
template <class T>
__global__ void k_tile_reduce(const T* __restrict__ in, uint64_t n, T* __restrict__ sums, uint32_t* err) {
  __shared__ T s_warp[kScanThreads / 32 + 1];
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
  T acc = 0;
  bool ovf = false;
#pragma unroll
  for (int j = 0; j < kScanItems; j++) {
    const uint64_t i = base + j;
    if (i < n) {
      T x = in[i];
      T s = acc + x;
      if (s < acc) ovf = true;
      acc = s;
    }
  }
  if (sizeof(T) == 8 && err != nullptr) {
    if (block_sum_overflows((uint64_t)acc, ovf, 0) && threadIdx.x == 0) atomicOr(err, kErrOverflow);
  }
  T total;
  block_exclusive_scan<T>(acc, s_warp, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// out[i] = offset[tile] + exclusive prefix; the last tile also writes
// out[n] = total when write_total.
template <class T>
__global__ void k_tile_scan(const T* in, uint64_t n, const T* __restrict__ offsets, T* out, bool write_total,
                            uint32_t* err) {
  __shared__ T s_warp[kScanThreads / 32 + 1];
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
  // a thread's items as 16-byte loads when they are whole and aligned
  const bool vec = base + kScanItems <= n && ((reinterpret_cast<uintptr_t>(in + base) |
                                               reinterpret_cast<uintptr_t>(out + base)) & 15) == 0;
  T v[kScanItems];
  if (vec) {
#pragma unroll
    for (int j = 0; j < (int)(kScanItems * sizeof(T) / 16); j++)
      reinterpret_cast<uint4*>(v)[j] = __ldcs(reinterpret_cast<const uint4*>(in + base) + j);
  } else {
#pragma unroll
    for (int j = 0; j < kScanItems; j++) v[j] = base + j < n ? in[base + j] : T(0);
  }
  T acc = 0;
  bool ovf = false;
#pragma unroll
  for (int j = 0; j < kScanItems; j++) {
    const T s = acc + v[j];
    if (s < acc) ovf = true;
    acc = s;
  }
  const T off = offsets ? offsets[blockIdx.x] : T(0);
  // uint64 with an error word: this tile's total plus its offset must fit
  if (sizeof(T) == 8 && err != nullptr) {
    if (block_sum_overflows((uint64_t)acc, ovf, (uint64_t)off) && threadIdx.x == 0) atomicOr(err, kErrOverflow);
  }
  T total;
  T ex = block_exclusive_scan<T>(acc, s_warp, &total);
  T run = off + ex;
#pragma unroll
  for (int j = 0; j < kScanItems; j++) {  // the exclusive prefix in place of the items
    const T x = v[j];
    v[j] = run;
    run += x;
  }
  if (vec) {
#pragma unroll
    for (int j = 0; j < (int)(kScanItems * sizeof(T) / 16); j++)
      reinterpret_cast<uint4*>(out + base)[j] = reinterpret_cast<const uint4*>(v)[j];
  } else {
#pragma unroll
    for (int j = 0; j < kScanItems; j++)
      if (base + j < n) out[base + j] = v[j];
  }
  if (write_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = off + total;
}

template <class T>
static tc_status scan_rec(const T* in, T* out, uint64_t n, bool write_total, uint32_t* d_err, cudaStream_t st) {
  if (n == 0) {
    if (write_total) TC_CUDA(cudaMemsetAsync(out, 0, sizeof(T), st));
    return TC_OK;
  }
  const uint64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles == 1) {
    k_tile_scan<T><<<1, kScanThreads, 0, st>>>(in, n, nullptr, out, write_total, d_err);
    TC_LAUNCHED(1);
    TC_CUDA(cudaGetLastError());
    return TC_OK;
  }
  T* sums = nullptr;
  TC_CUDA(pool_malloc(&sums, sizeof(T) * tiles, st));
  k_tile_reduce<T><<<(unsigned)tiles, kScanThreads, 0, st>>>(in, n, sums, d_err);
  TC_LAUNCHED(1);
  tc_status s = TC_OK;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) s = cuda_status(e, "k_tile_reduce");
  // in place: sums[i] <- exclusive prefix of sums (tile offsets)
  if (s == TC_OK) s = scan_rec<T>(sums, sums, tiles, false, d_err, st);
  if (s == TC_OK) {
    k_tile_scan<T><<<(unsigned)tiles, kScanThreads, 0, st>>>(in, n, sums, out, write_total, d_err);
    TC_LAUNCHED(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) s = cuda_status(e, "k_tile_scan");
  }
  cudaFreeAsync(sums, st);
  return s;
}

tc_status scan_u64(const uint64_t* in, uint64_t* out, uint64_t n, uint32_t* d_err, cudaStream_t st) {
  return scan_rec<uint64_t>(in, out, n, true, d_err, st);
}
tc_status scan_u32(const uint32_t* in, uint32_t* out, uint64_t n, cudaStream_t st) {
  return scan_rec<uint32_t>(in, out, n, true, nullptr, st);
}

uint64_t scan_u64_scratch_words(uint64_t n) {
  uint64_t words = 0;
  for (uint64_t tiles = (n + kScanTile - 1) / kScanTile; tiles > 1; tiles = (tiles + kScanTile - 1) / kScanTile)
    words += tiles;
  return words;
}

// The same reduce-then-scan as scan_rec, with the tile sums of every level
// placed in caller scratch (scan_u64_scratch_words(n) elements) instead of
// stream-ordered allocations.
template <class T>
static tc_status scan_in_scratch(const T* in, T* out, uint64_t n, bool write_total, uint32_t* d_err, T* scratch,
                                 uint64_t scratch_words, cudaStream_t st) {
  if (n == 0) {
    if (write_total) TC_CUDA(cudaMemsetAsync(out, 0, sizeof(T), st));
    return TC_OK;
  }
  const uint64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles == 1) {
    k_tile_scan<T><<<1, kScanThreads, 0, st>>>(in, n, nullptr, out, write_total, d_err);
    TC_LAUNCHED(1);
    TC_CUDA(cudaGetLastError());
    return TC_OK;
  }
  if (scratch_words < tiles) return set_error(TC_ERR_INVALID_ARG, "scan scratch too small");
  T* sums = scratch;
  k_tile_reduce<T><<<(unsigned)tiles, kScanThreads, 0, st>>>(in, n, sums, d_err);
  TC_LAUNCHED(1);
  TC_CUDA(cudaGetLastError());
  TC_TRY(scan_in_scratch<T>(sums, sums, tiles, false, d_err, scratch + tiles, scratch_words - tiles, st));
  k_tile_scan<T><<<(unsigned)tiles, kScanThreads, 0, st>>>(in, n, sums, out, write_total, d_err);
  TC_LAUNCHED(1);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

tc_status scan_u64_in_scratch(const uint64_t* in, uint64_t* out, uint64_t n, bool write_total, uint32_t* d_err,
                              uint64_t* scratch, uint64_t scratch_words, cudaStream_t st) {
  return scan_in_scratch<uint64_t>(in, out, n, write_total, d_err, scratch, scratch_words, st);
}

// The reduce-then-scan with the first level's tile sums already formed by
// the kernel that wrote in (sums[t] = the sum of in over tile t of
// kScanTile values, its overflow already reported): the sums are scanned in
// place into tile offsets, then each tile is scanned from its offset.
tc_status scan_u64_from_tile_sums(const uint64_t* in, uint64_t* out, uint64_t n, uint64_t* sums, uint32_t* d_err,
                                  uint64_t* scratch, uint64_t scratch_words, cudaStream_t st) {
  if (n == 0) {
    TC_CUDA(cudaMemsetAsync(out, 0, sizeof(uint64_t), st));
    return TC_OK;
  }
  const uint64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles > 1) TC_TRY(scan_in_scratch<uint64_t>(sums, sums, tiles, false, d_err, scratch, scratch_words, st));
  k_tile_scan<uint64_t><<<(unsigned)tiles, kScanThreads, 0, st>>>(in, n, tiles > 1 ? sums : nullptr, out, true, d_err);
  TC_LAUNCHED(1);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

uint64_t scan_tile_size() { return kScanTile; }

tc_status scan_u32_in_scratch(const uint32_t* in, uint32_t* out, uint64_t n, uint32_t* scratch,
                              uint64_t scratch_words, cudaStream_t st) {
  return scan_in_scratch<uint32_t>(in, out, n, true, nullptr, scratch, scratch_words, st);
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of (uint32 key, uint32 value).

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kMaxDigitBits = 11;
constexpr int kMaxRadix = 1 << kMaxDigitBits;

// warp w of a tile owns keys [w * 32 * kSortItems, (w + 1) * 32 * kSortItems)
__device__ __forceinline__ uint64_t sort_index(uint64_t tile, int warp, int item, int lane) {
  return tile * kSortTile + (uint64_t)warp * 32 * kSortItems + (uint64_t)item * 32 + lane;
}

// hist[d * tiles + tile] = keys of the tile whose digit (key >> bit) & (2^nbits - 1) is d
__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const uint32_t* __restrict__ keys, uint64_t n,
                                                           int bit, int nbits, uint32_t* __restrict__ hist,
                                                           uint32_t tiles) {
  extern __shared__ uint32_t s_hist[];
  const int radix = 1 << nbits;
  for (int i = threadIdx.x; i < radix; i += kSortThreads) s_hist[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t mask = (uint32_t)radix - 1u;
#pragma unroll 4
  for (int j = 0; j < kSortItems; j++) {
    const uint64_t i = sort_index(blockIdx.x, warp, j, lane);
    if (i < n) atomicAdd(&s_hist[(keys[i] >> bit) & mask], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < radix; d += kSortThreads) hist[(uint64_t)d * tiles + blockIdx.x] = s_hist[d];
}

// Stable scatter through shared memory: per-warp digit counts (warp-level
// multisplit with __match_any_sync) in input order give every key its rank
// among the tile's keys of the same digit; keys and values are staged in
// shared memory in (digit, rank) order and written out in that order, so
// each digit's run of the tile goes to consecutive global addresses.
// Shared memory: the per-warp counts (later the stage), the tile-local start
// and the global start of every digit.
__host__ __device__ constexpr int sort_scatter_words(int radix) {
  return (kSortWarps * radix > 2 * kSortTile ? kSortWarps * radix : 2 * kSortTile) + 2 * radix;
}

__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(const uint32_t* __restrict__ kin,
                                                              const uint32_t* __restrict__ vin, uint64_t n,
                                                              int bit, int nbits,
                                                              const uint32_t* __restrict__ offs,
                                                              uint32_t tiles, uint32_t* __restrict__ kout,
                                                              uint32_t* __restrict__ vout) {
  extern __shared__ uint32_t smem[];
  const int radix = 1 << nbits;
  const int cnt_words = kSortWarps * radix > 2 * kSortTile ? kSortWarps * radix : 2 * kSortTile;
  uint32_t* s_cnt = smem;                // [kSortWarps][radix]; afterwards the stage
  uint32_t* s_start = smem + cnt_words;  // [radix]
  uint32_t* s_base = s_start + radix;    // [radix]
  __shared__ uint32_t warp_tot[kSortWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t mask = (uint32_t)radix - 1u;
  const uint32_t lt = (1u << lane) - 1u;
  for (int i = threadIdx.x; i < kSortWarps * radix; i += kSortThreads) s_cnt[i] = 0;
  __syncthreads();
  uint32_t key[kSortItems], val[kSortItems];
#pragma unroll
  for (int j = 0; j < kSortItems; j++) {
    const uint64_t i = sort_index(blockIdx.x, warp, j, lane);
    key[j] = i < n ? kin[i] : 0u;
    val[j] = i < n ? vin[i] : 0u;
  }
  uint32_t* my = s_cnt + warp * radix;
#pragma unroll
  for (int j = 0; j < kSortItems; j++) {
    const uint64_t i = sort_index(blockIdx.x, warp, j, lane);
    const uint32_t d = i < n ? ((key[j] >> bit) & mask) : 0xFFFFFFFFu;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    if (d != 0xFFFFFFFFu && (peers & lt) == 0) my[d] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit: counts of earlier warps (in place), the tile total and the
  // digit's global start
  for (int d = threadIdx.x; d < radix; d += kSortThreads) {
    uint32_t run = 0;
    for (int w = 0; w < kSortWarps; w++) {
      const uint32_t c = s_cnt[w * radix + d];
      s_cnt[w * radix + d] = run;
      run += c;
    }
    s_start[d] = run;
    s_base[d] = offs[(uint64_t)d * tiles + blockIdx.x];
  }
  __syncthreads();
  {  // exclusive scan of the digit totals: thread t owns digits [t * per, (t + 1) * per)
    const int per = (radix + kSortThreads - 1) / kSortThreads;
    const int d0 = threadIdx.x * per;
    uint32_t local = 0;
    for (int j = 0; j < per; j++)
      if (d0 + j < radix) local += s_start[d0 + j];
    uint32_t incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    uint32_t run = incl - local;
    for (int w = 0; w < warp; w++) run += warp_tot[w];
    for (int j = 0; j < per; j++)
      if (d0 + j < radix) {
        const uint32_t c = s_start[d0 + j];
        s_start[d0 + j] = run;
        run += c;
      }
  }
  __syncthreads();
  // tile-local positions in (digit, rank) order
  uint32_t lp[kSortItems];
#pragma unroll
  for (int j = 0; j < kSortItems; j++) {
    const uint64_t i = sort_index(blockIdx.x, warp, j, lane);
    const uint32_t d = i < n ? ((key[j] >> bit) & mask) : 0xFFFFFFFFu;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    lp[j] = 0xFFFFFFFFu;
    if (d != 0xFFFFFFFFu) lp[j] = s_start[d] + my[d] + __popc(peers & lt);
    __syncwarp();
    if (d != 0xFFFFFFFFu && (peers & lt) == 0) my[d] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();  // the counts are no longer read: the stage reuses them
  uint32_t* stage_k = s_cnt;
  uint32_t* stage_v = s_cnt + kSortTile;
#pragma unroll
  for (int j = 0; j < kSortItems; j++)
    if (lp[j] != 0xFFFFFFFFu) {
      stage_k[lp[j]] = key[j];
      stage_v[lp[j]] = val[j];
    }
  __syncthreads();
  const uint64_t t0 = (uint64_t)blockIdx.x * kSortTile;
  const uint32_t count = (uint32_t)(n - t0 < (uint64_t)kSortTile ? n - t0 : (uint64_t)kSortTile);
  for (uint32_t i = threadIdx.x; i < count; i += kSortThreads) {
    const uint32_t k = stage_k[i];
    const uint32_t d = (k >> bit) & mask;
    const uint32_t g = s_base[d] + (i - s_start[d]);
    kout[g] = k;
    vout[g] = stage_v[i];
  }
}

// Sorts on bits [bit0, bit1) in ceil((bit1 - bit0) / 11) passes of equal
// width (at most 11 bits, 2048 digits).
tc_status radix_sort_pairs(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, uint64_t n, int bit0,
                           int bit1, cudaStream_t st) {
  if (n <= 1 || bit1 <= bit0) return TC_OK;
  static bool attr = false;
  if (!attr) {
    TC_CUDA(cudaFuncSetAttribute(k_sort_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(uint32_t) * sort_scatter_words(kMaxRadix))));
    attr = true;
  }
  const int total = bit1 - bit0;
  const int passes = (total + kMaxDigitBits - 1) / kMaxDigitBits;
  const int width = (total + passes - 1) / passes;
  const uint64_t tiles = (n + kSortTile - 1) / kSortTile;
  uint32_t* hist = nullptr;
  TC_CUDA(pool_malloc(&hist, sizeof(uint32_t) * ((uint64_t)(1 << width) * tiles + 1), st));
  tc_status s = TC_OK;
  uint32_t *ka = k0, *va = v0, *kb = k1, *vb = v1;
  for (int bit = bit0; bit < bit1 && s == TC_OK; bit += width) {
    const int nbits = std::min(width, bit1 - bit);
    const int radix = 1 << nbits;
    k_sort_hist<<<(unsigned)tiles, kSortThreads, sizeof(uint32_t) * radix, st>>>(ka, n, bit, nbits, hist,
                                                                                (uint32_t)tiles);
    TC_LAUNCHED(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { s = cuda_status(e, "k_sort_hist"); break; }
    s = scan_rec<uint32_t>(hist, hist, (uint64_t)radix * tiles, false, nullptr, st);
    if (s != TC_OK) break;
    k_sort_scatter<<<(unsigned)tiles, kSortThreads, sizeof(uint32_t) * sort_scatter_words(radix), st>>>(
        ka, va, n, bit, nbits, hist, (uint32_t)tiles, kb, vb);
    TC_LAUNCHED(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) { s = cuda_status(e, "k_sort_scatter"); break; }
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (s == TC_OK && ka != k0) {
    cudaError_t e = cudaMemcpyAsync(k0, ka, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(v0, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) s = cuda_status(e, "radix copy-back");
  }
  cudaFreeAsync(hist, st);
  return s;
}

// ---------------------------------------------------------------------------
// Graph build.  The input edges are first packed into one 16-byte record
// {src, dst, t} per input index, so that every later gather by a sorted
// permutation is one random load.

__global__ void k_check_pack(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                             const int64_t* __restrict__ t, uint64_t m, int64_t n, uint32_t* err, long long* tminmax,
                             OutEdge* __restrict__ pack) {
  long long lo = INT64_MAX, hi = INT64_MIN;
  bool bad = false;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
    OutEdge r;
    r.src = src[i];
    r.dst = dst[i];
    r.t = t[i];
    if (r.src < 0 || r.src >= n || r.dst < 0 || r.dst >= n) bad = true;
    lo = r.t < lo ? r.t : lo;
    hi = r.t > hi ? r.t : hi;
    pack[i] = r;
  }
  for (int o = 16; o > 0; o >>= 1) {
    long long l2 = __shfl_down_sync(0xffffffffu, lo, o), h2 = __shfl_down_sync(0xffffffffu, hi, o);
    lo = l2 < lo ? l2 : lo;
    hi = h2 > hi ? h2 : hi;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&tminmax[0], lo);
    atomicMax(&tminmax[1], hi);
  }
  if (bad) atomicOr(err, kErrBadId);
}

// keys = low or high 32 bits of (t - tmin), values = input index
__global__ void k_time_keys(const int64_t* __restrict__ t, uint64_t m, int64_t tmin, int high, uint32_t* keys,
                            uint32_t* vals) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t d = (uint64_t)t[i] - (uint64_t)tmin;
    keys[i] = high ? (uint32_t)(d >> 32) : (uint32_t)d;
    if (vals) vals[i] = (uint32_t)i;
  }
}

__global__ void k_high_time_keys(const OutEdge* __restrict__ pack, const uint32_t* __restrict__ perm, uint64_t m,
                                 int64_t tmin, uint32_t* keys) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x)
    keys[i] = (uint32_t)(((uint64_t)pack[perm[i]].t - (uint64_t)tmin) >> 32);
}

// keys[i] = col[perm[i]] (the 4-byte column stays in L2 better than the records)
__global__ void k_gather_key(const int32_t* __restrict__ col, const uint32_t* __restrict__ perm, uint64_t m,
                             uint32_t* keys) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x)
    keys[i] = (uint32_t)col[perm[i]];
}

// off[v] = first position whose (sorted) key is >= v, for v in [0, n]
__global__ void k_offsets(const uint32_t* __restrict__ sorted, uint64_t len, int64_t n, uint32_t* off) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= len; i += (uint64_t)gridDim.x * blockDim.x) {
    const int64_t prev = i == 0 ? -1 : (int64_t)sorted[i - 1];
    const int64_t cur = i == len ? n : (int64_t)sorted[i];
    for (int64_t v = prev + 1; v <= cur; v++) off[v] = (uint32_t)i;
  }
}

__global__ void k_fill_out(const OutEdge* __restrict__ pack, const uint32_t* __restrict__ perm, uint64_t m,
                           OutEdge* out_e, uint32_t* canon, int64_t tmin, uint32_t* __restrict__ out_t32) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t e = perm[i];
    const OutEdge r = pack[e];
    out_e[i] = r;
    canon[e] = (uint32_t)i;
    if (out_t32) out_t32[i] = (uint32_t)((uint64_t)r.t - (uint64_t)tmin);
  }
}

__global__ void k_fill_in(const OutEdge* __restrict__ pack, const uint32_t* __restrict__ perm,
                          const uint32_t* __restrict__ canon, uint64_t m, InEdge* in_e, uint32_t* in_eid,
                          int64_t tmin, uint32_t* __restrict__ in_t32) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t e = perm[i];
    const OutEdge r = pack[e];
    InEdge q;
    q.src = r.src;
    q.dst = r.dst;
    q.t = r.t;
    in_e[i] = q;
    in_eid[i] = canon[e];
    if (in_t32) in_t32[i] = (uint32_t)((uint64_t)r.t - (uint64_t)tmin);
  }
}

// pair order: destination, time and canonical id of each position
__global__ void k_pair_gather(const OutEdge* __restrict__ pack, const uint32_t* __restrict__ perm,
                              const uint32_t* __restrict__ canon, uint64_t m, int32_t* __restrict__ pdst,
                              int64_t* __restrict__ pair_t, uint32_t* __restrict__ pair_eid, int64_t tmin,
                              uint32_t* __restrict__ pair_t32) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t e = perm[i];
    const OutEdge r = pack[e];
    pdst[i] = r.dst;
    pair_t[i] = r.t;
    pair_eid[i] = canon[e];
    if (pair_t32) pair_t32[i] = (uint32_t)((uint64_t)r.t - (uint64_t)tmin);
  }
}

// pair flags: 1 where (src, dst) differs from the previous position
__global__ void k_pair_flags(const uint32_t* __restrict__ psrc, const int32_t* __restrict__ pdst, uint64_t m,
                             uint32_t* flags) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x)
    flags[i] = (i == 0 || psrc[i] != psrc[i - 1] || pdst[i] != pdst[i - 1]) ? 1u : 0u;
}

__global__ void k_fill_pairs(const uint32_t* __restrict__ psrc, const int32_t* __restrict__ pdst,
                             const uint32_t* __restrict__ flags, const uint32_t* __restrict__ pidx, uint64_t m,
                             int32_t* pair_dst, uint32_t* pair_eoff, uint32_t* pair_src) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
    if (flags[i]) {
      const uint32_t p = pidx[i];
      pair_dst[p] = pdst[i];
      pair_src[p] = psrc[i];
      pair_eoff[p] = (uint32_t)i;
    }
  }
}

__global__ void k_set_u32(uint32_t* p, uint32_t v) { *p = v; }

// Window-search anchors (delta-independent; see tc_graph::x_in).  For
// canonical edge i = (u, v, t): x_in[i] = the first position of u's in-list
// with time >= t, with its range word r_in[i], and the range word r_self[i]
// of i itself in u's out-list.  For in-list position p of edge c = in_eid[p]
// = (u, v, t): out2in[c] = p with its range word r_o2i[c] in v's in-list, and
// x_out[c] = the first position of v's out-list with time >= t, with r_out[c].
// The searches of consecutive threads run in the same list (edges of one
// vertex in time order), so their probes share sectors.
template <bool Compact>
__global__ void k_anchor_in(const OutEdge* __restrict__ out_e, const InEdge* __restrict__ in_e,
                            const uint32_t* __restrict__ in_off, const uint32_t* __restrict__ out_off,
                            const uint32_t* __restrict__ in_t32, int64_t tmin, uint64_t m,
                            uint32_t* __restrict__ x_in, uint32_t* __restrict__ r_in, uint32_t* __restrict__ r_self) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
    const OutEdge e = out_e[i];
    auto tt = [&](uint32_t p) -> int64_t { return Compact ? (int64_t)__ldg(in_t32 + p) + tmin : in_e[p].t; };
    const uint32_t s = __ldg(in_off + e.src), f = __ldg(in_off + e.src + 1);
    const uint32_t a = search_time<true>(s, f, e.t, tt);
    x_in[i] = a;
    r_in[i] = range_word(a, s, f);
    r_self[i] = range_word((uint32_t)i, __ldg(out_off + e.src), __ldg(out_off + e.src + 1));
  }
}

template <bool Compact>
__global__ void k_anchor_out(const OutEdge* __restrict__ out_e, const InEdge* __restrict__ in_e,
                             const uint32_t* __restrict__ in_eid, const uint32_t* __restrict__ out_off,
                             const uint32_t* __restrict__ in_off, const uint32_t* __restrict__ out_t32, int64_t tmin,
                             uint64_t m, uint32_t* __restrict__ x_out, uint32_t* __restrict__ out2in,
                             uint32_t* __restrict__ r_out, uint32_t* __restrict__ r_o2i) {
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < m; p += (uint64_t)gridDim.x * blockDim.x) {
    const InEdge e = in_e[p];
    auto tt = [&](uint32_t q) -> int64_t { return Compact ? (int64_t)__ldg(out_t32 + q) + tmin : out_e[q].t; };
    const uint32_t c = in_eid[p];
    const uint32_t s = __ldg(out_off + e.dst), f = __ldg(out_off + e.dst + 1);
    const uint32_t a = search_time<true>(s, f, e.t, tt);
    x_out[c] = a;
    r_out[c] = range_word(a, s, f);
    out2in[c] = (uint32_t)p;
    r_o2i[c] = range_word((uint32_t)p, __ldg(in_off + e.dst), __ldg(in_off + e.dst + 1));
  }
}

// Insert every distinct pair (x, y) with its list range into the hash table.
// Each pair is inserted once; a probe sequence ends at the first empty slot,
// which exists because the load factor is at most 1/2.
__global__ void k_pair_hash(const uint32_t* __restrict__ pair_src, const int32_t* __restrict__ pair_dst,
                            const uint32_t* __restrict__ pair_eoff, uint32_t P, PairSlot* table, uint64_t mask) {
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t x = pair_src[p], y = (uint32_t)pair_dst[p];
    const unsigned long long key = pair_key(x, y);
    uint64_t h = mix64(key) & mask;
    for (uint64_t probe = 0; probe <= mask; probe++) {
      unsigned long long* word = reinterpret_cast<unsigned long long*>(&table[h]);
      if (atomicCAS(word, kEmptyPairKey, key) == kEmptyPairKey) {
        table[h].begin = pair_eoff[p];
        table[h].end = pair_eoff[p + 1];
        break;
      }
      h = (h + 1) & mask;
    }
  }
}

static unsigned grid_for(uint64_t n, int threads = 256) {
  uint64_t b = (n + threads - 1) / threads;
  const uint64_t cap = (uint64_t)num_sms() * 16;
  if (b > cap) b = cap;
  if (b == 0) b = 1;
  return (unsigned)b;
}

template <class T>
static tc_status dmalloc(T** p, uint64_t count, cudaStream_t st) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = pool_malloc((void**)p, sizeof(T) * count, st);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return set_error(TC_ERR_OOM, "device allocation failed");
  }
  if (e != cudaSuccess) return cuda_status(e, "cudaMallocAsync");
  return TC_OK;
}

tc_status build_graph(int64_t n, int64_t m, const int32_t* d_src, const int32_t* d_dst, const int64_t* d_t,
                      cudaStream_t st, tc_graph* g) {
  const uint64_t M = (uint64_t)m;
  g->n = n;
  g->m = m;
  // graph arrays
  TC_TRY(dmalloc(&g->out_off, n + 1, st));
  TC_TRY(dmalloc(&g->out_e, M, st));
  TC_TRY(dmalloc(&g->perm, M, st));
  TC_TRY(dmalloc(&g->in_off, n + 1, st));
  TC_TRY(dmalloc(&g->in_e, M, st));
  TC_TRY(dmalloc(&g->in_eid, M, st));
  TC_TRY(dmalloc(&g->pair_off, n + 1, st));
  TC_TRY(dmalloc(&g->pair_t, M, st));
  TC_TRY(dmalloc(&g->pair_eid, M, st));

  // scratch
  uint32_t *err = nullptr, *ka = nullptr, *va = nullptr, *kb = nullptr, *vb = nullptr, *permT = nullptr,
           *canon = nullptr, *flags = nullptr, *pidx = nullptr, *pair_src = nullptr;
  long long* tmm = nullptr;
  OutEdge* pack = nullptr;
  int32_t* pdst = nullptr;
  tc_status s = TC_OK;
  auto done = [&](tc_status r) {
    for (void* p : {(void*)err, (void*)ka, (void*)va, (void*)kb, (void*)vb, (void*)permT, (void*)canon,
                    (void*)flags, (void*)pidx, (void*)pair_src, (void*)tmm, (void*)pack, (void*)pdst})
      if (p) cudaFreeAsync(p, st);
    return r;
  };
#define TRY_S(x)                 \
  do {                           \
    s = (x);                     \
    if (s != TC_OK) return done(s); \
  } while (0)
#define TRY_C(x, what)                                    \
  do {                                                    \
    cudaError_t _e = (x);                                 \
    if (_e != cudaSuccess) return done(cuda_status(_e, what)); \
  } while (0)

  TRY_S(dmalloc(&err, 1, st));
  TRY_S(dmalloc(&tmm, 2, st));
  TRY_S(dmalloc(&pack, M, st));
  TRY_C(cudaMemsetAsync(err, 0, sizeof(uint32_t), st), "memset");
  long long init[2] = {INT64_MAX, INT64_MIN};
  TRY_C(cudaMemcpyAsync(tmm, init, sizeof(init), cudaMemcpyHostToDevice, st), "memcpy");
  if (M) {
    k_check_pack<<<grid_for(M), 256, 0, st>>>(d_src, d_dst, d_t, M, n, err, tmm, pack);
    TC_LAUNCHED(1);
    TRY_C(cudaGetLastError(), "k_check_pack");
  }
  uint32_t h_err = 0;
  long long h_tmm[2];
  TRY_C(cudaMemcpyAsync(&h_err, err, sizeof(h_err), cudaMemcpyDeviceToHost, st), "memcpy");
  TRY_C(cudaMemcpyAsync(h_tmm, tmm, sizeof(h_tmm), cudaMemcpyDeviceToHost, st), "memcpy");
  TRY_C(cudaStreamSynchronize(st), "sync");
  if (h_err & kErrBadId) return done(set_error(TC_ERR_INVALID_ARG, "vertex id outside [0, n)"));
  g->tmin = M ? h_tmm[0] : 0;
  g->tmax = M ? h_tmm[1] : 0;

  TRY_S(dmalloc(&ka, M, st));
  TRY_S(dmalloc(&va, M, st));
  TRY_S(dmalloc(&kb, M, st));
  TRY_S(dmalloc(&vb, M, st));
  TRY_S(dmalloc(&permT, M, st));
  TRY_S(dmalloc(&canon, M, st));
  const unsigned gr = grid_for(M);
  const uint64_t span = (uint64_t)g->tmax - (uint64_t)g->tmin;
  g->out_t32 = g->in_t32 = g->pair_t32 = nullptr;
  if (M && span <= 0xFFFFFFFFull) {  // the list times as 32-bit offsets from tmin
    TRY_S(dmalloc(&g->out_t32, M, st));
    TRY_S(dmalloc(&g->in_t32, M, st));
    TRY_S(dmalloc(&g->pair_t32, M, st));
  }
  const int tbits = bitlen64(span);
  const int vbits = bitlen64((uint64_t)(n > 0 ? n - 1 : 0));

  // 1. by time (stable in input index): low word, then high word
  if (M) {
    k_time_keys<<<gr, 256, 0, st>>>(d_t, M, g->tmin, 0, ka, va);
    TC_LAUNCHED(1);
    TRY_C(cudaGetLastError(), "k_time_keys");
    TRY_S(radix_sort_pairs(ka, va, kb, vb, M, 0, std::min(tbits, 32), st));
    if (tbits > 32) {
      k_high_time_keys<<<gr, 256, 0, st>>>(pack, va, M, g->tmin, ka);
      TC_LAUNCHED(1);
      TRY_C(cudaGetLastError(), "k_high_time_keys");
      TRY_S(radix_sort_pairs(ka, va, kb, vb, M, 0, tbits - 32, st));
    }
    TRY_C(cudaMemcpyAsync(permT, va, sizeof(uint32_t) * M, cudaMemcpyDeviceToDevice, st), "memcpy");
  }

  // 2. out-lists: stable by src of the time order -> (src, t, index)
  if (M) {
    k_gather_key<<<gr, 256, 0, st>>>(d_src, permT, M, ka);
    TC_LAUNCHED(1);
    TRY_C(cudaMemcpyAsync(va, permT, sizeof(uint32_t) * M, cudaMemcpyDeviceToDevice, st), "memcpy");
    TRY_S(radix_sort_pairs(ka, va, kb, vb, M, 0, vbits, st));
    k_fill_out<<<gr, 256, 0, st>>>(pack, va, M, g->out_e, canon, g->tmin, g->out_t32);
    TC_LAUNCHED(1);
    TRY_C(cudaGetLastError(), "k_fill_out");
    TRY_C(cudaMemcpyAsync(g->perm, va, sizeof(uint32_t) * M, cudaMemcpyDeviceToDevice, st), "memcpy");
  }
  k_offsets<<<grid_for(M + 1), 256, 0, st>>>(ka, M, n, g->out_off);
  TC_LAUNCHED(1);
  TRY_C(cudaGetLastError(), "k_offsets");

  // 3. in-lists: stable by dst of the time order -> (dst, t, index)
  if (M) {
    k_gather_key<<<gr, 256, 0, st>>>(d_dst, permT, M, ka);
    TC_LAUNCHED(1);
    TRY_C(cudaMemcpyAsync(va, permT, sizeof(uint32_t) * M, cudaMemcpyDeviceToDevice, st), "memcpy");
    TRY_S(radix_sort_pairs(ka, va, kb, vb, M, 0, vbits, st));
    k_fill_in<<<gr, 256, 0, st>>>(pack, va, canon, M, g->in_e, g->in_eid, g->tmin, g->in_t32);
    TC_LAUNCHED(1);
    TRY_C(cudaGetLastError(), "k_fill_in");
  }
  k_offsets<<<grid_for(M + 1), 256, 0, st>>>(ka, M, n, g->in_off);
  TC_LAUNCHED(1);
  TRY_C(cudaGetLastError(), "k_offsets");

  // window-search anchors of the weights (x_in, x_out, out2in) and their range words
  TRY_S(dmalloc(&g->x_in, M, st));
  TRY_S(dmalloc(&g->x_out, M, st));
  TRY_S(dmalloc(&g->out2in, M, st));
  TRY_S(dmalloc(&g->r_in, M, st));
  TRY_S(dmalloc(&g->r_out, M, st));
  TRY_S(dmalloc(&g->r_o2i, M, st));
  TRY_S(dmalloc(&g->r_self, M, st));
  if (M) {
    if (g->in_t32) {
      k_anchor_in<true><<<gr, 256, 0, st>>>(g->out_e, g->in_e, g->in_off, g->out_off, g->in_t32, g->tmin, M, g->x_in,
                                            g->r_in, g->r_self);
      k_anchor_out<true><<<gr, 256, 0, st>>>(g->out_e, g->in_e, g->in_eid, g->out_off, g->in_off, g->out_t32,
                                             g->tmin, M, g->x_out, g->out2in, g->r_out, g->r_o2i);
    } else {
      k_anchor_in<false><<<gr, 256, 0, st>>>(g->out_e, g->in_e, g->in_off, g->out_off, nullptr, 0, M, g->x_in,
                                             g->r_in, g->r_self);
      k_anchor_out<false><<<gr, 256, 0, st>>>(g->out_e, g->in_e, g->in_eid, g->out_off, g->in_off, nullptr, 0, M,
                                              g->x_out, g->out2in, g->r_out, g->r_o2i);
    }
    TC_LAUNCHED(2);
    TRY_C(cudaGetLastError(), "k_anchor");
  }

  // 4. pair lists: stable by src of the in-list order -> (src, dst, t, index)
  uint32_t P = 0;
  if (M) {
    k_gather_key<<<gr, 256, 0, st>>>(d_src, va, M, ka);
    TC_LAUNCHED(1);
    TRY_S(radix_sort_pairs(ka, va, kb, vb, M, 0, vbits, st));
    TRY_S(dmalloc(&flags, M, st));
    TRY_S(dmalloc(&pidx, M + 1, st));
    TRY_S(dmalloc(&pdst, M, st));
    k_pair_gather<<<gr, 256, 0, st>>>(pack, va, canon, M, pdst, g->pair_t, g->pair_eid, g->tmin, g->pair_t32);
    TC_LAUNCHED(1);
    TRY_C(cudaGetLastError(), "k_pair_gather");
    k_pair_flags<<<gr, 256, 0, st>>>(ka, pdst, M, flags);
    TC_LAUNCHED(1);
    TRY_C(cudaGetLastError(), "k_pair_flags");
    TRY_S(scan_u32(flags, pidx, M, st));
    TRY_C(cudaMemcpyAsync(&P, pidx + M, sizeof(uint32_t), cudaMemcpyDeviceToHost, st), "memcpy");
    TRY_C(cudaStreamSynchronize(st), "sync");
  }
  g->P = P;
  TRY_S(dmalloc(&g->pair_dst, P, st));
  TRY_S(dmalloc(&g->pair_eoff, (uint64_t)P + 1, st));
  TRY_S(dmalloc(&pair_src, P, st));
  if (M) {
    k_fill_pairs<<<gr, 256, 0, st>>>(ka, pdst, flags, pidx, M, g->pair_dst, g->pair_eoff, pair_src);
    TC_LAUNCHED(1);
    TRY_C(cudaGetLastError(), "k_fill_pairs");
  }
  k_set_u32<<<1, 1, 0, st>>>(g->pair_eoff + P, (uint32_t)M);
  TC_LAUNCHED(1);
  TRY_C(cudaGetLastError(), "k_set_u32");
  k_offsets<<<grid_for((uint64_t)P + 1), 256, 0, st>>>(pair_src, P, n, g->pair_off);
  TC_LAUNCHED(1);
  TRY_C(cudaGetLastError(), "k_offsets");
  // pair hash table, capacity the power of two >= max(2, 2P)
  uint64_t cap = 2;
  while (cap < 2ull * P) cap <<= 1;
  g->hash_mask = cap - 1;
  TRY_S(dmalloc(&g->pair_hash, cap, st));
  TRY_C(cudaMemsetAsync(g->pair_hash, 0xFF, sizeof(PairSlot) * cap, st), "memset");
  if (P) {
    k_pair_hash<<<grid_for(P), 256, 0, st>>>(pair_src, g->pair_dst, g->pair_eoff, P, g->pair_hash, g->hash_mask);
    TC_LAUNCHED(1);
    TRY_C(cudaGetLastError(), "k_pair_hash");
  }
  TRY_C(cudaStreamSynchronize(st), "sync");
#undef TRY_S
#undef TRY_C
  return done(TC_OK);
}

// Canonical position -> input index widened to int64 (tc_graph_edge_order).
__global__ void k_widen_u32(const uint32_t* __restrict__ in, uint64_t n, int64_t* __restrict__ out) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = (int64_t)in[i];
}

tc_status launch_widen_u32(const uint32_t* in, uint64_t n, int64_t* out, cudaStream_t st) {
  if (n == 0) return TC_OK;
  uint64_t blocks = (n + 255) / 256;
  const uint64_t cap = (uint64_t)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  k_widen_u32<<<(unsigned)blocks, 256, 0, st>>>(in, n, out);
  TC_LAUNCHED(1);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

}  // namespace tc
