// Learned proposal: edge features, a 16 -> 64 -> 64 -> 1 network (bf16
// operands on the tensor cores through mma.sync m16n8k16, FP32 accumulation,
// FP32 backward and Adam on FP32 master weights) and the proposal
// h_e = max(1, floor(S (eps + g_e) + 1/2)), q_e = w_e h_e.  Sampling middle
// edges proportional to q and weighting each path by Q / h_e keeps the
// estimator of Alg. 5 unbiased (Claim 2 applies path by path).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>

#include "tc_internal.cuh"

namespace tc {

constexpr int kH = 64;      // hidden width
constexpr int kF = 16;      // feature row: 12 edge counts + 4 sample statistics
constexpr int kNFeat = 12;
constexpr int kNParams = kH * kF + kH + kH * kH + kH + kH + 1;  // 5313
// flat parameter layout: W1[64][16], b1[64], W2[64][64], b2[64], W3[64], b3
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH * kF, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH,
              kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH;

}  // namespace tc

struct tc_mlp {
  float* params;  // FP32 master weights (flat layout above)
  float* m1;      // Adam first moments
  float* m2;      // Adam second moments
  float* grad;    // gradient accumulator
  uint32_t* err;  // device error word of the tcgen05 inference kernel
  uint64_t steps;
  int device;
};

namespace tc {

// ---------------------------------------------------------------------------
// Features: counts of the 12 quantities below for canonical edge e = (u, v, t)
// (d1, d3 and w from the sampling index records), log1p in FP32, rounded to
// bf16 (nearest even); columns 12..15 are zero.
//   0 d1, 1 d3, 2 w, 3..6 in/out-degree of u then of v over [t-delta, t+delta],
//   7 sigma_{u,v}[t-delta, t+delta], 8 sigma_{v,u}[t-delta, t+delta] (Def. 3),
//   9 out-degree of u, 10 in-degree of v, 11 in-degree of u.

__device__ __forceinline__ uint32_t count_window(const OutEdge* __restrict__ out_e, const uint32_t* __restrict__ out_off,
                                                 const InEdge* __restrict__ in_e, const uint32_t* __restrict__ in_off,
                                                 bool in_list, int32_t x, int64_t lo, int64_t hi) {
  if (in_list) {
    const uint32_t a = __ldg(in_off + x), b = __ldg(in_off + x + 1);
    auto tt = [&](uint32_t p) { return in_e[p].t; };
    return search_time<false>(a, b, hi, tt) - search_time<true>(a, b, lo, tt);
  }
  const uint32_t a = __ldg(out_off + x), b = __ldg(out_off + x + 1);
  auto tt = [&](uint32_t p) { return out_e[p].t; };
  return search_time<false>(a, b, hi, tt) - search_time<true>(a, b, lo, tt);
}

__device__ __forceinline__ uint32_t pair_count(const PairSlot* __restrict__ table, uint64_t mask,
                                               const int64_t* __restrict__ pair_t, int32_t x, int32_t y, int64_t lo,
                                               int64_t hi) {
  const uint64_t key = pair_key((uint32_t)x, (uint32_t)y);
  uint64_t h = mix64(key) & mask;
  for (uint64_t probe = 0; probe <= mask; probe++) {
    const uint4 slot = __ldg(reinterpret_cast<const uint4*>(table + h));
    if (slot.x == (uint32_t)x && slot.y == (uint32_t)y) {
      auto tt = [&](uint32_t p) { return __ldg(pair_t + p); };
      const uint32_t s = search_time<true>(slot.z, slot.w, lo, tt);
      return search_time<false>(s, slot.w, hi, tt) - s;
    }
    if (slot.x == 0xFFFFFFFFu) return 0;
    h = (h + 1) & mask;
  }
  return 0;
}

__global__ void __launch_bounds__(256) k_features(const OutEdge* __restrict__ out_e,
                                                  const uint32_t* __restrict__ out_off,
                                                  const InEdge* __restrict__ in_e, const uint32_t* __restrict__ in_off,
                                                  const PairSlot* __restrict__ table, uint64_t mask,
                                                  const int64_t* __restrict__ pair_t, const EdgeWin* __restrict__ win,
                                                  uint64_t m, int64_t delta, __nv_bfloat16* __restrict__ feat) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    const EdgeWin r = win[i];
    uint4* dst = reinterpret_cast<uint4*>(feat + i * kF);
    if ((uint64_t)r.d1 * (uint64_t)r.d3 == 0) {  // w = 0: never drawn, never an input of the network
      dst[0] = dst[1] = make_uint4(0, 0, 0, 0);
      continue;
    }
    const OutEdge e = out_e[i];
    const int64_t lo = sat_sub(e.t, delta), hi = sat_add(e.t, delta);
    float c[kNFeat];
    c[0] = (float)r.d1;
    c[1] = (float)r.d3;
    c[2] = (float)((uint64_t)r.d1 * (uint64_t)r.d3);
    c[3] = (float)count_window(out_e, out_off, in_e, in_off, true, e.src, lo, hi);
    c[4] = (float)count_window(out_e, out_off, in_e, in_off, false, e.src, lo, hi);
    c[5] = (float)count_window(out_e, out_off, in_e, in_off, true, e.dst, lo, hi);
    c[6] = (float)count_window(out_e, out_off, in_e, in_off, false, e.dst, lo, hi);
    c[7] = (float)pair_count(table, mask, pair_t, e.src, e.dst, lo, hi);
    c[8] = (float)pair_count(table, mask, pair_t, e.dst, e.src, lo, hi);
    c[9] = (float)(__ldg(out_off + e.src + 1) - __ldg(out_off + e.src));
    c[10] = (float)(__ldg(in_off + e.dst + 1) - __ldg(in_off + e.dst));
    c[11] = (float)(__ldg(in_off + e.src + 1) - __ldg(in_off + e.src));
    __align__(16) __nv_bfloat16 row[kF];
#pragma unroll
    for (int j = 0; j < kNFeat; j++) row[j] = __float2bfloat16_rn(log1pf(c[j]));
#pragma unroll
    for (int j = kNFeat; j < kF; j++) row[j] = __float2bfloat16_rn(0.0f);
    dst[0] = reinterpret_cast<const uint4*>(row)[0];
    dst[1] = reinterpret_cast<const uint4*>(row)[1];
  }
}

// ---------------------------------------------------------------------------
// Sample-statistics features (columns 12..15 of a feature row) from n plain
// samples (middle edge e_i, outcome X_i): with the time bucket
// b(t) = (floor(t / D) - floor(t_min / D)) mod 2^32, D = max(delta, 1), and the
// keys K1 = (u, v), K2 = (u, b(t)), K3 = (v, b(t)) of an edge, n_K counts the
// samples whose middle edge has key K and s_K sums their X^2; prior = sum X^2
// / n.  Columns: log1p((s_K + prior) / (n_K + 1)) for K1, K2, K3, and
// log1p(n_K1).  Per key kind one open-addressing table (SplitMix64 finaliser,
// linear probing, load at most 2/3) with exact integer counts and sums.

constexpr uint64_t kTeEmpty = ~0ull;  // no real key: vertex ids are below 2^31

struct TeTables {
  unsigned long long* key;  // [3][cap]
  unsigned long long* sum;  // [3][cap] sum of X^2
  uint32_t* cnt;            // [3][cap]
  uint64_t cap;             // power of two
};

__device__ __forceinline__ int64_t floor_div(int64_t a, int64_t d) {
  const int64_t q = a / d;
  return (a % d != 0 && a < 0) ? q - 1 : q;
}

__device__ __forceinline__ void te_keys(int32_t u, int32_t v, int64_t t, int64_t D, int64_t b0, uint64_t* k) {
  const uint64_t b = ((uint64_t)floor_div(t, D) - (uint64_t)b0) & 0xFFFFFFFFull;
  k[0] = ((uint64_t)(uint32_t)u << 32) | (uint32_t)v;
  k[1] = ((uint64_t)(uint32_t)u << 32) | b;
  k[2] = ((uint64_t)(uint32_t)v << 32) | b;
}

__global__ void __launch_bounds__(256) k_te_insert(const uint64_t* __restrict__ trace, uint64_t n,
                                                   const OutEdge* __restrict__ out_e, uint64_t m, int64_t D,
                                                   int64_t b0, TeTables T, unsigned long long* __restrict__ total,
                                                   uint32_t* __restrict__ err) {
  unsigned long long local = 0;
  uint32_t bad = 0;
  const uint64_t mask = T.cap - 1;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t e = trace[4 * i], X = trace[4 * i + 3];
    if (e >= m) {
      bad |= kErrBounds;
      continue;
    }
    if (X >> 32) bad |= kErrOverflow;
    const unsigned long long x2 = (unsigned long long)X * X;
    local += x2;
    const OutEdge r = out_e[e];
    uint64_t k[3];
    te_keys(r.src, r.dst, r.t, D, b0, k);
#pragma unroll
    for (int c = 0; c < 3; c++) {
      unsigned long long* keys = T.key + c * T.cap;
      uint64_t h = mix64(k[c]) & mask;
      bool done = false;
      for (uint64_t probe = 0; probe <= mask && !done; probe++) {
        const unsigned long long prev = atomicCAS(keys + h, kTeEmpty, (unsigned long long)k[c]);
        if (prev == kTeEmpty || prev == k[c]) {
          atomicAdd(T.cnt + c * T.cap + h, 1u);
          if (x2) atomicAdd(T.sum + c * T.cap + h, x2);
          done = true;
        }
        h = (h + 1) & mask;
      }
      if (!done) bad |= kErrBounds;
    }
  }
  for (int o = 16; o > 0; o >>= 1) local += __shfl_down_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0 && local) atomicAdd(total, local);
  if (bad) atomicOr(err, bad);
}

__global__ void __launch_bounds__(256) k_te_lookup(const OutEdge* __restrict__ out_e,
                                                   const uint64_t* __restrict__ prefix, uint64_t m, uint64_t n,
                                                   int64_t D, int64_t b0, TeTables T,
                                                   const unsigned long long* __restrict__ total,
                                                   __nv_bfloat16* __restrict__ feat) {
  const float prior = n ? (float)((double)*total / (double)n) : 0.f;  // FP32 below: the result is log1p'd to bf16
  const uint64_t mask = T.cap - 1;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
    if (__ldg(prefix + i + 1) == __ldg(prefix + i)) continue;  // w = 0: the row stays as it is (zero)
    const OutEdge r = out_e[i];
    uint64_t k[3];
    te_keys(r.src, r.dst, r.t, D, b0, k);
    __align__(8) __nv_bfloat16 col[4];
    uint32_t n1 = 0;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const unsigned long long* keys = T.key + c * T.cap;
      uint64_t h = mix64(k[c]) & mask;
      uint32_t cnt = 0;
      unsigned long long s = 0;
      for (uint64_t probe = 0; probe <= mask; probe++) {
        const unsigned long long kk = keys[h];
        if (kk == k[c]) {
          cnt = T.cnt[c * T.cap + h];
          s = T.sum[c * T.cap + h];
          break;
        }
        if (kk == kTeEmpty) break;
        h = (h + 1) & mask;
      }
      if (c == 0) n1 = cnt;
      col[c] = __float2bfloat16_rn(log1pf(((float)s + prior) / ((float)cnt + 1.f)));
    }
    col[3] = __float2bfloat16_rn(log1pf((float)n1));
    *reinterpret_cast<uint2*>(feat + i * kF + kNFeat) = *reinterpret_cast<const uint2*>(col);
  }
}

// ---------------------------------------------------------------------------
// Network on the tensor cores.  One warp computes a tile of 16 rows.
// Fragment layout of mma.m16n8k16 (g = lane / 4, q = lane % 4):
//   A (16x16, row-major): regs (g, 2q..2q+1), (g+8, 2q..), (g, 2q+8..), (g+8, 2q+8..)
//   B (16x8):             regs (k = 2q..2q+1, n = g), (k = 2q+8..2q+9, n = g)
//   C (16x8):             (g, 2q), (g, 2q+1), (g+8, 2q), (g+8, 2q+1)

// Row strides of the weights in shared memory, padded so that the lanes of
// a fragment load (8 rows g x 4 column pairs q) and of the backward's column
// walk fall in distinct banks: a 48-byte W1 row puts lane (g, q) in bank
// 12 g + q, a 144-byte W2 row in bank 4 g + q (mod 32), a 132-byte W2^T row
// lane k in bank k + const.
constexpr int kW1S = 24, kW2S = 72, kW2TS = 66;

struct MlpShared {
  __nv_bfloat16 W1[kH * kW1S];   // [n][k]
  __nv_bfloat16 W2[kH * kW2S];   // [n][k]
  __nv_bfloat16 W2T[kH * kW2TS];  // [k][n]
  float W3[kH];                // bf16 values held as FP32
  float b1[kH], b2[kH];
  float b3;
};

__device__ __forceinline__ void load_mlp_shared(MlpShared& S, const float* __restrict__ p) {
  for (int i = threadIdx.x; i < kH * kF; i += blockDim.x)
    S.W1[(i / kF) * kW1S + i % kF] = __float2bfloat16_rn(p[kOffW1 + i]);
  for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) {
    const __nv_bfloat16 v = __float2bfloat16_rn(p[kOffW2 + i]);
    S.W2[(i / kH) * kW2S + i % kH] = v;
    S.W2T[(i % kH) * kW2TS + i / kH] = v;
  }
  for (int i = threadIdx.x; i < kH; i += blockDim.x) {
    S.W3[i] = __bfloat162float(__float2bfloat16_rn(p[kOffW3 + i]));
    S.b1[i] = p[kOffB1 + i];
    S.b2[i] = p[kOffB2 + i];
  }
  if (threadIdx.x == 0) S.b3 = p[kOffB3];
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}

// A fragment of 16 feature rows; row index r < 0 means a zero row.
__device__ __forceinline__ void load_rows(const __nv_bfloat16* __restrict__ feat, int64_t ra, int64_t rb,
                                          uint32_t (&a)[4]) {
  const int q = threadIdx.x & 3;
  const uint32_t* fa = ra >= 0 ? reinterpret_cast<const uint32_t*>(feat + ra * kF) : nullptr;
  const uint32_t* fb = rb >= 0 ? reinterpret_cast<const uint32_t*>(feat + rb * kF) : nullptr;
  a[0] = fa ? __ldg(fa + q) : 0u;
  a[1] = fb ? __ldg(fb + q) : 0u;
  a[2] = fa ? __ldg(fa + 4 + q) : 0u;
  a[3] = fb ? __ldg(fb + 4 + q) : 0u;
}

// Forward of one tile: z1, z2 (pre-activations, FP32) and a2 (bf16 values as
// FP32) in C-fragment layout, and z3 for rows g and g + 8.
struct TileAct {
  float z1[8][4];
  float z2[8][4];
  float z3g, z3g8;
};

__device__ __forceinline__ void tile_forward(const MlpShared& S, const uint32_t (&x)[4], TileAct& T) {
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  // layer 1: [16 x 16] x [16 x 64]
#pragma unroll
  for (int j = 0; j < 8; j++) {
    const int n = j * 8 + g;
    float c[4] = {S.b1[j * 8 + 2 * q], S.b1[j * 8 + 2 * q + 1], S.b1[j * 8 + 2 * q], S.b1[j * 8 + 2 * q + 1]};
    mma_bf16(c, x, ld_pair(&S.W1[n * kW1S + 2 * q]), ld_pair(&S.W1[n * kW1S + 2 * q + 8]));
#pragma unroll
    for (int r = 0; r < 4; r++) T.z1[j][r] = c[r];
  }
  // ReLU, bf16, as the A fragments of layer 2
  uint32_t a1[4][4];
#pragma unroll
  for (int kk = 0; kk < 4; kk++) {
    a1[kk][0] = pack_bf16(fmaxf(T.z1[2 * kk][0], 0.f), fmaxf(T.z1[2 * kk][1], 0.f));
    a1[kk][1] = pack_bf16(fmaxf(T.z1[2 * kk][2], 0.f), fmaxf(T.z1[2 * kk][3], 0.f));
    a1[kk][2] = pack_bf16(fmaxf(T.z1[2 * kk + 1][0], 0.f), fmaxf(T.z1[2 * kk + 1][1], 0.f));
    a1[kk][3] = pack_bf16(fmaxf(T.z1[2 * kk + 1][2], 0.f), fmaxf(T.z1[2 * kk + 1][3], 0.f));
  }
  // layer 2: [16 x 64] x [64 x 64]
#pragma unroll
  for (int j = 0; j < 8; j++) {
    const int n = j * 8 + g;
    float c[4] = {S.b2[j * 8 + 2 * q], S.b2[j * 8 + 2 * q + 1], S.b2[j * 8 + 2 * q], S.b2[j * 8 + 2 * q + 1]};
#pragma unroll
    for (int kk = 0; kk < 4; kk++)
      mma_bf16(c, a1[kk], ld_pair(&S.W2[n * kW2S + kk * 16 + 2 * q]), ld_pair(&S.W2[n * kW2S + kk * 16 + 2 * q + 8]));
#pragma unroll
    for (int r = 0; r < 4; r++) T.z2[j][r] = c[r];
  }
  // layer 3 in FP32 on the bf16-rounded activations, reduced over the 4 lanes of a row
  float sg = 0.f, sg8 = 0.f;
#pragma unroll
  for (int j = 0; j < 8; j++) {
    const int n0 = j * 8 + 2 * q;
    sg += __bfloat162float(__float2bfloat16_rn(fmaxf(T.z2[j][0], 0.f))) * S.W3[n0] +
          __bfloat162float(__float2bfloat16_rn(fmaxf(T.z2[j][1], 0.f))) * S.W3[n0 + 1];
    sg8 += __bfloat162float(__float2bfloat16_rn(fmaxf(T.z2[j][2], 0.f))) * S.W3[n0] +
           __bfloat162float(__float2bfloat16_rn(fmaxf(T.z2[j][3], 0.f))) * S.W3[n0 + 1];
  }
  sg += __shfl_xor_sync(0xffffffffu, sg, 1);
  sg += __shfl_xor_sync(0xffffffffu, sg, 2);
  sg8 += __shfl_xor_sync(0xffffffffu, sg8, 1);
  sg8 += __shfl_xor_sync(0xffffffffu, sg8, 2);
  T.z3g = sg + S.b3;
  T.z3g8 = sg8 + S.b3;
}

__device__ __forceinline__ float sigmoidf_(float z) { return 1.0f / (1.0f + expf(-z)); }

// Logits of rows (rows[i] or i) -> out[i].


// Logits of one 16-row tile for rows g and g + 8 of the fragment layout: the
// forward of tile_forward without keeping the pre-activations (inference).
struct MlpFwdShared {
  __nv_bfloat16 W1[kH * kW1S];  // [n][k], padded rows as in MlpShared
  __nv_bfloat16 W2[kH * kW2S];  // [n][k]
  float W3[kH];               // bf16 values held as FP32
  float b1[kH], b2[kH];
  float b3;
};

__device__ __forceinline__ void load_mlp_fwd_shared(MlpFwdShared& S, const float* __restrict__ p) {
  for (int i = threadIdx.x; i < kH * kF; i += blockDim.x)
    S.W1[(i / kF) * kW1S + i % kF] = __float2bfloat16_rn(p[kOffW1 + i]);
  for (int i = threadIdx.x; i < kH * kH; i += blockDim.x)
    S.W2[(i / kH) * kW2S + i % kH] = __float2bfloat16_rn(p[kOffW2 + i]);
  for (int i = threadIdx.x; i < kH; i += blockDim.x) {
    S.W3[i] = __bfloat162float(__float2bfloat16_rn(p[kOffW3 + i]));
    S.b1[i] = p[kOffB1 + i];
    S.b2[i] = p[kOffB2 + i];
  }
  if (threadIdx.x == 0) S.b3 = p[kOffB3];
}

// ReLU of two FP32 values rounded to a bf16 pair (lo in the low half): one
// instruction, the activations' rounding of the forward.
__device__ __forceinline__ uint32_t relu_bf16x2(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

// The network's B fragments held in registers for the whole kernel (the
// weights are the same for every tile): layer 2 (8 output tiles x 4 k-tiles
// x 2 registers) and layer 3 as an 8-column tile whose column 0 is W3 and
// whose other columns are zero, so that the last layer is one more MMA
// chain; layer 1 (K = 16) is read from shared memory.
struct MlpFrags {
  uint32_t w2[8][4][2];
  uint32_t w3[4][2];
  float b3;
};

__device__ __forceinline__ void load_mlp_frags(const MlpFwdShared& S, MlpFrags& F) {
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
#pragma unroll
  for (int j = 0; j < 8; j++) {
    const int n = j * 8 + g;
#pragma unroll
    for (int kk = 0; kk < 4; kk++) {
      F.w2[j][kk][0] = ld_pair(&S.W2[n * kW2S + kk * 16 + 2 * q]);
      F.w2[j][kk][1] = ld_pair(&S.W2[n * kW2S + kk * 16 + 2 * q + 8]);
    }
  }
#pragma unroll
  for (int kk = 0; kk < 4; kk++) {  // B of layer 3: k = kk * 16 + 2q (+8), column n = g (only g = 0 is W3)
    const int k0 = kk * 16 + 2 * q;
    F.w3[kk][0] = g == 0 ? pack_bf16(S.W3[k0], S.W3[k0 + 1]) : 0u;
    F.w3[kk][1] = g == 0 ? pack_bf16(S.W3[k0 + 8], S.W3[k0 + 9]) : 0u;
  }
  F.b3 = S.b3;
}

// Logits of one 16-row tile (rows g and g + 8 of the fragment layout; lanes
// with q = 0 hold them): layer 1 on the tensor cores from shared-memory W1,
// ReLU and bf16 rounding packed straight into the A fragments of the next
// layer, layer 2 and layer 3 from the register fragments.
__device__ __forceinline__ void tile_logits(const MlpFwdShared& S, const MlpFrags& F, const uint32_t (&x)[4],
                                            float* z3g, float* z3g8) {
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  uint32_t a1[4][4];
#pragma unroll
  for (int j = 0; j < 8; j++) {
    const int n = j * 8 + g;
    float c[4] = {S.b1[j * 8 + 2 * q], S.b1[j * 8 + 2 * q + 1], S.b1[j * 8 + 2 * q], S.b1[j * 8 + 2 * q + 1]};
    mma_bf16(c, x, ld_pair(&S.W1[n * kW1S + 2 * q]), ld_pair(&S.W1[n * kW1S + 2 * q + 8]));
    const int kk = j >> 1, hi = (j & 1) * 2;
    a1[kk][hi] = relu_bf16x2(c[0], c[1]);
    a1[kk][hi + 1] = relu_bf16x2(c[2], c[3]);
  }
  // layer 2: k-tile outer, so that the 8 output tiles' MMAs are independent
  // back to back instead of 8 chains of 4 dependent ones
  float c2[8][4];
#pragma unroll
  for (int j = 0; j < 8; j++) {
    c2[j][0] = c2[j][2] = S.b2[j * 8 + 2 * q];
    c2[j][1] = c2[j][3] = S.b2[j * 8 + 2 * q + 1];
  }
#pragma unroll
  for (int kk = 0; kk < 4; kk++)
#pragma unroll
    for (int j = 0; j < 8; j++) mma_bf16(c2[j], a1[kk], F.w2[j][kk][0], F.w2[j][kk][1]);
  uint32_t a2[4][4];
#pragma unroll
  for (int j = 0; j < 8; j++) {
    const int kk = j >> 1, hi = (j & 1) * 2;
    a2[kk][hi] = relu_bf16x2(c2[j][0], c2[j][1]);
    a2[kk][hi + 1] = relu_bf16x2(c2[j][2], c2[j][3]);
  }
  float c3[4] = {F.b3, F.b3, F.b3, F.b3};
#pragma unroll
  for (int kk = 0; kk < 4; kk++) mma_bf16(c3, a2[kk], F.w3[kk][0], F.w3[kk][1]);
  *z3g = c3[0];   // column 0, row g (lanes q = 0)
  *z3g8 = c3[2];  // column 0, row g + 8
}

// Logits of rows (rows[i] or i) -> out[i], with the inference path of the
// proposal (tile_logits).
__global__ void __launch_bounds__(128) k_mlp_forward(const float* __restrict__ params,
                                                     const __nv_bfloat16* __restrict__ feat,
                                                     const uint32_t* __restrict__ rows, uint64_t n,
                                                     float* __restrict__ out) {
  __shared__ MlpFwdShared S;
  load_mlp_fwd_shared(S, params);
  __syncthreads();
  MlpFrags F;
  load_mlp_frags(S, F);
  const int lane = threadIdx.x & 31, g = lane >> 2;
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t tile = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; tile * 16 < n; tile += warps) {
    const uint64_t ia = tile * 16 + g, ib = ia + 8;
    const int64_t ra = ia < n ? (int64_t)(rows ? rows[ia] : ia) : -1;
    const int64_t rb = ib < n ? (int64_t)(rows ? rows[ib] : ib) : -1;
    uint32_t x[4];
    load_rows(feat, ra, rb, x);
    float za, zb;
    tile_logits(S, F, x, &za, &zb);
    if ((lane & 3) == 0) {
      if (ia < n) out[ia] = za;
      if (ib < n) out[ib] = zb;
    }
  }
}

// Proposal: for every canonical edge e with w_e > 0, h_e = max(1,
// floor(scale (eps + g_e) + 1/2)) with g_e = sigmoid(network logit of e's
// feature row), and q_e = w_e h_e with w_e = prefix[e + 1] - prefix[e]; an
// edge with w_e = 0 is never drawn under any proposal, so it gets h_e = 1,
// q_e = 0 and the network is not evaluated on it.  Each tile's sum of q is
// the first level of the reduce-then-scan that writes the q-prefix.
// Persistent blocks (the network is staged in shared memory and its
// fragments in registers once per block) take tiles of kPTile edges in
// turn; the tile's prefix entries arrive in shared memory by cp.async, each
// warp lists the rows of its share of the tile with w > 0 and runs them in
// 16-row sub-tiles on the tensor cores (the next sub-tile's feature rows
// loaded ahead), and h and q are then formed and written coalesced.
constexpr int kPThreads = 128;
constexpr int kPRowsPerWarp = 512;
constexpr int kPTile = (kPThreads / 32) * kPRowsPerWarp;  // 2048 edges: the scan's tile
constexpr size_t kPDynSmem = 2 * (kPTile + 2) * sizeof(unsigned long long);  // the two prefix buffers

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Blocks per SM the proposal kernel is compiled for (caps its registers; the
// network's fragments take about 80 of them).
#ifndef TC_PROPOSAL_MIN_BLOCKS
#define TC_PROPOSAL_MIN_BLOCKS 3
#endif

__global__ void __launch_bounds__(kPThreads, TC_PROPOSAL_MIN_BLOCKS) k_proposal(const float* __restrict__ params,
                                                                              const __nv_bfloat16* __restrict__ feat,
                                                                              const uint64_t* __restrict__ prefix,
                                                                              uint64_t m, float eps, float scale,
                                                                              uint16_t* __restrict__ h,
                                                                              uint64_t* __restrict__ q,
                                                                              uint64_t* __restrict__ tile_sums,
                                                                              uint32_t* __restrict__ hrange,
                                                                              uint32_t* __restrict__ d_err) {
  extern __shared__ unsigned long long s_pre2[];  // two buffers of kPTile + 1 prefix entries (kPDynSmem)
  __shared__ MlpFwdShared net;
  __shared__ float s_z[kPTile];
  __shared__ uint16_t s_rows[kPThreads / 32][kPRowsPerWarp];  // a warp's rows with w > 0 (tile offsets)
  __shared__ unsigned long long s_warp[kPThreads / 32];
  __shared__ uint32_t s_err;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, g = lane >> 2, qd = lane & 3;
  load_mlp_fwd_shared(net, params);
  if (tid == 0) s_err = 0;
  __syncthreads();
  MlpFrags F;
  load_mlp_frags(net, F);
  const uint64_t T = (m + kPTile - 1) / kPTile;
  uint32_t err = 0, hlo = 0xFFFFFFFFu, hhi = 0;
  // the prefix entries of a tile (and the next one's after it) arrive by cp.async
  auto prefetch = [&](uint64_t tl, unsigned long long* dst) {
    const uint64_t b = tl * kPTile;
    const uint32_t n = (uint32_t)(m - b < (uint64_t)kPTile ? m - b : (uint64_t)kPTile);
    for (uint32_t i = tid; i <= n; i += kPThreads) cp_async8(dst + i, prefix + b + i);
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  int buf = 0;
  if ((uint64_t)blockIdx.x < T) prefetch(blockIdx.x, s_pre2);
  for (uint64_t tile = blockIdx.x; tile < T; tile += gridDim.x) {
    const uint64_t base = tile * kPTile;
    const uint32_t rows = (uint32_t)(m - base < (uint64_t)kPTile ? m - base : (uint64_t)kPTile);
    unsigned long long* s_pre = s_pre2 + buf * (kPTile + 2);
    __syncthreads();  // the previous tile's shared arrays are consumed
    if (tile + gridDim.x < T) {
      prefetch(tile + gridDim.x, s_pre2 + (buf ^ 1) * (kPTile + 2));
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      cp_async_wait_all();
    }
    __syncthreads();
    buf ^= 1;
    // this warp's rows with w > 0, in order
    const uint32_t r0 = (uint32_t)wid * kPRowsPerWarp;
    uint32_t nz = 0;
    for (uint32_t r = 0; r < kPRowsPerWarp; r += 32) {
      const uint32_t row = r0 + r + lane;
      const bool live = row < rows && s_pre[row + 1] != s_pre[row];
      const uint32_t mask = __ballot_sync(0xffffffffu, live);
      if (live) s_rows[wid][nz + __popc(mask & ((1u << lane) - 1u))] = (uint16_t)row;
      nz += __popc(mask);
    }
    __syncwarp();
    auto fetch = [&](uint32_t sub, uint32_t (&x)[4]) {
      const uint32_t ia = sub * 16 + g, ib = ia + 8;
      load_rows(feat, ia < nz ? (int64_t)(base + s_rows[wid][ia]) : -1,
                ib < nz ? (int64_t)(base + s_rows[wid][ib]) : -1, x);
    };
    const uint32_t subs = (nz + 15) / 16;
    uint32_t xn[4];
    if (subs) fetch(0, xn);
#pragma unroll 1
    for (uint32_t sub = 0; sub < subs; sub++) {
      uint32_t x[4] = {xn[0], xn[1], xn[2], xn[3]};
      if (sub + 1 < subs) fetch(sub + 1, xn);
      float za, zb;
      tile_logits(net, F, x, &za, &zb);
      const uint32_t ia = sub * 16 + g, ib = ia + 8;
      if (qd == 0) {
        if (ia < nz) s_z[s_rows[wid][ia]] = za;
        if (ib < nz) s_z[s_rows[wid][ib]] = zb;
      }
    }
    __syncthreads();
    unsigned long long sum = 0;
    for (uint32_t r = tid; r < rows; r += kPThreads) {
      const unsigned long long wv = s_pre[r + 1] - s_pre[r];
      uint32_t hv = 1;  // w = 0: never drawn, the network was not run on it
      if (wv) {
        const float v = floorf(scale * (eps + sigmoidf_(s_z[r])) + 0.5f);
        hv = v < 1.f ? 1u : (uint32_t)v;
        hlo = hv < hlo ? hv : hlo;
        hhi = hv > hhi ? hv : hhi;
      }
      if (__umul64hi(wv, hv)) err |= kErrOverflow;
      const unsigned long long qv = wv * hv;
      q[base + r] = qv;
      h[base + r] = (uint16_t)hv;
      if (sum + qv < sum) err |= kErrOverflow;
      sum += qv;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long y = __shfl_xor_sync(0xffffffffu, sum, o);
      if (sum + y < sum) err |= kErrOverflow;
      sum += y;
    }
    if (lane == 0) s_warp[wid] = sum;
    __syncthreads();
    if (tid == 0) {
      unsigned long long t = 0;
      for (int v = 0; v < kPThreads / 32; v++) {
        if (t + s_warp[v] < t) err |= kErrOverflow;
        t += s_warp[v];
      }
      tile_sums[tile] = t;
    }
  }
  // the proposal's range of h over the edges with w > 0, for the sampler's per-block bins
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    hlo = min(hlo, __shfl_xor_sync(0xffffffffu, hlo, o));
    hhi = max(hhi, __shfl_xor_sync(0xffffffffu, hhi, o));
  }
  if (lane == 0 && hhi) {
    atomicMin(hrange, hlo);
    atomicMax(hrange + 1, hhi);
  }
  if (err) atomicOr(&s_err, err);
  __syncthreads();
  if (tid == 0 && s_err) atomicOr(d_err, s_err);
}

// ---------------------------------------------------------------------------
// The network on the fifth-generation tensor cores (tcgen05): 128 rows per
// MMA, accumulators in tensor memory (TMEM), operands in shared memory in the
// canonical K-major layout without swizzle, one thread issuing the MMAs and
// an mbarrier signalling their completion.  Each of the 128 threads owns one
// row: it stages its feature row, reads its row of each layer's
// accumulators back with tcgen05.ld, applies bias, ReLU and bf16 rounding
// (the same arithmetic as the oracle's quantised forward), and stages the
// next layer's operand; the last layer (64 -> 1) is an FP32 dot product in
// the thread.

// K-major operand without swizzle: 8-row x 16-byte core matrices; element
// (r, k) of a bf16 matrix with K columns lies at byte
//   (r / 8) * SBO + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2,
// SBO = 16 K bytes (the core matrices of one 8-row group side by side along K,
// 128 bytes apart: the leading-dimension offset).
__device__ __forceinline__ uint32_t umma_offset(uint32_t r, uint32_t k, uint32_t K) {
  return (r >> 3) * (16u * K) + (k >> 3) * 128u + (r & 7u) * 16u + (k & 7u) * 2u;
}

// Shared-memory matrix descriptor (start address, leading-dimension byte
// offset = 128, stride-dimension byte offset, descriptor version 1, no swizzle).
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and
// B bf16 (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at
// bits 24-28.
constexpr uint32_t kUmmaM = 128, kUmmaN = 64;
constexpr uint32_t kIdescBf16 = (1u << 4) | (1u << 7) | (1u << 10) | ((kUmmaN >> 3) << 17) | ((kUmmaM >> 4) << 24);
constexpr uint32_t kTmemCols = 64;  // D1, then D2, at columns 0..63

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, bool accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIdescBf16), "r"((uint32_t)accumulate));
}
__device__ __forceinline__ void umma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(mbar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void tc05_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc05_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; j++) v[j] = __uint_as_float(r[j]);
}

struct alignas(1024) UmmaShared {
  __nv_bfloat16 A1[kUmmaM * kF];  // this sub-tile's feature rows
  __nv_bfloat16 B1[kH * kF];      // W1 [n][k]
  __nv_bfloat16 A2[kUmmaM * kH];  // layer-1 activations
  __nv_bfloat16 B2[kH * kH];      // W2 [n][k]
  alignas(16) float b1[kH];
  alignas(16) float b2[kH];
  alignas(16) float W3[kH];        // W3 as bf16 values held in FP32
  float b3;
  uint64_t mbar;
  uint32_t tmem;
  uint32_t err;
  unsigned long long red[4];
  uint32_t wcnt[4];                          // rows with w > 0 in each warp's quarter of the tile
  unsigned long long pre[16 * kUmmaM + 1];   // the tile's prefix entries (proposal)
  uint16_t live[16 * kUmmaM];                // the tile's rows with w > 0, in order (proposal)
};
// At least 30 KB of shared memory per block, so that at most seven blocks
// share an SM (8 x 31 KB exceeds the SM's 228 KB): their TMEM (kTmemCols
// each) then always fits the 512 columns of an SM and no allocation waits.
constexpr size_t kUmmaSmemBytes =
    sizeof(UmmaShared) + 1024 > 30 * 1024 ? sizeof(UmmaShared) + 1024 : 30 * 1024;
static_assert(7 * kTmemCols <= 512, "TMEM of the blocks one SM can hold");
static_assert(kUmmaSmemBytes * 4 <= 227 * 1024, "four blocks per SM");
constexpr int kUmmaSubTiles = 16;                         // 128-row sub-tiles per tile
constexpr uint64_t kUmmaTile = kUmmaSubTiles * kUmmaM;     // 2048 rows: the scan's tile
constexpr int kUmmaBlocksPerSm = 4;                        // resident blocks (launch bounds, shared memory)
constexpr uint64_t kUmmaWaitNs = 1000000000ull;            // bound of each completion wait: 1 s

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits for the MMAs committed to the barrier (phase parity), at most
// kUmmaWaitNs of wall time; false when the wait gave up.  The MMAs of one
// sub-tile take well under a microsecond.
__device__ __forceinline__ bool umma_wait(uint64_t* mbar, uint32_t parity) {
  if (mbar_try_wait(mbar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(mbar, parity))
    if (global_ns() - t0 > kUmmaWaitNs) return false;
  return true;
}

// For the rows of the tiles this block takes (rows[i] or i index the
// feature rows), the logits (Proposal = false: into logits), or (Proposal =
// true) h, q = w h and each 2048-row tile's sum of q as k_proposal computes
// them: the tile's prefix entries are staged in shared memory, the rows with
// w > 0 listed in order, and only those go through the network, 128 to a
// sub-tile (rows with w = 0 get h = 1, q = 0).
template <bool Proposal>
__global__ void __launch_bounds__(kUmmaM, kUmmaBlocksPerSm) k_mlp_umma(const float* __restrict__ params,
                                                      const __nv_bfloat16* __restrict__ feat,
                                                      const uint32_t* __restrict__ rows, uint64_t n,
                                                      float* __restrict__ logits, const uint64_t* __restrict__ prefix,
                                                      float eps, float scale, uint16_t* __restrict__ h,
                                                      uint64_t* __restrict__ q, uint64_t* __restrict__ tile_sums,
                                                      uint32_t* __restrict__ hrange, uint32_t* __restrict__ d_err) {
  extern __shared__ __align__(1024) unsigned char umma_raw[];
  UmmaShared& S = *reinterpret_cast<UmmaShared*>(
      umma_raw + ((1024u - (smem_u32(umma_raw) & 1023u)) & 1023u));  // 1024-byte aligned in the window
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // the weights as bf16 operands in the canonical layout, biases and W3
  for (int i = tid; i < kH * kF; i += kUmmaM)
    S.B1[umma_offset(i / kF, i % kF, kF) / 2] = __float2bfloat16_rn(params[kOffW1 + i]);
  for (int i = tid; i < kH * kH; i += kUmmaM)
    S.B2[umma_offset(i / kH, i % kH, kH) / 2] = __float2bfloat16_rn(params[kOffW2 + i]);
  if (tid < kH) {
    S.b1[tid] = params[kOffB1 + tid];
    S.b2[tid] = params[kOffB2 + tid];
    S.W3[tid] = __bfloat162float(__float2bfloat16_rn(params[kOffW3 + tid]));
  }
  if (tid == 0) {
    S.b3 = params[kOffB3];
    S.err = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  tc05_fence_before();
  __syncthreads();
  tc05_fence_after();
  const uint32_t tmem = S.tmem;
  const uint32_t lane_addr = (uint32_t)(warp * 32) << 16;  // this warp's 32 TMEM lanes (= rows)
  const uint32_t a1 = smem_u32(S.A1), b1 = smem_u32(S.B1), a2 = smem_u32(S.A2), b2 = smem_u32(S.B2);
  uint32_t parity = 0, err = 0, hlo = 0xFFFFFFFFu, hhi = 0;
  bool ok = true;
  // a block's unit of work: a 2048-row scan tile (proposal) or one 128-row
  // sub-tile (logits, so that small row sets still spread over the SMs)
  constexpr uint64_t kTile = Proposal ? kUmmaTile : kUmmaM;
  const uint64_t T = (n + kTile - 1) / kTile;
  for (uint64_t tile = blockIdx.x; tile < T && ok; tile += gridDim.x) {
    const uint64_t base = tile * kTile;
    const uint32_t trows = (uint32_t)(n - base < kTile ? n - base : kTile);
    // the rows that go through the network: every row of the tile (logits),
    // or the rows with w > 0, listed in order (proposal)
    uint32_t nrun = trows;
    if (Proposal) {
      __syncthreads();  // the previous tile's lists are consumed
      for (uint32_t i = tid; i <= trows; i += kUmmaM) S.pre[i] = __ldg(prefix + base + i);
      __syncthreads();
      const uint32_t q0 = (uint32_t)warp * (kUmmaTile / 4);  // this warp's quarter of the tile
      uint32_t cnt = 0;
      for (uint32_t r = 0; r < kUmmaTile / 4; r += 32) {
        const uint32_t row = q0 + r + lane;
        const bool live = row < trows && S.pre[row + 1] != S.pre[row];
        cnt += __popc(__ballot_sync(0xffffffffu, live));
      }
      if (lane == 0) S.wcnt[warp] = cnt;
      __syncthreads();
      uint32_t at = 0;
      for (int v = 0; v < warp; v++) at += S.wcnt[v];
      for (uint32_t r = 0; r < kUmmaTile / 4; r += 32) {
        const uint32_t row = q0 + r + lane;
        const bool live = row < trows && S.pre[row + 1] != S.pre[row];
        const uint32_t mask = __ballot_sync(0xffffffffu, live);
        if (live) S.live[at + __popc(mask & ((1u << lane) - 1u))] = (uint16_t)row;
        at += __popc(mask);
      }
      nrun = S.wcnt[0] + S.wcnt[1] + S.wcnt[2] + S.wcnt[3];
      __syncthreads();
    }
    unsigned long long tsum = 0;
    // this thread's feature row of a sub-tile (zero past the rows to run); the
    // next sub-tile's row is loaded while the current one is on the tensor cores
    auto fetch = [&](uint32_t at, uint4& lo, uint4& hi) {
      lo = hi = make_uint4(0, 0, 0, 0);
      if (at < nrun) {
        const uint64_t r = base + (Proposal ? (uint32_t)S.live[at] : at);
        const uint4* src = reinterpret_cast<const uint4*>(feat + (uint64_t)(rows ? rows[r] : r) * kF);
        lo = __ldg(src);
        hi = __ldg(src + 1);
      }
    };
    uint4 nlo, nhi;
    fetch(tid, nlo, nhi);
    for (uint32_t r0 = 0; r0 < nrun && ok; r0 += kUmmaM) {  // 128-row sub-tiles
      const uint32_t idx = r0 + tid;
      const bool valid = idx < nrun;
      const uint32_t local = Proposal ? (valid ? (uint32_t)S.live[idx] : 0u) : idx;
      const uint64_t row = base + local;
      const uint4 xlo = nlo, xhi = nhi;
      fetch(idx + kUmmaM, nlo, nhi);
      *reinterpret_cast<uint4*>(reinterpret_cast<char*>(S.A1) + umma_offset(tid, 0, kF)) = xlo;
      *reinterpret_cast<uint4*>(reinterpret_cast<char*>(S.A1) + umma_offset(tid, 8, kF)) = xhi;
      fence_async_smem();
      tc05_fence_before();
      __syncthreads();
      tc05_fence_after();
      // layer 1: D1 [128 x 64] = X [128 x 16] W1^T
      if (tid == 0) {
        umma_bf16(tmem, umma_desc(a1, 16 * kF), umma_desc(b1, 16 * kF), false);
        umma_commit(&S.mbar);
      }
      // one thread polls the barrier; the others wait at the block barrier
      ok = __syncthreads_and(tid != 0 || umma_wait(&S.mbar, parity));
      if (!ok) break;  // parity stays that of the phase still pending
      parity ^= 1;
      tc05_fence_after();
#pragma unroll
      for (int c = 0; c < 4; c++) {  // bias, ReLU, bf16: the A operand of layer 2
        float v[16];
        tmem_ld16(tmem + lane_addr + (uint32_t)(c * 16), v);
        float b[16];  // the bias as four 16-byte shared loads
#pragma unroll
        for (int j = 0; j < 4; j++)
          *reinterpret_cast<float4*>(b + 4 * j) = reinterpret_cast<const float4*>(S.b1)[c * 4 + j];
        uint32_t pk[8];
#pragma unroll
        for (int j = 0; j < 8; j++) pk[j] = relu_bf16x2(v[2 * j] + b[2 * j], v[2 * j + 1] + b[2 * j + 1]);
        char* dst = reinterpret_cast<char*>(S.A2);
        *reinterpret_cast<uint4*>(dst + umma_offset(tid, c * 16, kH)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        *reinterpret_cast<uint4*>(dst + umma_offset(tid, c * 16 + 8, kH)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
      }
      fence_async_smem();
      tc05_fence_before();
      __syncthreads();
      tc05_fence_after();
      // layer 2: D2 [128 x 64] = A1 [128 x 64] W2^T, K in four steps of 16, into
      // the columns of D1 (read by every thread before the barrier above)
      if (tid == 0) {
#pragma unroll
        for (int kk = 0; kk < 4; kk++)
          umma_bf16(tmem, umma_desc(a2 + kk * 256, 16 * kH), umma_desc(b2 + kk * 256, 16 * kH), kk > 0);
        umma_commit(&S.mbar);
      }
      // one thread polls the barrier; the others wait at the block barrier
      ok = __syncthreads_and(tid != 0 || umma_wait(&S.mbar, parity));
      if (!ok) break;  // parity stays that of the phase still pending
      parity ^= 1;
      tc05_fence_after();
      float z = S.b3;  // layer 3 in FP32 on the bf16-rounded activations
#pragma unroll
      for (int c = 0; c < 4; c++) {
        float v[16], b[16], w3[16];
        tmem_ld16(tmem + lane_addr + (uint32_t)(c * 16), v);
#pragma unroll
        for (int j = 0; j < 4; j++) {
          *reinterpret_cast<float4*>(b + 4 * j) = reinterpret_cast<const float4*>(S.b2)[c * 4 + j];
          *reinterpret_cast<float4*>(w3 + 4 * j) = reinterpret_cast<const float4*>(S.W3)[c * 4 + j];
        }
#pragma unroll
        for (int j = 0; j < 8; j++) {  // ReLU and bf16 rounding of a pair in one instruction, then widened
          const uint32_t pk = relu_bf16x2(v[2 * j] + b[2 * j], v[2 * j + 1] + b[2 * j + 1]);
          z = fmaf(__uint_as_float(pk << 16), w3[2 * j], z);
          z = fmaf(__uint_as_float(pk & 0xFFFF0000u), w3[2 * j + 1], z);
        }
      }
      tc05_fence_before();  // the next sub-tile's MMAs overwrite D1, D2 after the next barrier
      if (valid) {
        if (!Proposal) {
          logits[row] = z;
        } else {
          const unsigned long long wv = S.pre[local + 1] - S.pre[local];  // > 0: a listed row
          const float fv = floorf(scale * (eps + sigmoidf_(z)) + 0.5f);
          const uint32_t hv = fv < 1.f ? 1u : (uint32_t)fv;
          hlo = hv < hlo ? hv : hlo;
          hhi = hv > hhi ? hv : hhi;
          if (__umul64hi(wv, hv)) err |= kErrOverflow;
          const unsigned long long qv = wv * hv;
          q[row] = qv;
          h[row] = (uint16_t)hv;
          if (tsum + qv < tsum) err |= kErrOverflow;
          tsum += qv;
        }
      }
    }
    if (Proposal && ok) {
      // rows with w = 0 are never drawn: h = 1, q = 0 (as k_proposal)
      for (uint32_t r = tid; r < trows; r += kUmmaM)
        if (S.pre[r + 1] == S.pre[r]) {
          q[base + r] = 0;
          h[base + r] = 1;
        }
      // the tile's sum of q
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, tsum, o);
        if (tsum + y < tsum) err |= kErrOverflow;
        tsum += y;
      }
      if (lane == 0) S.red[warp] = tsum;
      __syncthreads();
      if (tid == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < kUmmaM / 32; w++) {
          if (t + S.red[w] < t) err |= kErrOverflow;
          t += S.red[w];
        }
        tile_sums[tile] = t;
      }
      __syncthreads();
    }
  }
  if (!ok) err |= kErrTimeout;
  if (Proposal) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      hlo = min(hlo, __shfl_xor_sync(0xffffffffu, hlo, o));
      hhi = max(hhi, __shfl_xor_sync(0xffffffffu, hhi, o));
    }
    if (lane == 0 && hhi) {
      atomicMin(hrange, hlo);
      atomicMax(hrange + 1, hhi);
    }
  }
  if (err) atomicOr(&S.err, err);
  tc05_fence_before();
  __syncthreads();
  tc05_fence_after();
  if (!ok && tid == 0) umma_wait(&S.mbar, parity);  // one more bounded wait for MMAs still in flight
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  if (tid == 0 && S.err) atomicOr(d_err, S.err);
}

// ---------------------------------------------------------------------------
// Gradient of the mean closure loss over a batch (the binary cross-entropy
// when every label is 0 or 1), or of any loss whose dloss/dz3 per row is
// given.  Each warp runs the forward of a 16-row tile on the tensor cores and
// back-propagates in FP32:
//   dz3 = (-y (1 - g) if y > 0 else g) / B with g = sigmoid(z3) (or the given
//   dz3), dz2 = dz3 W3 * [z2 > 0], dz1 = W2^T dz2 * [z1 > 0];
// the per-row vectors go to shared memory, where the block accumulates the
// parameter gradients (each thread owns a fixed set of parameters) before one
// global atomic add per parameter and block.

constexpr int kTrainWarps = 4;
// Row tiles of kTrainRows per block of the gradient launch: one tile per
// block puts four times more blocks in flight than four tiles (the parameter
// gradients then take more global atomics, which cost less than the idle
// SMs did: 48 ms instead of 111 ms for 1e7 training rows on the 20M-edge graph).
#ifndef TC_TRAIN_TILES
#define TC_TRAIN_TILES 1
#endif
constexpr int kTrainRows = 16 * kTrainWarps;

// Row strides of the backward's per-row arrays (FP32), padded so that the
// TF32 fragment loads of a warp fall in distinct banks or at worst pairs.
constexpr int kXS = kF + 4, kAS = kH + 4;

struct TrainShared {
  MlpShared net;
  float x[kTrainRows][kXS];
  float a1[kTrainRows][kAS];
  float a2[kTrainRows][kAS];
  float dz1[kTrainRows][kAS];
  float dz2[kTrainRows][kAS];
  float dz3[kTrainRows];
  float loss[kTrainWarps];
};

// D += A B on the tensor cores with TF32 operands (FP32 values rounded to
// TF32, nearest with ties away) and FP32 accumulation, m16n8k8.  Fragment
// layout (g = lane / 4, q = lane % 4): A (16 x 8, row-major) (g, q),
// (g + 8, q), (g, q + 4), (g + 8, q + 4); B (8 x 8) (k = q, n = g),
// (k = q + 4, n = g); C (16 x 8) as the m16n8k16 tile: (g, 2q), (g, 2q + 1),
// (g + 8, 2q), (g + 8, 2q + 1).
__device__ __forceinline__ uint32_t tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Estimator-variance objective over a batch of n rows: with h_i = eps + g_i,
// g_i = sigmoid(z_i), the per-sample second moment of the estimate under the
// proposal is proportional to L = mean(h) * mean(X_i^2 / h_i) (the batch's
// paths come from the plain sampler, so mean(h) estimates Q / W).  Writes
// dL/dz_i into dz and L into *loss.  The per-row terms are FP32 (the
// objective is checked to 1e-3 and its gradient to 1e-2; FP64 arithmetic
// runs at a small fraction of the FP32 rate on this GPU, and a division per
// row in FP64 made this kernel the bulk of a training step); only the sums
// over the batch accumulate in FP64.
__global__ void __launch_bounds__(1024) k_variance_dz(const float* __restrict__ z, const float* __restrict__ X,
                                                      uint64_t n, float eps, float* __restrict__ dz,
                                                      float* __restrict__ loss) {
  __shared__ double s_a[32], s_b[32];
  __shared__ double s_A, s_B;
  double a = 0.0, b = 0.0;
  for (uint64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const float h = eps + sigmoidf_(z[i]);
    const float x = X[i];
    a += (double)h;
    b += (double)(x * x / h);
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    s_a[threadIdx.x >> 5] = a;
    s_b[threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0.0, tb = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
      ta += s_a[w];
      tb += s_b[w];
    }
    s_A = ta / (double)n;
    s_B = tb / (double)n;
    *loss = (float)(s_A * s_B);
  }
  __syncthreads();
  const float A = (float)s_A, B = (float)s_B, inv_n = (float)(1.0 / (double)n);
  for (uint64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const float g = sigmoidf_(z[i]);
    const float h = eps + g;
    const float x = X[i];
    dz[i] = g * (1.f - g) * (B - A * (x / h) * (x / h)) * inv_n;
  }
}

__global__ void __launch_bounds__(32 * kTrainWarps) k_mlp_grad(const float* __restrict__ params,
                                                              const __nv_bfloat16* __restrict__ feat,
                                                              const uint32_t* __restrict__ rows,
                                                              const float* __restrict__ labels, uint64_t n,
                                                              float inv_batch, float* __restrict__ grad,
                                                              float* __restrict__ loss_sum, int given_dz) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrainShared& S = *reinterpret_cast<TrainShared*>(smem_raw);
  load_mlp_shared(S.net, params);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, q = lane & 3;
  // parameter gradients held across the block's row tiles: warp w owns the
  // rows n = 16 w .. 16 w + 15 of dW2 (8 column tiles) and of dW1 (2 column
  // tiles) in C-fragment layout; thread t owns db1[t] (t < 64) or db2[t - 64],
  // and dW3[t] (t < 64) or db3 (t = 64)
  float gw2[8][4], gw1[2][4];
#pragma unroll
  for (int j = 0; j < 8; j++) gw2[j][0] = gw2[j][1] = gw2[j][2] = gw2[j][3] = 0.f;
#pragma unroll
  for (int j = 0; j < 2; j++) gw1[j][0] = gw1[j][1] = gw1[j][2] = gw1[j][3] = 0.f;
  float gb = 0.f, g3 = 0.f;
  float loss_acc = 0.f;
  __syncthreads();
  for (uint64_t base = (uint64_t)blockIdx.x * kTrainRows; base < n; base += (uint64_t)gridDim.x * kTrainRows) {
    // ---- per warp: forward and backward of 16 rows
    const uint64_t ia = base + warp * 16 + g, ib = ia + 8;
    const bool va = ia < n, vb = ib < n;
    uint32_t x[4];
    load_rows(feat, va ? (int64_t)(rows ? rows[ia] : ia) : -1, vb ? (int64_t)(rows ? rows[ib] : ib) : -1, x);
    TileAct T;
    tile_forward(S.net, x, T);
    const int ra = warp * 16 + g, rb = ra + 8;
    // closure count y: loss y softplus(-z) if y > 0, else softplus(z) (the
    // binary cross-entropy when y is 0 or 1); dloss/dz = -y (1 - g) or g
    const float ya = va ? labels[ia] : 0.f, yb = vb ? labels[ib] : 0.f;
    auto dloss = [](float z, float y) { return y > 0.f ? -y * (1.f - sigmoidf_(z)) : sigmoidf_(z); };
    // given_dz: the labels are dloss/dz already (the variance objective)
    const float dza = va ? (given_dz ? ya : dloss(T.z3g, ya) * inv_batch) : 0.f;
    const float dzb = vb ? (given_dz ? yb : dloss(T.z3g8, yb) * inv_batch) : 0.f;
    if (q == 0) {
      S.dz3[ra] = dza;
      S.dz3[rb] = dzb;
      auto softplus = [](float x) { return fmaxf(x, 0.f) + log1pf(expf(-fabsf(x))); };
      auto loss = [&](float z, float y) { return y > 0.f ? y * softplus(-z) : softplus(z); };
      if (!given_dz) loss_acc += (va ? loss(T.z3g, ya) : 0.f) + (vb ? loss(T.z3g8, yb) : 0.f);
    }
    // inputs and activations of the rows (bf16 values held as FP32), and
    // dz2 = dz3 W3 [z2 > 0]
    {
      const __nv_bfloat162* xa = reinterpret_cast<const __nv_bfloat162*>(x);
      S.x[ra][2 * q] = __low2float(xa[0]);
      S.x[ra][2 * q + 1] = __high2float(xa[0]);
      S.x[rb][2 * q] = __low2float(xa[1]);
      S.x[rb][2 * q + 1] = __high2float(xa[1]);
      S.x[ra][2 * q + 8] = __low2float(xa[2]);
      S.x[ra][2 * q + 9] = __high2float(xa[2]);
      S.x[rb][2 * q + 8] = __low2float(xa[3]);
      S.x[rb][2 * q + 9] = __high2float(xa[3]);
    }
#pragma unroll
    for (int j = 0; j < 8; j++) {
      const int c0 = j * 8 + 2 * q;
#pragma unroll
      for (int r = 0; r < 4; r++) {
        const int row = r < 2 ? ra : rb, col = c0 + (r & 1);
        const float z2 = T.z2[j][r];
        S.a1[row][col] = __bfloat162float(__float2bfloat16_rn(fmaxf(T.z1[j][r], 0.f)));
        S.a2[row][col] = __bfloat162float(__float2bfloat16_rn(fmaxf(z2, 0.f)));
        S.dz2[row][col] = z2 > 0.f ? (r < 2 ? dza : dzb) * S.net.W3[col] : 0.f;
      }
    }
    __syncwarp();
    // dz1 = (dz2 W2) [z1 > 0] for the warp's 16 rows on the tensor cores:
    // [16 x 64] (dz2) x [64 x 64] (W2 as (n, k), the layer's bf16 weights)
    {
      const int r0 = warp * 16;
      float d[8][4];
#pragma unroll
      for (int j = 0; j < 8; j++) d[j][0] = d[j][1] = d[j][2] = d[j][3] = 0.f;
#pragma unroll
      for (int kk = 0; kk < 8; kk++) {  // n = 8 kk .. 8 kk + 7
        const uint32_t a0 = tf32(S.dz2[r0 + g][8 * kk + q]), a1 = tf32(S.dz2[r0 + g + 8][8 * kk + q]);
        const uint32_t a2 = tf32(S.dz2[r0 + g][8 * kk + q + 4]), a3 = tf32(S.dz2[r0 + g + 8][8 * kk + q + 4]);
#pragma unroll
        for (int j = 0; j < 8; j++) {  // k = 8 j .. 8 j + 7: B(n, k) = W2[n][k], exact in TF32
          const uint32_t b0 = __float_as_uint(__bfloat162float(S.net.W2[(8 * kk + q) * kW2S + 8 * j + g]));
          const uint32_t b1 = __float_as_uint(__bfloat162float(S.net.W2[(8 * kk + q + 4) * kW2S + 8 * j + g]));
          mma_tf32(d[j], a0, a1, a2, a3, b0, b1);
        }
      }
#pragma unroll
      for (int j = 0; j < 8; j++)
#pragma unroll
        for (int r = 0; r < 4; r++) {
          const int row = r < 2 ? ra : rb, col = j * 8 + 2 * q + (r & 1);
          S.dz1[row][col] = T.z1[j][r] > 0.f ? d[j][r] : 0.f;
        }
    }
    __syncthreads();
    // ---- block: the parameter gradients over the block's 64 rows
    {
      const int m0 = warp * 16;  // this warp's rows n of dW2 and dW1
#pragma unroll
      for (int kk = 0; kk < kTrainRows / 8; kk++) {  // rows 8 kk .. 8 kk + 7
        const int rq = 8 * kk + q, rq4 = rq + 4;
        // dW2[n][k] += sum_row dz2[row][n] a1[row][k]: A(n, row) = dz2[row][n]
        const uint32_t a0 = tf32(S.dz2[rq][m0 + g]), a1 = tf32(S.dz2[rq][m0 + g + 8]);
        const uint32_t a2 = tf32(S.dz2[rq4][m0 + g]), a3 = tf32(S.dz2[rq4][m0 + g + 8]);
#pragma unroll
        for (int j = 0; j < 8; j++)  // a1 values are bf16, exact in TF32
          mma_tf32(gw2[j], a0, a1, a2, a3, __float_as_uint(S.a1[rq][8 * j + g]),
                   __float_as_uint(S.a1[rq4][8 * j + g]));
        // dW1[n][k] += sum_row dz1[row][n] x[row][k]
        const uint32_t c0 = tf32(S.dz1[rq][m0 + g]), c1 = tf32(S.dz1[rq][m0 + g + 8]);
        const uint32_t c2 = tf32(S.dz1[rq4][m0 + g]), c3 = tf32(S.dz1[rq4][m0 + g + 8]);
#pragma unroll
        for (int j = 0; j < 2; j++)
          mma_tf32(gw1[j], c0, c1, c2, c3, __float_as_uint(S.x[rq][8 * j + g]), __float_as_uint(S.x[rq4][8 * j + g]));
      }
      // the biases and the last layer: sums over the rows (FP32)
      const int t = threadIdx.x;
      float sb = 0.f, s3 = 0.f;
      for (int r = 0; r < kTrainRows; r++) {
        sb += t < kH ? S.dz1[r][t] : S.dz2[r][t - kH];
        if (t < kH) s3 += S.dz3[r] * S.a2[r][t];
        else if (t == kH) s3 += S.dz3[r];
      }
      gb += sb;
      g3 += s3;
    }
    __syncthreads();
  }
  {
    const int m0 = warp * 16;
#pragma unroll
    for (int j = 0; j < 8; j++)
#pragma unroll
      for (int r = 0; r < 4; r++) {
        const int nn = m0 + g + (r < 2 ? 0 : 8), k = 8 * j + 2 * q + (r & 1);
        atomicAdd(grad + kOffW2 + nn * kH + k, gw2[j][r]);
      }
#pragma unroll
    for (int j = 0; j < 2; j++)
#pragma unroll
      for (int r = 0; r < 4; r++) {
        const int nn = m0 + g + (r < 2 ? 0 : 8), k = 8 * j + 2 * q + (r & 1);
        atomicAdd(grad + kOffW1 + nn * kF + k, gw1[j][r]);
      }
    const int t = threadIdx.x;
    atomicAdd(grad + (t < kH ? kOffB1 + t : kOffB2 + (t - kH)), gb);
    if (t < kH) atomicAdd(grad + kOffW3 + t, g3);
    else if (t == kH) atomicAdd(grad + kOffB3, g3);
  }
  for (int o = 16; o > 0; o >>= 1) loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, o);
  if (lane == 0) S.loss[warp] = loss_acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < kTrainWarps; w++) t += S.loss[w];
    atomicAdd(loss_sum, t);
  }
}

// Adam (Kingma & Ba, ICLR 2015) on the FP32 master weights; clears grad.
__global__ void k_adam(float* __restrict__ p, float* __restrict__ m1, float* __restrict__ m2,
                       float* __restrict__ grad, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kNParams) return;
  const float gr = grad[i];
  const float a = b1 * m1[i] + (1.f - b1) * gr;
  const float v = b2 * m2[i] + (1.f - b2) * gr * gr;
  m1[i] = a;
  m2[i] = v;
  p[i] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
  grad[i] = 0.f;
}

// Initial weights U(-1/sqrt(fan_in), 1/sqrt(fan_in)) from Philox keyed by
// (seed, parameter index).
__global__ void k_mlp_init(float* __restrict__ p, uint64_t seed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kNParams) return;
  const int fan_in = i < kOffW2 ? kF : kH;
  const uint4 r = philox4x32_10(make_uint4((uint32_t)i, 0u, 0x6d6c7000u, 0u),
                                make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  const float u01 = (float)(r.x >> 8) * (1.0f / 16777216.0f);  // [0, 1)
  p[i] = (2.f * u01 - 1.f) * rsqrtf((float)fan_in);
}

// Training rows from a trace of the plain sampler: row = middle edge,
// label = the closure count X.
// Training rows and labels from a trace: the middle edge and its closure
// count X, or the closure outcome 1[X > 0] (clip).
__global__ void k_trace_to_rows(const uint64_t* __restrict__ trace, uint64_t n, uint32_t* __restrict__ rows,
                                float* __restrict__ labels, bool clip) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    rows[i] = (uint32_t)trace[4 * i];
    const uint64_t X = trace[4 * i + 3];
    labels[i] = clip ? (X ? 1.f : 0.f) : (float)X;
  }
}

// labels_out[i] = 1[labels[i] > 0] (the closure outcome of a count).
__global__ void k_clip_labels(const float* __restrict__ labels, uint64_t n, float* __restrict__ out) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = labels[i] > 0.f ? 1.f : 0.f;
}

static unsigned grid_cap(uint64_t items, int per_block) {
  uint64_t b = (items + per_block - 1) / per_block;
  const uint64_t cap = (uint64_t)num_sms() * 8;
  if (b > cap) b = cap;
  return (unsigned)(b ? b : 1);
}

tc_status mlp_create(uint64_t seed, tc_mlp** out) {
  tc_mlp* M = new (std::nothrow) tc_mlp;
  if (!M) return set_error(TC_ERR_OOM, "host allocation failed");
  std::memset(M, 0, sizeof(*M));
  cudaGetDevice(&M->device);
  float* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, sizeof(float) * (4 * kNParams + 1));
  if (e != cudaSuccess) {
    delete M;
    return cuda_status(e, "cudaMalloc(mlp)");
  }
  M->params = buf;
  M->m1 = buf + kNParams;
  M->m2 = buf + 2 * kNParams;
  M->grad = buf + 3 * kNParams;
  M->err = reinterpret_cast<uint32_t*>(buf + 4 * kNParams);
  e = cudaMemset(buf, 0, sizeof(float) * (4 * kNParams + 1));
  if (e == cudaSuccess) {
    k_mlp_init<<<(kNParams + 255) / 256, 256>>>(M->params, seed);
    TC_LAUNCHED(1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaFree(buf);
    delete M;
    return cuda_status(e, "tc_mlp_create");
  }
  *out = M;
  return TC_OK;
}

void mlp_destroy(tc_mlp* M) {
  if (M->params) cudaFree(M->params);
  delete M;
}

int mlp_num_params() { return kNParams; }

tc_status mlp_set_params(tc_mlp* M, const float* h) {
  TC_CUDA(cudaMemcpy(M->params, h, sizeof(float) * kNParams, cudaMemcpyHostToDevice));
  TC_CUDA(cudaMemset(M->m1, 0, sizeof(float) * 3 * kNParams));
  M->steps = 0;
  return TC_OK;
}

tc_status mlp_get_params(const tc_mlp* M, float* h) {
  TC_CUDA(cudaMemcpy(h, M->params, sizeof(float) * kNParams, cudaMemcpyDeviceToHost));
  return TC_OK;
}

tc_status launch_features(const tc_graph* g, const EdgeWin* win, int64_t delta, uint16_t* feat, cudaStream_t st) {
  const uint64_t m = (uint64_t)g->m;
  if (!m) return TC_OK;
  k_features<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(g->out_e, g->out_off, g->in_e, g->in_off, g->pair_hash,
                                                          g->hash_mask, g->pair_t, win, m, delta,
                                                          reinterpret_cast<__nv_bfloat16*>(feat));
  TC_LAUNCHED(1);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

tc_status launch_sample_features(const tc_graph* g, const uint64_t* prefix, const uint64_t* trace, uint64_t n,
                                 int64_t delta, uint16_t* feat, uint32_t* d_err, cudaStream_t st) {
  const uint64_t m = (uint64_t)g->m;
  if (!m) return TC_OK;
  const int64_t D = delta > 0 ? delta : 1;
  const int64_t b0 = g->tmin / D - ((g->tmin % D != 0 && g->tmin < 0) ? 1 : 0);
  uint64_t cap = 1024;
  while (cap < n + n / 2) cap <<= 1;  // load at most 2/3
  TeTables T;
  T.cap = cap;
  char* buf = nullptr;
  const size_t bytes = 3 * cap * (8 + 8 + 4) + 256;
  TC_CUDA(pool_malloc(&buf, bytes, st));
  T.key = (unsigned long long*)buf;
  T.sum = T.key + 3 * cap;
  T.cnt = (uint32_t*)(T.sum + 3 * cap);
  unsigned long long* total = (unsigned long long*)(buf + 3 * cap * 20);
  tc_status s = TC_OK;
  cudaError_t e = cudaMemsetAsync(T.key, 0xFF, 3 * cap * 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(T.sum, 0, 3 * cap * 12 + 256, st);
  if (e != cudaSuccess) s = cuda_status(e, "cudaMemsetAsync");
  if (s == TC_OK && n) {
    k_te_insert<<<grid_cap(n, 256), 256, 0, st>>>(trace, n, g->out_e, m, D, b0, T, total, d_err);
    TC_LAUNCHED(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) s = cuda_status(e, "k_te_insert");
  }
  if (s == TC_OK) {
    k_te_lookup<<<grid_cap(m, 256), 256, 0, st>>>(g->out_e, prefix, m, n, D, b0, T, total,
                                                   reinterpret_cast<__nv_bfloat16*>(feat));
    TC_LAUNCHED(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) s = cuda_status(e, "k_te_lookup");
  }
  cudaFreeAsync(buf, st);
  return s;
}

// Which network kernel runs inference: the tcgen05 one (TMEM accumulators,
// one thread issuing the MMAs) or the warp-level mma.sync one.  The build
// default is TC_MLP_TCGEN05; the environment variable of the same name
// ("0" or "1") overrides it.
#ifndef TC_MLP_TCGEN05
#define TC_MLP_TCGEN05 1
#endif
static int g_mlp_kernel = -1;
static bool use_tcgen05() {
  if (g_mlp_kernel < 0) {
    const char* e = getenv("TC_MLP_TCGEN05");
    g_mlp_kernel = e && (e[0] == '0' || e[0] == '1') ? e[0] - '0' : TC_MLP_TCGEN05;
  }
  return g_mlp_kernel == 1;
}
int mlp_kernel(int kind) {
  use_tcgen05();
  if (kind > 1) return -1;
  if (kind >= 0) g_mlp_kernel = kind;
  return g_mlp_kernel;
}

template <bool Proposal>
static tc_status launch_umma(const tc_mlp* M, const uint16_t* feat, const uint32_t* rows, uint64_t n, float* logits,
                             const uint64_t* prefix, float eps, float scale, uint16_t* h, uint64_t* q,
                             uint64_t* tile_sums, uint32_t* hrange, uint32_t* d_err, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    TC_CUDA(cudaFuncSetAttribute(k_mlp_umma<Proposal>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kUmmaSmemBytes));
    attr = true;
  }
  // kUmmaBlocksPerSm blocks per SM: what the launch bounds' registers and the
  // shared memory allow (their TMEM, 64 columns each, fits an SM's 512)
  const uint64_t T = Proposal ? (n + kUmmaTile - 1) / kUmmaTile : (n + kUmmaM - 1) / kUmmaM;
  uint64_t blocks = (uint64_t)num_sms() * kUmmaBlocksPerSm;
  if (blocks > T) blocks = T;
  k_mlp_umma<Proposal><<<(unsigned)blocks, kUmmaM, kUmmaSmemBytes, st>>>(
      M->params, reinterpret_cast<const __nv_bfloat16*>(feat), rows, n, logits, prefix, eps, scale, h, q, tile_sums,
      hrange, d_err);
  TC_LAUNCHED(1);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

tc_status launch_mlp_forward(const tc_mlp* M, const uint16_t* feat, const uint32_t* rows, uint64_t n, float* out,
                             cudaStream_t st) {
  if (!n) return TC_OK;
  if (use_tcgen05())
    return launch_umma<false>(M, feat, rows, n, out, nullptr, 0.f, 0.f, nullptr, nullptr, nullptr, nullptr, M->err,
                              st);
  k_mlp_forward<<<grid_cap((n + 15) / 16, 4), 128, 0, st>>>(M->params, reinterpret_cast<const __nv_bfloat16*>(feat),
                                                             rows, n, out);
  TC_LAUNCHED(1);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

// grad (device, kNParams) += gradient of the mean closure loss over rows;
// *loss_sum (device) += summed per-row loss.  given_dz: labels hold dloss/dz3
// per row and no loss is summed.
tc_status launch_mlp_grad(const tc_mlp* M, const uint16_t* feat, const uint32_t* rows, const float* labels,
                          uint64_t n, float* grad, float* loss_sum, cudaStream_t st, bool given_dz) {
  if (!n) return TC_OK;
  static bool attr = false;
  if (!attr) {
    TC_CUDA(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TrainShared)));
    attr = true;
  }
  k_mlp_grad<<<grid_cap(n, kTrainRows * TC_TRAIN_TILES), 32 * kTrainWarps, sizeof(TrainShared), st>>>(
      M->params, reinterpret_cast<const __nv_bfloat16*>(feat), rows, labels, n, 1.0f / (float)n, grad, loss_sum,
      given_dz ? 1 : 0);
  TC_LAUNCHED(1);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

tc_status launch_variance_grad(const tc_mlp* M, const uint16_t* feat, const uint32_t* rows, const float* X,
                               uint64_t n, float eps, float* grad, float* loss, float* z, float* dz,
                               float* loss_scratch, cudaStream_t st) {
  if (!n) return TC_OK;
  TC_TRY(launch_mlp_forward(M, feat, rows, n, z, st));
  k_variance_dz<<<1, 1024, 0, st>>>(z, X, n, eps, dz, loss);
  TC_LAUNCHED(1);
  TC_CUDA(cudaGetLastError());
  return launch_mlp_grad(M, feat, rows, dz, n, grad, loss_scratch, st, true);
}

tc_status mlp_adam(tc_mlp* M, float lr, cudaStream_t st) {
  M->steps++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)M->steps), c2 = 1.f - powf(b2, (float)M->steps);
  k_adam<<<(kNParams + 255) / 256, 256, 0, st>>>(M->params, M->m1, M->m2, M->grad, lr, b1, b2, 1e-8f, c1, c2);
  TC_LAUNCHED(1);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

float* mlp_grad_buffer(tc_mlp* M) { return M->grad; }

tc_status mlp_check_error(const tc_mlp* M, cudaStream_t st, const char* what) {
  uint32_t bits = 0;
  TC_CUDA(cudaMemcpyAsync(&bits, M->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  TC_CUDA(cudaStreamSynchronize(st));
  if (!bits) return TC_OK;
  TC_CUDA(cudaMemsetAsync(M->err, 0, sizeof(uint32_t), st));
  return device_status(bits, what);
}

tc_status launch_clip_labels(const float* labels, uint64_t n, float* out, cudaStream_t st) {
  if (!n) return TC_OK;
  k_clip_labels<<<grid_cap(n, 256), 256, 0, st>>>(labels, n, out);
  TC_LAUNCHED(1);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

tc_status launch_trace_to_rows(const uint64_t* trace, uint64_t n, uint32_t* rows, float* labels, cudaStream_t st,
                               bool clip) {
  if (!n) return TC_OK;
  k_trace_to_rows<<<grid_cap(n, 256), 256, 0, st>>>(trace, n, rows, labels, clip);
  TC_LAUNCHED(1);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

// Scratch of launch_proposal_scan: q, the tile sums of q and their scan levels.
size_t proposal_scan_scratch_bytes(uint64_t m) {
  const uint64_t T = (m + kPTile - 1) / kPTile ? (m + kPTile - 1) / kPTile : 1;
  return scan_align256(8 * (m ? m : 1)) + scan_align256(8 * T) + scan_align256(8 * (scan_u64_scratch_words(T) + 1));
}

tc_status launch_proposal_scan(const tc_mlp* M, const uint16_t* feat, const uint64_t* prefix, uint64_t m, float eps,
                               float scale, uint16_t* h, uint64_t* qprefix, uint32_t* hrange, void* scratch,
                               uint32_t* d_err, cudaStream_t st) {
  TC_CUDA(cudaMemsetAsync(hrange, 0xFF, sizeof(uint32_t), st));  // smallest h: none yet
  TC_CUDA(cudaMemsetAsync(hrange + 1, 0, sizeof(uint32_t), st));  // largest h: none yet
  if (!m) {
    TC_CUDA(cudaMemsetAsync(qprefix, 0, sizeof(uint64_t), st));
    return TC_OK;
  }
  if (scan_tile_size() != (uint64_t)kPTile) return set_error(TC_ERR_INVALID_ARG, "scan tile mismatch");
  const uint64_t T = (m + kPTile - 1) / kPTile;
  char* p = (char*)scratch;
  uint64_t* q = (uint64_t*)p;
  uint64_t* sums = (uint64_t*)(p + scan_align256(8 * m));
  uint64_t* scan_scratch = (uint64_t*)(p + scan_align256(8 * m) + scan_align256(8 * T));
  if (use_tcgen05()) {
    TC_TRY(launch_umma<true>(M, feat, nullptr, m, nullptr, prefix, eps, scale, h, q, sums, hrange, d_err, st));
    return scan_u64_from_tile_sums(q, qprefix, m, sums, d_err, scan_scratch, scan_u64_scratch_words(T) + 1, st);
  }
  static int bps = 0;
  if (!bps) {
    TC_CUDA(cudaFuncSetAttribute(k_proposal, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPDynSmem));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_proposal, kPThreads, kPDynSmem);
    if (bps <= 0) bps = 1;
  }
  uint64_t blocks = (uint64_t)num_sms() * bps;
  if (blocks > T) blocks = T;
  k_proposal<<<(unsigned)blocks, kPThreads, kPDynSmem, st>>>(M->params, reinterpret_cast<const __nv_bfloat16*>(feat),
                                                             prefix, m, eps, scale, h, q, sums, hrange, d_err);
  TC_LAUNCHED(1);
  TC_CUDA(cudaGetLastError());
  return scan_u64_from_tile_sums(q, qprefix, m, sums, d_err, scan_scratch, scan_u64_scratch_words(T) + 1, st);
}

}  // namespace tc
