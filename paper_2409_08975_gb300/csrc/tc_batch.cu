// Batched queries (tc_batch_*): many (graph, motif, delta, k) queries
// answered by one fixed launch sequence.  Weights, prefix and index are
// built once per distinct (graph, anchor class, window kind, delta) -- the
// weights of Claim 1 depend on nothing else -- every query's samples are put
// in key order, and one persistent launch samples all queries (Alg. 2-5 per
// query).  The sequence allocates nothing, so it can be captured once into
// a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "tc_internal.cuh"

using namespace tc;

namespace {

struct Slot {
  const tc_graph* g;
  Plan plan;
  int64_t delta;
  uint64_t* prefix;  // m + 1
  char* index;       // index_bytes(m), 256-byte aligned
};

struct Query {
  tc_query q;
  Plan plan;
  int slot;
  uint32_t* order;  // key order (chunk after chunk) or NULL
};

constexpr int kBlockSizes[3] = {128, 256, 512};
constexpr uint32_t kTiles[3] = {2048, 8192, 32768};

}  // namespace

struct tc_batch {
  std::vector<Query> queries;
  std::vector<Slot> slots;
  std::vector<void*> allocations;  // every cudaMalloc of the batch
  uint64_t device_bytes = 0;
  void* scan_scratch = nullptr;    // tile states of the weights scan, for the largest graph
  void* sort_scratch = nullptr;
  uint32_t* err = nullptr;         // one error word per slot
  char* records = nullptr;         // nq * kBatchQueryBytes
  uint64_t* tile_begin = nullptr;  // nq + 1
  unsigned long long* next_item = nullptr;
  SampleSums* sums = nullptr;      // nq
  SampleSums* h_sums = nullptr;    // pinned, nq
  uint64_t* h_W = nullptr;         // pinned, one per slot
  uint32_t* h_err = nullptr;       // pinned, one per slot
  int block_size = 256;
  uint32_t tile = 8192;
  unsigned blocks = 0;
  bool use_graph = true;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};  // run start, sampling start, sampling end
  uint64_t launches_per_run = 0;
};

static_assert(offsetof(tc_query, delta) == 64 && sizeof(tc_query) == 96, "tc_query layout");
static_assert(sizeof(tc_batch_options) == 16, "tc_batch_options layout");

namespace {

tc_status batch_alloc(tc_batch* b, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(e == cudaErrorMemoryAllocation ? TC_ERR_OOM : TC_ERR_CUDA, "tc_batch_create: cudaMalloc");
  }
  b->allocations.push_back(*p);
  b->device_bytes += bytes;
  return TC_OK;
}

void batch_free(tc_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (cudaEvent_t e : b->ev)
    if (e) cudaEventDestroy(e);
  for (void* p : b->allocations) cudaFree(p);
  if (b->h_sums) cudaFreeHost(b->h_sums);
  if (b->h_W) cudaFreeHost(b->h_W);
  if (b->h_err) cudaFreeHost(b->h_err);
  delete b;
}

// Item numbering for the current tile size.
tc_status upload_tiles(tc_batch* b) {
  std::vector<uint64_t> tb(b->queries.size() + 1, 0);
  for (size_t q = 0; q < b->queries.size(); q++) tb[q + 1] = tb[q] + (b->queries[q].q.k + b->tile - 1) / b->tile;
  TC_CUDA(cudaMemcpy(b->tile_begin, tb.data(), sizeof(uint64_t) * tb.size(), cudaMemcpyHostToDevice));
  const int bps = sample_batch_blocks_per_sm(b->block_size);
  if (bps == 0) return set_error(TC_ERR_INVALID_ARG, "batch block size must be 128, 256 or 512");
  uint64_t blocks = (uint64_t)num_sms() * bps;
  const uint64_t need = (tb.back() ? tb.back() : 1);
  b->blocks = (unsigned)std::min<uint64_t>(blocks, need);
  return TC_OK;
}

// Everything before the sampling launch: clear the sums, build each slot's
// weights, prefix and index, and put each query's samples in key order.
tc_status enqueue_prologue(tc_batch* b, cudaStream_t st) {
  const size_t nq = b->queries.size(), ns = b->slots.size();
  TC_CUDA(cudaMemsetAsync(b->sums, 0, sizeof(SampleSums) * nq, st));
  TC_CUDA(cudaMemsetAsync(b->err, 0, sizeof(uint32_t) * ns, st));
  for (size_t s = 0; s < ns; s++) {
    const Slot& S = b->slots[s];
    const uint64_t m = (uint64_t)S.g->m;
    EdgeWin* win = (EdgeWin*)(S.index + kIndexHeaderBytes);
    TC_TRY(launch_weights_scan(S.g, S.plan, S.delta, win, S.prefix, nullptr, b->scan_scratch, b->err + s, st));
    TC_TRY(launch_guide(S.g, S.plan, S.delta, S.prefix, S.index, b->err + s, st));
  }
  for (const Query& Q : b->queries) {
    if (!Q.order) continue;
    const Slot& S = b->slots[Q.slot];
    for (uint64_t base = 0; base < Q.q.k; base += kChunkSamples) {
      const uint64_t count = std::min<uint64_t>(Q.q.k - base, kChunkSamples);
      TC_TRY(sort_sample_ids((const IndexHeader*)S.index, Q.q.seed, Q.q.sample_offset + base, count, b->sort_scratch,
                             Q.order + base, st));
    }
  }
  return TC_OK;
}

tc_status enqueue_sampling(tc_batch* b, cudaStream_t st) {
  TC_CUDA(cudaMemsetAsync(b->next_item, 0, sizeof(unsigned long long), st));
  return launch_sample_batch(b->block_size, b->tile, b->blocks, b->records, b->tile_begin,
                             (uint32_t)b->queries.size(), b->next_item, b->sums, st);
}

tc_status enqueue_epilogue(tc_batch* b, cudaStream_t st) {
  const size_t nq = b->queries.size(), ns = b->slots.size();
  TC_CUDA(cudaMemcpyAsync(b->h_sums, b->sums, sizeof(SampleSums) * nq, cudaMemcpyDeviceToHost, st));
  for (size_t s = 0; s < ns; s++) {
    const uint64_t m = (uint64_t)b->slots[s].g->m;
    TC_CUDA(cudaMemcpyAsync(b->h_W + s, b->slots[s].prefix + m, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
  }
  TC_CUDA(cudaMemcpyAsync(b->h_err, b->err, sizeof(uint32_t) * ns, cudaMemcpyDeviceToHost, st));
  return TC_OK;
}

// The events become graph nodes when the sequence is captured (the external
// flag is only valid during a capture).
tc_status enqueue_all(tc_batch* b, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  TC_CUDA(cudaStreamIsCapturing(st, &cs));
  const unsigned flags = cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
  TC_CUDA(cudaEventRecordWithFlags(b->ev[0], st, flags));
  TC_TRY(enqueue_prologue(b, st));
  TC_CUDA(cudaEventRecordWithFlags(b->ev[1], st, flags));
  TC_TRY(enqueue_sampling(b, st));
  TC_CUDA(cudaEventRecordWithFlags(b->ev[2], st, flags));
  return enqueue_epilogue(b, st);
}

// Times the sampling launch for every (block size, tile) candidate on the
// prepared batch and keeps the fastest; the prologue runs once before.
tc_status autotune(tc_batch* b, bool tune_bs, bool tune_tile, cudaStream_t st) {
  TC_TRY(enqueue_prologue(b, st));
  cudaEvent_t e0, e1;
  TC_CUDA(cudaEventCreate(&e0));
  TC_CUDA(cudaEventCreate(&e1));
  tc_status s = TC_OK;
  float best = 0.0f;
  int best_bs = b->block_size;
  uint32_t best_tile = b->tile;
  bool first = true;
  for (int bs : kBlockSizes) {
    if (!tune_bs && bs != b->block_size) continue;
    for (uint32_t tile : kTiles) {
      if (!tune_tile && tile != b->tile) continue;
      b->block_size = bs;
      b->tile = tile;
      s = upload_tiles(b);
      for (int rep = 0; rep < (first ? 2 : 1) && s == TC_OK; rep++) {  // the first candidate warms the caches
        cudaError_t e = cudaMemsetAsync(b->sums, 0, sizeof(SampleSums) * b->queries.size(), st);
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        if (e != cudaSuccess) s = cuda_status(e, "autotune");
        if (s == TC_OK) s = enqueue_sampling(b, st);
        if (s == TC_OK) {
          e = cudaEventRecord(e1, st);
          if (e == cudaSuccess) e = cudaEventSynchronize(e1);
          if (e != cudaSuccess) s = cuda_status(e, "autotune");
        }
      }
      if (s != TC_OK) break;
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (first || ms < best) {
        best = ms;
        best_bs = bs;
        best_tile = tile;
      }
      first = false;
    }
    if (s != TC_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  TC_TRY(s);
  b->block_size = best_bs;
  b->tile = best_tile;
  return upload_tiles(b);
}

tc_status capture(tc_batch* b) {
  TC_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
  const uint64_t before = tc_kernel_launches();
  TC_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  tc_status s = enqueue_all(b, b->cap);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
  b->graph = graph;
  if (s != TC_OK) return s;
  if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture");
  b->launches_per_run = tc_kernel_launches() - before;
  TC_CUDA(cudaGraphInstantiate(&b->exec, graph, 0));
  return TC_OK;
}

tc_status create(const tc_query* hq, int64_t nq, const tc_batch_options* opts, cudaStream_t st, tc_batch* b) {
  // queries and their weight slots
  std::map<std::tuple<uint64_t, int, int, int, int, int, int64_t>, int> slot_of;
  uint64_t max_m = 0, max_sort = 0, order_words = 0;
  for (int64_t i = 0; i < nq; i++) {
    Query Q;
    Q.q = hq[i];
    Q.order = nullptr;
    if (!Q.q.graph) return set_error(TC_ERR_INVALID_ARG, "query graph is NULL");
    TC_TRY(compile_plan_checked(&Q.q.motif, &Q.plan));
    if (Q.q.delta < 0) return set_error(TC_ERR_INVALID_ARG, "delta must be >= 0");
    if (Q.q.k > (1ull << 40)) return set_error(TC_ERR_INVALID_ARG, "batch query k must be at most 2^40");
    const Plan& P = Q.plan;
    auto key = std::make_tuple(Q.q.graph->id, P.alpha1, P.alpha3, P.beta1, P.beta3, P.closed, Q.q.delta);
    auto it = slot_of.find(key);
    if (it == slot_of.end()) {
      Slot S;
      S.g = Q.q.graph;
      S.plan = P;
      S.delta = Q.q.delta;
      S.prefix = nullptr;
      S.index = nullptr;
      it = slot_of.emplace(key, (int)b->slots.size()).first;
      b->slots.push_back(S);
      max_m = std::max<uint64_t>(max_m, (uint64_t)S.g->m);
    }
    Q.slot = it->second;
    if (Q.q.k >= kSortedMinSamples) {
      max_sort = std::max<uint64_t>(max_sort, std::min<uint64_t>(Q.q.k, kChunkSamples));
      order_words += (Q.q.k + 63) & ~63ull;  // 256-byte aligned starts
    }
    b->queries.push_back(Q);
  }
  // device memory
  for (Slot& S : b->slots) {
    const uint64_t m = (uint64_t)S.g->m;
    TC_TRY(batch_alloc(b, (void**)&S.prefix, sizeof(uint64_t) * (m + 1)));
    TC_TRY(batch_alloc(b, (void**)&S.index, index_bytes(m)));
  }
  TC_TRY(batch_alloc(b, (void**)&b->scan_scratch, weights_scan_scratch_bytes(max_m)));
  TC_TRY(batch_alloc(b, (void**)&b->err, sizeof(uint32_t) * b->slots.size()));
  if (max_sort) TC_TRY(batch_alloc(b, &b->sort_scratch, sort_scratch_bytes(max_sort)));
  uint32_t* order = nullptr;
  if (order_words) TC_TRY(batch_alloc(b, (void**)&order, sizeof(uint32_t) * order_words));
  for (Query& Q : b->queries) {
    if (Q.q.k < kSortedMinSamples) continue;
    Q.order = order;
    order += (Q.q.k + 63) & ~63ull;
  }
  TC_TRY(batch_alloc(b, (void**)&b->records, kBatchQueryBytes * (size_t)nq));
  TC_TRY(batch_alloc(b, (void**)&b->tile_begin, sizeof(uint64_t) * (size_t)(nq + 1)));
  TC_TRY(batch_alloc(b, (void**)&b->next_item, sizeof(unsigned long long)));
  TC_TRY(batch_alloc(b, (void**)&b->sums, sizeof(SampleSums) * (size_t)nq));
  TC_CUDA(cudaMallocHost((void**)&b->h_sums, sizeof(SampleSums) * (size_t)(nq ? nq : 1)));
  TC_CUDA(cudaMallocHost((void**)&b->h_W, sizeof(uint64_t) * (b->slots.size() + 1)));
  TC_CUDA(cudaMallocHost((void**)&b->h_err, sizeof(uint32_t) * (b->slots.size() + 1)));
  {  // per-query argument records
    std::vector<char> rec(kBatchQueryBytes * (size_t)nq);
    for (int64_t i = 0; i < nq; i++) {
      const Query& Q = b->queries[i];
      const Slot& S = b->slots[Q.slot];
      batch_query_record(rec.data() + kBatchQueryBytes * i, Q.q.graph, Q.plan, Q.q.delta, S.prefix, S.index, Q.q.k,
                         Q.q.seed, Q.q.sample_offset, Q.order);
    }
    TC_CUDA(cudaMemcpy(b->records, rec.data(), rec.size(), cudaMemcpyHostToDevice));
  }
  for (cudaEvent_t& e : b->ev) TC_CUDA(cudaEventCreate(&e));
  // launch shape
  const int bs = opts ? opts->block_size : 0;
  const uint32_t tile = opts ? opts->tile : 0;
  b->use_graph = opts ? opts->use_graph != 0 : true;
  if (bs && !sample_batch_blocks_per_sm(bs)) return set_error(TC_ERR_INVALID_ARG, "block_size must be 128, 256 or 512");
  if (tile && (tile % (bs ? bs : 512)) != 0) return set_error(TC_ERR_INVALID_ARG, "tile must be a multiple of block_size");
  b->block_size = bs ? bs : 256;
  b->tile = tile ? tile : 8192;
  TC_TRY(upload_tiles(b));
  if (!bs || !tile) TC_TRY(autotune(b, bs == 0, tile == 0, st));
  TC_CUDA(cudaStreamSynchronize(st));
  if (b->use_graph) TC_TRY(capture(b));
  return TC_OK;
}

}  // namespace

extern "C" {

tc_status tc_batch_create(const tc_query* h_queries, int64_t nq, const tc_batch_options* opts, void* stream,
                          tc_batch** out) {
  if (!out) return set_error(TC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nq < 0 || (nq > 0 && !h_queries)) return set_error(TC_ERR_INVALID_ARG, "bad query list");
  if (nq > (1 << 24)) return set_error(TC_ERR_INVALID_ARG, "too many queries");
  tc_batch* b = new tc_batch();
  tc_status s = create(h_queries, nq, opts, (cudaStream_t)stream, b);
  if (s != TC_OK) {
    cudaStreamSynchronize((cudaStream_t)stream);
    batch_free(b);
    return s;
  }
  *out = b;
  return TC_OK;
}

tc_status tc_batch_run(tc_batch* b, tc_estimate* h_out, void* stream) {
  if (!b) return set_error(TC_ERR_INVALID_ARG, "batch is NULL");
  if (!h_out && !b->queries.empty()) return set_error(TC_ERR_INVALID_ARG, "out is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  if (b->queries.empty()) return TC_OK;
  if (b->use_graph) {
    TC_CUDA(cudaGraphLaunch(b->exec, st));
    note_launches((unsigned)b->launches_per_run);
  } else {
    const uint64_t before = tc_kernel_launches();
    TC_TRY(enqueue_all(b, st));
    b->launches_per_run = tc_kernel_launches() - before;
  }
  TC_CUDA(cudaStreamSynchronize(st));
  tc_status status = TC_OK;
  for (size_t i = 0; i < b->queries.size(); i++) {
    const Query& Q = b->queries[i];
    const SampleSums& h = b->h_sums[i];
    tc_estimate& o = h_out[i];
    std::memset(&o, 0, sizeof(o));
    o.W = b->h_W[Q.slot];
    o.k = Q.q.k;
    o.sum_x = h.sum_x;
    o.sum_x2_lo = h.sum_x2_lo;
    o.sum_x2_hi = h.sum_x2_hi;
    o.hits = h.hits;
    o.checked = h.checked;
    const uint32_t bits = h.err | b->h_err[Q.slot];
    if (bits) {
      if (status == TC_OK) status = device_status(bits, "tc_batch_run");
      continue;
    }
    finish_estimate(&o);
  }
  return status;
}

tc_status tc_batch_info(const tc_batch* b, tc_batch_options* h_opts, uint64_t* h_launches_per_run,
                        uint64_t* h_device_bytes, uint64_t* h_weight_slots) {
  if (!b) return set_error(TC_ERR_INVALID_ARG, "batch is NULL");
  if (h_opts) {
    h_opts->block_size = b->block_size;
    h_opts->tile = b->tile;
    h_opts->use_graph = b->use_graph ? 1 : 0;
    h_opts->reserved = 0;
  }
  if (h_launches_per_run) *h_launches_per_run = b->launches_per_run;
  if (h_device_bytes) *h_device_bytes = b->device_bytes;
  if (h_weight_slots) *h_weight_slots = b->slots.size();
  return TC_OK;
}

tc_status tc_batch_timing(const tc_batch* b, float* h_run_ms, float* h_sampling_ms) {
  if (!b) return set_error(TC_ERR_INVALID_ARG, "batch is NULL");
  if (b->queries.empty()) return set_error(TC_ERR_INVALID_ARG, "empty batch has no timing");
  float run = 0.0f, samp = 0.0f;
  TC_CUDA(cudaEventElapsedTime(&run, b->ev[0], b->ev[2]));
  TC_CUDA(cudaEventElapsedTime(&samp, b->ev[1], b->ev[2]));
  if (h_run_ms) *h_run_ms = run;
  if (h_sampling_ms) *h_sampling_ms = samp;
  return TC_OK;
}

tc_status tc_batch_destroy(tc_batch* b) {
  if (!b) return TC_OK;
  batch_free(b);
  return TC_OK;
}

}  // extern "C"
