// tc_prefix_sum_noalloc: the exact uint64 prefix sum without any device
// allocation, for callers that cannot allocate device memory (see tc.h).
// Its scratch (the scan's per-tile sums and an error word) is one file-scope
// device array that every device loading this library holds until exit.
#include <cuda_runtime.h>

#include <mutex>

#include "tc_internal.cuh"

namespace {

constexpr uint64_t kMaxEdges = TC_NOALLOC_MAX_EDGES;
constexpr uint64_t kErrWords = 32;  // first 256 bytes: the device error word
// tile sums of all scan levels for kMaxEdges elements (2048 per tile):
// 2^28 / 2048 = 131072 at the first level, 64 at the second
constexpr uint64_t kSumWords = 131072 + 64;
constexpr uint64_t kScratchWords = kErrWords + kSumWords;

}  // namespace

static __device__ __align__(256) unsigned long long g_noalloc_scratch[kScratchWords];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned long long* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  The name
// g_noalloc_scratch in host code is only a host-side stand-in, so the
// address is looked up once per device with that device current.
tc_status scratch_on_current_device(unsigned long long** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return tc::cuda_status(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return tc::set_error(TC_ERR_INVALID_ARG, "device index beyond 63");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return tc::cuda_status(e, "cudaGetSymbolAddress");
    g_scratch_addr[dev] = (unsigned long long*)p;
  }
  *out = g_scratch_addr[dev];
  return TC_OK;
}

}  // namespace

extern "C" tc_status tc_prefix_sum_noalloc(const uint64_t* d_w, uint64_t m, uint64_t* d_prefix, uint64_t* h_W,
                                           void* stream) {
  if (!d_prefix || (m > 0 && !d_w)) return tc::set_error(TC_ERR_INVALID_ARG, "w or prefix is NULL");
  if (m > kMaxEdges)
    return tc::set_error(TC_ERR_INVALID_ARG, "m exceeds TC_NOALLOC_MAX_EDGES (2^28); use tc_path_weights");
  static_assert(kSumWords >= 131072 + 64, "scratch sized for 2^28 elements");
  if (tc::scan_u64_scratch_words(m) > kSumWords) return tc::set_error(TC_ERR_INVALID_ARG, "scratch too small");
  unsigned long long* base = nullptr;
  TC_TRY(scratch_on_current_device(&base));
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t* d_err = (uint32_t*)base;
  uint64_t* sums = (uint64_t*)(base + kErrWords);
  TC_CUDA(cudaMemsetAsync(d_err, 0, sizeof(uint32_t), st));  // the array keeps the last call's contents
  TC_TRY(tc::scan_u64_in_scratch(d_w, d_prefix, m, true, d_err, sums, kSumWords, st));
  if (h_W) {
    uint32_t h_err = 0;
    TC_CUDA(cudaMemcpyAsync(h_W, d_prefix + m, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaMemcpyAsync(&h_err, d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaStreamSynchronize(st));
    if (h_err) return tc::device_status(h_err, "tc_prefix_sum_noalloc");
  }
  return TC_OK;
}
