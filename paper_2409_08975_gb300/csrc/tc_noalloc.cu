// tc_prefix_sum_noalloc: the exact uint64 prefix sum without any device
// allocation, for callers that cannot allocate device memory (see tc.h).
// Its scratch (the scan's per-tile sums and an error word) is one file-scope
// device array that every device loading this library holds until exit.
#include <cuda.h>
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

// The looked-up address per device, valid for the context it was looked up
// in: a device reset destroys that context and unloads the module, so the
// address is looked up again whenever the current context differs.
struct ScratchAddr {
  unsigned long long ctx_id;
  unsigned long long* ptr;
};
ScratchAddr g_scratch_addr[kMaxDevices] = {};

typedef CUresult (*ctx_get_current_fn)(CUcontext*);
typedef CUresult (*ctx_get_id_fn)(CUcontext, unsigned long long*);

// Unique id of the calling thread's current context (driver entry points
// reached through the runtime, so the library does not link libcuda).
tc_status current_context_id(int dev, unsigned long long* id) {
  static ctx_get_current_fn get_current = nullptr;
  static ctx_get_id_fn get_id = nullptr;
  if (!get_current || !get_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
    if (e != cudaSuccess || q1 != cudaDriverEntryPointSuccess || !f1)
      return tc::set_error(TC_ERR_CUDA, "cuCtxGetCurrent entry point unavailable");
    e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
    if (e != cudaSuccess || q2 != cudaDriverEntryPointSuccess || !f2)
      return tc::set_error(TC_ERR_CUDA, "cuCtxGetId entry point unavailable");
    get_current = (ctx_get_current_fn)f1;
    get_id = (ctx_get_id_fn)f2;
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) {
    // no context current yet: make the device's primary context current
    cudaError_t e = cudaSetDevice(dev);
    if (e != cudaSuccess) return tc::cuda_status(e, "cudaSetDevice");
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return tc::set_error(TC_ERR_CUDA, "no current CUDA context");
  }
  if (get_id(ctx, id) != CUDA_SUCCESS) return tc::set_error(TC_ERR_CUDA, "cuCtxGetId failed");
  return TC_OK;
}

// Device address of the scratch array on the current device.  The name
// g_noalloc_scratch in host code is only a host-side stand-in, so the
// address is looked up with that device current: once per device and
// context (again after a device reset).
tc_status scratch_on_current_device(unsigned long long** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return tc::cuda_status(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return tc::set_error(TC_ERR_INVALID_ARG, "device index beyond 63");
  std::lock_guard<std::mutex> lock(g_mu);
  unsigned long long ctx_id = 0;
  TC_TRY(current_context_id(dev, &ctx_id));
  ScratchAddr& a = g_scratch_addr[dev];
  if (!a.ptr || a.ctx_id != ctx_id) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return tc::cuda_status(e, "cudaGetSymbolAddress");
    a.ptr = (unsigned long long*)p;
    a.ctx_id = ctx_id;
  }
  *out = a.ptr;
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
