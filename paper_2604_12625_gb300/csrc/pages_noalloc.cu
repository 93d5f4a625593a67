// Page decode without any allocation: ndgi_decode_pages_static.
//
// Some callers cannot call cudaMalloc at all: code running inside a custom
// memory arena or a frame allocator that must not fragment, real-time
// render loops where an allocation may block on the driver, or hosts that
// forbid the CUDA allocator after start-up.  The plan-based page decode
// allocates a small device block (model table, error word) when the plan is
// created, so those callers cannot use it.  This variant keeps that state in
// a file-scope static device array instead, which every GPU that loads the
// library holds until the process exits.
//
// Limits and sharing: the array holds at most kMaxStaticModels model
// descriptors.  Every call shares it and it keeps the last call's contents;
// each call rewrites the model table and clears the error word on its
// stream before the decode (one small kernel that receives the descriptors
// by value, so no host memory is read after the call returns and the host
// never waits for the stream), so calls that overlap on the GPU (on
// different streams, or on the same stream from different host threads)
// race on it.
//
// Set-up: the device address of the array is looked up with
// cudaGetSymbolAddress once per device, on the first call made while that
// device is current.  That first call should come before any stream capture.
#include <mutex>

#include "ndgi_internal.h"

namespace ndgi {
namespace {

constexpr int kMaxStaticModels = 64;
constexpr int kMaxDevices = 64;
constexpr size_t kModelsBytes = sizeof(DevModel) * kMaxStaticModels;
constexpr size_t kErrorOffset = (kModelsBytes + 255) / 256 * 256;
constexpr size_t kScratchBytes = kErrorOffset + 256;

// Model table [kMaxStaticModels] followed by the error word.
static __device__ __align__(256) unsigned char g_pages_scratch[kScratchBytes];

// The descriptors of one call, passed by value to the set-up kernel.
struct StaticTable {
  DevModel m[kMaxStaticModels];
};
static_assert(sizeof(StaticTable) <= 16 * 1024, "kernel parameter block");

// Writes the model table into the static array and clears the error word.
__global__ void k_static_setup(const StaticTable tbl, int n, unsigned char* base) {
  DevModel* dst = reinterpret_cast<DevModel*>(base);
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = tbl.m[i];
  if (threadIdx.x == 0) *reinterpret_cast<int32_t*>(base + kErrorOffset) = 0;
}

std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

// Device address of g_pages_scratch on the current device (looked up once per device).
ndgi_status scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e, "ndgi_decode_pages_static: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices)
    return set_error(NDGI_ERR_UNSUPPORTED, "ndgi_decode_pages_static: device ordinal %d >= %d", dev, kMaxDevices);
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_pages_scratch);
    if (e != cudaSuccess) return cuda_status(e, "ndgi_decode_pages_static: cudaGetSymbolAddress");
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return NDGI_OK;
}

}  // namespace
}  // namespace ndgi

using namespace ndgi;

extern "C" ndgi_status ndgi_decode_pages_static(const ndgi_model_desc* models, int32_t n_models,
                                                const ndgi_page_req* reqs_dev, const int32_t* n_dev,
                                                int32_t max_reqs, int32_t out_format, void* phys, int64_t phys_w,
                                                int64_t phys_h, int32_t* device_error, void* stream) {
  if (!models || n_models <= 0)
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_decode_pages_static: no models");
  if (n_models > kMaxStaticModels)
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_decode_pages_static: %d models exceed the static maximum of %d",
                     n_models, kMaxStaticModels);
  if (!reqs_dev || !n_dev || ((uintptr_t)reqs_dev % 16) || ((uintptr_t)n_dev % 4))
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_decode_pages_static: reqs (16-byte aligned) and n_dev required");
  if (max_reqs <= 0 || max_reqs > (1 << 24))
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_decode_pages_static: max_reqs must be in 1..2^24");
  if (out_format != NDGI_RGBA32F && out_format != NDGI_RGBA16F)
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_decode_pages_static: bad out_format");
  if (!phys || phys_w <= 0 || phys_h <= 0 || ((uintptr_t)phys % 16))
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_decode_pages_static: phys must be a 16-byte aligned texture");
  StaticTable table;
  for (int i = 0; i < n_models; ++i) {
    const ndgi_model_desc& m = models[i];
    ndgi_status st = check_model(&m, "ndgi_decode_pages_static");
    if (st != NDGI_OK) return st;
    if (m.cs != models[0].cs || m.ct != models[0].ct || m.hidden != models[0].hidden)
      return set_error(NDGI_ERR_UNSUPPORTED, "ndgi_decode_pages_static: all models must share cs, ct and hidden");
    table.m[i] = to_dev(m);
  }
  void* base = nullptr;
  ndgi_status st = scratch_address(&base);
  if (st != NDGI_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* b = static_cast<unsigned char*>(base);
  // The descriptors travel in the kernel's parameter block: nothing on this
  // stack frame is read after the launch returns.
  k_static_setup<<<1, 64, 0, s>>>(table, n_models, b);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e, "ndgi_decode_pages_static: scratch set-up");
  PagesCtx c{};
  c.models = reinterpret_cast<const DevModel*>(b);
  c.ws = nullptr;
  c.n_models = n_models;
  c.max_reqs = max_reqs;
  c.out_format = out_format;
  c.phys = phys;
  c.phys_w = phys_w;
  c.phys_h = phys_h;
  c.work_counter = nullptr;
  c.error_word = reinterpret_cast<int*>(b + kErrorOffset);
  e = launch_pages_f32(c, models[0].cs, models[0].ct, models[0].hidden, reqs_dev, n_dev, num_sms() * 8, s);
  if (e == cudaSuccess && device_error)
    e = cudaMemcpyAsync(device_error, b + kErrorOffset, sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
  return cuda_status(e, "ndgi_decode_pages_static");
}
