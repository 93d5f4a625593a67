// C ABI of libndgi.so (declared in include/ndgi.h): argument validation,
// error reporting, precision/shape dispatch, and the page-decode plan.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "ndgi_internal.h"
#include "tc_decode.h"

namespace ndgi {

static thread_local std::string g_msg;
static thread_local ndgi_status g_status = NDGI_OK;

ndgi_status set_error(ndgi_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_msg = buf;
  g_status = s;
  return s;
}

ndgi_status cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return NDGI_OK;
  if (e == cudaErrorMemoryAllocation) return set_error(NDGI_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  return set_error(NDGI_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int num_sms() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  if (cache[dev] == 0) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cache[dev] = n > 0 ? n : 1;
  }
  return cache[dev];
}

static bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

// Host-side checks of a model descriptor common to every decode.
ndgi_status check_model(const ndgi_model_desc* m, const char* who) {
  if (!m) return set_error(NDGI_ERR_INVALID_ARG, "%s: model is NULL", who);
  if (m->lm_w <= 0 || m->lm_h <= 0) return set_error(NDGI_ERR_INVALID_ARG, "%s: lightmap size must be > 0", who);
  if (m->feat_w <= 0 || m->feat_h <= 0 || m->feat_w % 4 || m->feat_h % 4)
    return set_error(NDGI_ERR_INVALID_ARG, "%s: feature size %dx%d must be positive multiples of 4", who,
                     m->feat_w, m->feat_h);
  if ((int64_t)m->feat_w * m->feat_h > (int64_t)1 << 30)
    return set_error(NDGI_ERR_INVALID_ARG, "%s: feature plane larger than 2^30 texels", who);
  if (m->cs <= 0 || m->ct < 0 || m->t_count <= 0 || m->hidden <= 0)
    return set_error(NDGI_ERR_INVALID_ARG, "%s: cs, t_count, hidden must be > 0 and ct >= 0", who);
  if (!m->bc4 || !m->w1 || !m->b1 || !m->w2 || !m->b2 || !m->w3 || !m->b3 || (m->ct > 0 && !m->temporal))
    return set_error(NDGI_ERR_INVALID_ARG, "%s: a model pointer is NULL", who);
  if (!aligned(m->bc4, 16)) return set_error(NDGI_ERR_INVALID_ARG, "%s: bc4 must be 16-byte aligned", who);
  if (m->temporal_dtype != NDGI_FP32 && m->temporal_dtype != NDGI_FP16)
    return set_error(NDGI_ERR_INVALID_ARG, "%s: temporal_dtype must be NDGI_FP32 or NDGI_FP16", who);
  if (m->address_mode != 0 && m->address_mode != 1)
    return set_error(NDGI_ERR_INVALID_ARG, "%s: address_mode must be 0 or 1", who);
  if (!simt_supported(m->cs, m->ct, m->hidden))
    return set_error(NDGI_ERR_UNSUPPORTED, "%s: shape cs=%d ct=%d hidden=%d is not built", who, m->cs, m->ct,
                     m->hidden);
  return NDGI_OK;
}

}  // namespace ndgi

using namespace ndgi;

extern "C" {

const char* ndgi_version(void) { return "ndgi-gb300 0.1 (sm_103a)"; }

ndgi_status ndgi_last_error(char* buf, size_t buf_len) {
  if (buf && buf_len) {
    strncpy(buf, g_msg.c_str(), buf_len - 1);
    buf[buf_len - 1] = 0;
  }
  return g_status;
}

ndgi_status ndgi_check(void* stream) {
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e, "ndgi_check");
  return NDGI_OK;
}

// Writes one int of device memory on the stream (no host memory is read after the launch returns).
__global__ void k_set_word(int* p, int v) { *p = v; }

ndgi_status ndgi_workspace_check(const ndgi_model_desc* model, ndgi_precision precision, const void* ws,
                                 int32_t* device_error, void* stream) {
  ndgi_status st = check_model(model, "ndgi_workspace_check");
  if (st != NDGI_OK) return st;
  if ((precision != NDGI_FP16 && precision != NDGI_BF16) || !tc_supported(model->cs, model->ct, model->hidden))
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_workspace_check: needs an FP16/BF16 workspace of a built shape");
  if (!ws || !aligned(ws, 256)) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_workspace_check: ws missing or unaligned");
  int* w = reinterpret_cast<int*>(static_cast<unsigned char*>(const_cast<void*>(ws)) +
                                  tc_error_offset(model->cs, model->ct, model->hidden));
  cudaStream_t s = (cudaStream_t)stream;
  int32_t err = 0;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemcpy(&err, w, sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && err) {
    k_set_word<<<1, 1, 0, s>>>(w, 0);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (e != cudaSuccess) return cuda_status(e, "ndgi_workspace_check");
  if (device_error) *device_error = err;
  if (err & kErrTimeout)
    return set_error(NDGI_ERR_TIMEOUT, "ndgi_workspace_check: a tensor-core barrier wait timed out (0x%x)", err);
  return NDGI_OK;
}

ndgi_status ndgi_debug_workspace_inject(const ndgi_model_desc* model, ndgi_precision precision, void* ws,
                                        int32_t flags, void* stream) {
  ndgi_status st = check_model(model, "ndgi_debug_workspace_inject");
  if (st != NDGI_OK) return st;
  if ((precision != NDGI_FP16 && precision != NDGI_BF16) || !tc_supported(model->cs, model->ct, model->hidden))
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_debug_workspace_inject: needs an FP16/BF16 workspace");
  if (!ws || !aligned(ws, 256) || (flags & ~kDbgInjectTimeout))
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_debug_workspace_inject: bad workspace or flags");
  int* w = reinterpret_cast<int*>(static_cast<unsigned char*>(ws) + tc_error_offset(model->cs, model->ct,
                                                                                     model->hidden)) + 1;
  k_set_word<<<1, 1, 0, (cudaStream_t)stream>>>(w, flags);
  return cuda_status(cudaGetLastError(), "ndgi_debug_workspace_inject");
}

size_t ndgi_prepare_workspace_size(const ndgi_model_desc* model, ndgi_precision precision) {
  if (!model) return 0;
  if (precision == NDGI_FP16 || precision == NDGI_BF16)
    return tc_workspace_bytes(model->cs, model->ct, model->hidden, model->feat_w, model->feat_h);
  if (precision == NDGI_FP8_E4M3)
    return tc_fp8_workspace_bytes(model->cs, model->ct, model->hidden, model->feat_w, model->feat_h);
  return 0;
}

ndgi_status ndgi_calibrate_fp8(const ndgi_model_desc* model, const float* uvt, int64_t n, float* act_max,
                               void* stream) {
  ndgi_status st = check_model(model, "ndgi_calibrate_fp8");
  if (st != NDGI_OK) return st;
  if (n <= 0 || !uvt || !act_max || !aligned(uvt, 4) || !aligned(act_max, 4))
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_calibrate_fp8: need n > 0 queries and a 3-float act_max");
  if (!simt_supported(model->cs, model->ct, model->hidden))
    return set_error(NDGI_ERR_UNSUPPORTED, "ndgi_calibrate_fp8: shape cs=%d ct=%d hidden=%d not built", model->cs,
                     model->ct, model->hidden);
  return cuda_status(launch_fp8_calibrate(to_dev(*model), uvt, n, act_max, (cudaStream_t)stream),
                     "ndgi_calibrate_fp8");
}

ndgi_status ndgi_prepare_fp8(const ndgi_model_desc* model, const float act_max[3], void* ws, size_t ws_bytes,
                             void* stream) {
  ndgi_status st = check_model(model, "ndgi_prepare_fp8");
  if (st != NDGI_OK) return st;
  if (!act_max) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_prepare_fp8: act_max is NULL");
  for (int i = 0; i < 3; ++i)
    if (!(act_max[i] >= 0.0f && act_max[i] <= 3.0e38f))
      return set_error(NDGI_ERR_INVALID_ARG, "ndgi_prepare_fp8: act_max[%d] must be finite and >= 0", i);
  if (!tc_fp8_pages_supported(model->cs, model->ct, model->hidden))
    return set_error(NDGI_ERR_UNSUPPORTED, "ndgi_prepare_fp8: FP8 shape cs=%d ct=%d hidden=%d not built (cs = 16, "
                     "hidden a multiple of 32)", model->cs, model->ct, model->hidden);
  const size_t need = tc_fp8_workspace_bytes(model->cs, model->ct, model->hidden, model->feat_w, model->feat_h);
  if (!ws || ws_bytes < need || !aligned(ws, 256))
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_prepare_fp8: ws must be 256-byte aligned with >= %zu bytes", need);
  cudaStream_t s = (cudaStream_t)stream;
  st = cuda_status(launch_tc_prepare8(to_dev(*model), act_max, ws, s), "ndgi_prepare_fp8");
  if (st != NDGI_OK) return st;
  uint32_t status = 0;
  const unsigned char* sp = static_cast<const unsigned char*>(ws) + tc_fp8_status_offset(model->cs, model->ct,
                                                                                         model->hidden);
  cudaError_t e = cudaMemcpyAsync(&status, sp, sizeof status, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e, "ndgi_prepare_fp8: status read");
  if (status & 1u)
    return set_error(NDGI_ERR_UNSUPPORTED, "ndgi_prepare_fp8: a bias is too large for its layer's output unit");
  if (status & 2u)
    return set_error(NDGI_ERR_UNSUPPORTED, "ndgi_prepare_fp8: act_max[0] too small (1/a1 above 2^14)");
  return NDGI_OK;
}

ndgi_status ndgi_fp8_unpack(const ndgi_model_desc* model, const void* ws, float* out, size_t out_len,
                            size_t* needed) {
  if (!model || !ws) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_fp8_unpack: NULL argument");
  const size_t bytes = tc_fp8_workspace_bytes(model->cs, model->ct, model->hidden, 0, 0);   // the image, not the slice
  if (!bytes) return set_error(NDGI_ERR_UNSUPPORTED, "ndgi_fp8_unpack: no FP8 image for this shape");
  const size_t n = tc_fp8_unpack(model->cs, model->ct, model->hidden, nullptr, nullptr, 0);
  if (needed) *needed = n;
  if (!out) return NDGI_OK;
  if (out_len < n) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_fp8_unpack: out needs %zu floats", n);
  std::vector<unsigned char> img(bytes);
  cudaError_t e = cudaMemcpy(img.data(), ws, bytes, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e, "ndgi_fp8_unpack: copy");
  tc_fp8_unpack(model->cs, model->ct, model->hidden, img.data(), out, out_len);
  return NDGI_OK;
}

ndgi_status ndgi_prepare(const ndgi_model_desc* model, ndgi_precision precision, void* ws, size_t ws_bytes,
                         void* stream) {
  ndgi_status st = check_model(model, "ndgi_prepare");
  if (st != NDGI_OK) return st;
  if (precision == NDGI_FP32) return NDGI_OK;
  if (precision == NDGI_FP8_E4M3)
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_prepare: FP8 needs calibration maxima; use ndgi_prepare_fp8");
  if (precision != NDGI_FP16 && precision != NDGI_BF16)
    return set_error(NDGI_ERR_UNSUPPORTED, "ndgi_prepare: precision %d not supported", (int)precision);
  if (!tc_supported(model->cs, model->ct, model->hidden))
    return set_error(NDGI_ERR_UNSUPPORTED, "ndgi_prepare: tensor-core shape cs=%d ct=%d hidden=%d not built",
                     model->cs, model->ct, model->hidden);
  const size_t need = tc_workspace_bytes(model->cs, model->ct, model->hidden, model->feat_w, model->feat_h);
  if (!ws || ws_bytes < need || !aligned(ws, 256))
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_prepare: ws must be 256-byte aligned with >= %zu bytes", need);
  return cuda_status(launch_tc_prepare(to_dev(*model), precision == NDGI_BF16, ws, (cudaStream_t)stream),
                     "ndgi_prepare");
}

}  // extern "C"

namespace ndgi {

// The point decode with an explicit gather policy (kPointsAuto for the ABI
// call; the host-buffer pipe builds the decoded-texel cache once per call).
ndgi_status decode_points_mode(const ndgi_model_desc* model, ndgi_precision precision, const void* ws,
                               const float* uvt, int64_t n, float* rgb, void* stream, int mode) {
  ndgi_status st = check_model(model, "ndgi_decode_points");
  if (st != NDGI_OK) return st;
  if (n < 0) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_decode_points: n < 0");
  if (n == 0) return NDGI_OK;
  if (!uvt || !rgb) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_decode_points: uvt or rgb is NULL");
  if (!aligned(uvt, 4) || !aligned(rgb, 4))
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_decode_points: uvt and rgb must be 4-byte aligned");
  const DevModel m = to_dev(*model);
  if (precision == NDGI_FP32)
    return cuda_status(launch_points_f32(m, uvt, n, rgb, (cudaStream_t)stream), "ndgi_decode_points");
  if (precision == NDGI_FP16 || precision == NDGI_BF16) {
    if (!tc_supported(model->cs, model->ct, model->hidden))
      return set_error(NDGI_ERR_UNSUPPORTED, "ndgi_decode_points: tensor-core shape cs=%d ct=%d hidden=%d not built",
                       model->cs, model->ct, model->hidden);
    if (!ws || !aligned(ws, 256))
      return set_error(NDGI_ERR_INVALID_ARG, "ndgi_decode_points: ws (from ndgi_prepare) missing or unaligned");
    return cuda_status(launch_tc_points(m, precision == NDGI_BF16, ws, uvt, n, rgb, (cudaStream_t)stream, mode),
                       "ndgi_decode_points");
  }
  if (precision == NDGI_FP8_E4M3)
    return set_error(NDGI_ERR_UNSUPPORTED, "ndgi_decode_points: FP8 is built for the page decode only");
  return set_error(NDGI_ERR_UNSUPPORTED, "ndgi_decode_points: precision %d not supported", (int)precision);
}

}  // namespace ndgi

extern "C" {

ndgi_status ndgi_decode_points(const ndgi_model_desc* model, ndgi_precision precision, const void* ws,
                               const float* uvt, int64_t n, float* rgb, void* stream) {
  return decode_points_mode(model, precision, ws, uvt, n, rgb, stream, kPointsAuto);
}

int32_t ndgi_decode_points_path(const ndgi_model_desc* model, ndgi_precision precision, int64_t n) {
  if (!model || (precision != NDGI_FP16 && precision != NDGI_BF16)) return 0;
  if (!tc_supported(model->cs, model->ct, model->hidden)) return 0;
  if (!tc_points_cache_path(to_dev(*model), n, kPointsAuto)) return 0;
  return tc_points_ws_built(model->cs, model->ct, model->hidden) ? 2 : 1;
}

ndgi_status ndgi_debug_features_cache(const ndgi_model_desc* model, const void* ws, const float* uvt, int64_t n,
                                      float* x, void* stream) {
  ndgi_status st = check_model(model, "ndgi_debug_features_cache");
  if (st != NDGI_OK) return st;
  if (n < 0) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_debug_features_cache: n < 0");
  if (n == 0) return NDGI_OK;
  if (!uvt || !x || !ws || !aligned(ws, 256))
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_debug_features_cache: NULL argument or unaligned workspace");
  if (!tc_supported(model->cs, model->ct, model->hidden))
    return set_error(NDGI_ERR_UNSUPPORTED, "ndgi_debug_features_cache: tensor-core shape not built");
  const DevModel m = to_dev(*model);
  if (!tc_points_cache_path(m, n, kPointsBuild))
    return set_error(NDGI_ERR_UNSUPPORTED, "ndgi_debug_features_cache: the map's cache exceeds 64 MiB");
  return cuda_status(launch_debug_features_cache(m, ws, uvt, n, x, (cudaStream_t)stream),
                     "ndgi_debug_features_cache");
}

ndgi_status ndgi_debug_features(const ndgi_model_desc* model, const float* uvt, int64_t n, float* x, int32_t* p35,
                                void* stream) {
  ndgi_status st = check_model(model, "ndgi_debug_features");
  if (st != NDGI_OK) return st;
  if (n < 0) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_debug_features: n < 0");
  if (n == 0) return NDGI_OK;
  if (!uvt || !x) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_debug_features: uvt or x is NULL");
  return cuda_status(launch_debug_features(to_dev(*model), uvt, n, x, p35, (cudaStream_t)stream),
                     "ndgi_debug_features");
}

ndgi_status ndgi_debug_features_tc(const ndgi_model_desc* model, const void* ws, const float* uvt, int64_t n,
                                   float* x, void* stream) {
  ndgi_status st = check_model(model, "ndgi_debug_features_tc");
  if (st != NDGI_OK) return st;
  if (n < 0) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_debug_features_tc: n < 0");
  if (n == 0) return NDGI_OK;
  if (!uvt || !x || !ws || !aligned(ws, 256))
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_debug_features_tc: NULL argument or unaligned workspace");
  if (!tc_supported(model->cs, model->ct, model->hidden))
    return set_error(NDGI_ERR_UNSUPPORTED, "ndgi_debug_features_tc: tensor-core shape not built");
  return cuda_status(launch_debug_features_tc(to_dev(*model), ws, uvt, n, x, (cudaStream_t)stream),
                     "ndgi_debug_features_tc");
}

ndgi_status ndgi_bc_pack(const float* ea, const float* eb, const float* w, int32_t cs, int32_t feat_w,
                         int32_t feat_h, uint8_t* bc4_out, void* stream) {
  if (!ea || !eb || !w || !bc4_out) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_bc_pack: NULL pointer");
  if (cs <= 0 || feat_w <= 0 || feat_h <= 0 || feat_w % 4 || feat_h % 4)
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_bc_pack: cs > 0 and positive multiple-of-4 sizes required");
  if (!aligned(bc4_out, 8) || !aligned(w, 16))
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_bc_pack: bc4_out must be 8-byte and w 16-byte aligned");
  return cuda_status(launch_bc_pack(ea, eb, w, cs, feat_w, feat_h, bc4_out, (cudaStream_t)stream), "ndgi_bc_pack");
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Page-decode plan
// ---------------------------------------------------------------------------
struct ndgi_pages_plan {
  int device = 0;
  ndgi_precision precision = NDGI_FP32;
  int n_models = 0, max_reqs = 0, out_format = 0;
  int cs = 0, ct = 0, hidden = 0;
  bool staged = false;   // every model's features at most half its lightmap resolution
  void* phys = nullptr;
  int64_t phys_w = 0, phys_h = 0;
  void* dblock = nullptr;
  PagesCtx ctx{};
  TcPagesShape shape{};
  int simt_grid = 0;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t exec = nullptr;
  const void* g_reqs = nullptr;
  const void* g_n = nullptr;
  TcPagesShape g_shape{};
  int g_simt_grid = -1;
};

namespace ndgi {

static cudaError_t enqueue_pages(ndgi_pages_plan* p, const ndgi_page_req* reqs, const int32_t* n_dev,
                                 cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(p->ctx.work_counter, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  if (p->precision == NDGI_FP32)
    return launch_pages_f32(p->ctx, p->cs, p->ct, p->hidden, reqs, n_dev, p->simt_grid, s);
  const int prec = p->precision == NDGI_BF16 ? 1 : (p->precision == NDGI_FP8_E4M3 ? 2 : 0);
  return launch_tc_pages(p->ctx, prec, p->cs, p->ct, p->hidden, p->shape, p->staged, reqs, n_dev, s);
}

static ndgi_status ensure_graph(ndgi_pages_plan* p, const ndgi_page_req* reqs, const int32_t* n_dev) {
  if (p->exec && p->g_reqs == reqs && p->g_n == n_dev && p->g_simt_grid == p->simt_grid &&
      memcmp(&p->g_shape, &p->shape, sizeof(TcPagesShape)) == 0)
    return NDGI_OK;
  if (p->exec) {
    cudaGraphExecDestroy(p->exec);
    p->exec = nullptr;
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_status(e, "ndgi_decode_pages: begin capture");
  cudaError_t le = enqueue_pages(p, reqs, n_dev, p->cap_stream);
  e = cudaStreamEndCapture(p->cap_stream, &g);
  if (le != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_status(le, "ndgi_decode_pages: launch during capture");
  }
  if (e != cudaSuccess) return cuda_status(e, "ndgi_decode_pages: end capture");
  e = cudaGraphInstantiate(&p->exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_status(e, "ndgi_decode_pages: instantiate");
  p->g_reqs = reqs;
  p->g_n = n_dev;
  p->g_shape = p->shape;
  p->g_simt_grid = p->simt_grid;
  return NDGI_OK;
}

}  // namespace ndgi

extern "C" {

ndgi_status ndgi_pages_plan_create(const ndgi_model_desc* models, const void* const* ws, int32_t n_models,
                                   ndgi_precision precision, int32_t max_reqs, int32_t out_format, void* phys,
                                   int64_t phys_w, int64_t phys_h, ndgi_pages_plan** plan) {
  if (!plan) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_pages_plan_create: plan is NULL");
  *plan = nullptr;
  if (!models || n_models <= 0) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_pages_plan_create: no models");
  if (max_reqs <= 0 || max_reqs > (1 << 24))
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_pages_plan_create: max_reqs must be in 1..2^24");
  if (out_format != NDGI_RGBA32F && out_format != NDGI_RGBA16F)
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_pages_plan_create: bad out_format");
  if (!phys || phys_w <= 0 || phys_h <= 0 || !aligned(phys, 16))
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_pages_plan_create: phys must be a 16-byte aligned texture");
  if (precision != NDGI_FP32 && precision != NDGI_FP16 && precision != NDGI_BF16 && precision != NDGI_FP8_E4M3)
    return set_error(NDGI_ERR_UNSUPPORTED, "ndgi_pages_plan_create: precision %d not supported", (int)precision);
  if (precision == NDGI_FP8_E4M3 && !tc_fp8_pages_supported(models[0].cs, models[0].ct, models[0].hidden))
    return set_error(NDGI_ERR_UNSUPPORTED, "ndgi_pages_plan_create: FP8 needs cs = 16 and hidden a multiple of 32");
  for (int i = 0; i < n_models; ++i) {
    ndgi_status st = check_model(&models[i], "ndgi_pages_plan_create");
    if (st != NDGI_OK) return st;
    if (models[i].cs != models[0].cs || models[i].ct != models[0].ct || models[i].hidden != models[0].hidden)
      return set_error(NDGI_ERR_UNSUPPORTED, "ndgi_pages_plan_create: all models must share cs, ct and hidden");
    if (precision != NDGI_FP32) {
      if (!ws || !ws[i] || !aligned(ws[i], 256))
        return set_error(NDGI_ERR_INVALID_ARG, "ndgi_pages_plan_create: model %d has no prepared workspace", i);
    }
  }
  if (precision != NDGI_FP32 && !tc_pages_supported(models[0].cs, models[0].ct, models[0].hidden))
    return set_error(NDGI_ERR_UNSUPPORTED, "ndgi_pages_plan_create: tensor-core page shape not built (cs must be 16)");

  ndgi_pages_plan* p = new (std::nothrow) ndgi_pages_plan();
  if (!p) return set_error(NDGI_ERR_OOM, "ndgi_pages_plan_create: host allocation failed");
  cudaGetDevice(&p->device);
  p->precision = precision;
  p->n_models = n_models;
  p->max_reqs = max_reqs;
  p->out_format = out_format;
  p->cs = models[0].cs;
  p->ct = models[0].ct;
  p->hidden = models[0].hidden;
  p->phys = phys;
  p->phys_w = phys_w;
  p->phys_h = phys_h;
  p->staged = true;
  for (int i = 0; i < n_models; ++i)
    p->staged = p->staged && 2 * models[i].feat_w <= models[i].lm_w && 2 * models[i].feat_h <= models[i].lm_h;
  const size_t models_bytes = sizeof(DevModel) * n_models;
  const size_t ws_off = (models_bytes + 255) / 256 * 256;
  const size_t ctr_off = ws_off + (sizeof(void*) * n_models + 255) / 256 * 256;
  const size_t total = ctr_off + 256;   // work counter at +0, error word at +64, debug word at +128
  cudaError_t e = cudaMalloc(&p->dblock, total);
  if (e != cudaSuccess) {
    delete p;
    return cuda_status(e, "ndgi_pages_plan_create: device block");
  }
  std::vector<unsigned char> host(total, 0);
  for (int i = 0; i < n_models; ++i) {
    DevModel dm = to_dev(models[i]);
    memcpy(host.data() + i * sizeof(DevModel), &dm, sizeof(DevModel));
    const void* w = ws ? ws[i] : nullptr;
    memcpy(host.data() + ws_off + i * sizeof(void*), &w, sizeof(void*));
  }
  e = cudaMemcpy(p->dblock, host.data(), total, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cudaFree(p->dblock);
    delete p;
    return cuda_status(e, "ndgi_pages_plan_create: upload");
  }
  unsigned char* base = static_cast<unsigned char*>(p->dblock);
  p->ctx.models = reinterpret_cast<const DevModel*>(base);
  p->ctx.ws = reinterpret_cast<const void* const*>(base + ws_off);
  p->ctx.n_models = n_models;
  p->ctx.max_reqs = max_reqs;
  p->ctx.out_format = out_format;
  p->ctx.phys = phys;
  p->ctx.phys_w = phys_w;
  p->ctx.phys_h = phys_h;
  p->ctx.work_counter = reinterpret_cast<unsigned int*>(base + ctr_off);
  p->ctx.error_word = reinterpret_cast<int*>(base + ctr_off + 64);
  p->ctx.debug_word = reinterpret_cast<const int*>(base + ctr_off + 128);
  p->simt_grid = num_sms() * 8;
  p->shape = tc_default_pages_shape();
  *plan = p;
  return NDGI_OK;
}

ndgi_status ndgi_decode_pages(ndgi_pages_plan* plan, const ndgi_page_req* reqs_dev, const int32_t* n_dev,
                              void* stream) {
  if (!plan || !reqs_dev || !n_dev) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_decode_pages: NULL argument");
  if (!aligned(reqs_dev, 16) || !aligned(n_dev, 4))
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_decode_pages: reqs must be 16-byte aligned");
  ndgi_status st = ensure_graph(plan, reqs_dev, n_dev);
  if (st != NDGI_OK) return st;
  return cuda_status(cudaGraphLaunch(plan->exec, (cudaStream_t)stream), "ndgi_decode_pages: graph launch");
}

ndgi_status ndgi_pages_autotune(ndgi_pages_plan* plan, const ndgi_page_req* reqs_dev, const int32_t* n_dev,
                                int32_t n_host, void* stream) {
  if (!plan || !reqs_dev || !n_dev || n_host < 0)
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_pages_autotune: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return set_error(NDGI_ERR_CUDA, "ndgi_pages_autotune: event creation failed");
  float best = 1e30f;
  const int sms = num_sms();
  std::vector<int> simt_cands = {sms * 2, sms * 4, sms * 8, sms * 16};
  std::vector<TcPagesShape> tc_cands = tc_pages_candidates(sms);
  const int n_cands = plan->precision == NDGI_FP32 ? (int)simt_cands.size() : (int)tc_cands.size();
  int best_i = 0;
  ndgi_status st = NDGI_OK;
  for (int i = 0; i < n_cands && st == NDGI_OK; ++i) {
    if (plan->precision == NDGI_FP32) plan->simt_grid = simt_cands[i];
    else plan->shape = tc_cands[i];
    st = ensure_graph(plan, reqs_dev, n_dev);
    if (st != NDGI_OK) break;
    float ms_best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
      cudaEventRecord(e0, s);
      cudaGraphLaunch(plan->exec, s);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        st = cuda_status(cudaGetLastError(), "ndgi_pages_autotune: timing run");
        break;
      }
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && ms < ms_best) ms_best = ms;
    }
    if (ms_best < best) {
      best = ms_best;
      best_i = i;
    }
  }
  if (plan->precision == NDGI_FP32) plan->simt_grid = simt_cands[best_i];
  else plan->shape = tc_cands[best_i];
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  (void)n_host;
  return st;
}

ndgi_status ndgi_pages_check(ndgi_pages_plan* plan, int32_t* device_error, void* stream) {
  if (!plan) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_pages_check: plan is NULL");
  int32_t err = 0;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(&err, plan->ctx.error_word, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemsetAsync(plan->ctx.error_word, 0, sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e, "ndgi_pages_check");
  if (device_error) *device_error = err;
  if (err & kErrTimeout)
    return set_error(NDGI_ERR_TIMEOUT, "ndgi_decode_pages: a tensor-core barrier wait timed out (0x%x)", err);
  if (err) return set_error(NDGI_ERR_DEVICE_CHECK, "ndgi_decode_pages: device checks rejected requests (0x%x)", err);
  return NDGI_OK;
}

ndgi_status ndgi_pages_plan_set_debug(ndgi_pages_plan* plan, int32_t flags) {
  if (!plan || (flags & ~kDbgInjectTimeout))
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_pages_plan_set_debug: bad plan or flags");
  const int v = flags;
  return cuda_status(cudaMemcpy(const_cast<int*>(plan->ctx.debug_word), &v, sizeof(int), cudaMemcpyHostToDevice),
                     "ndgi_pages_plan_set_debug");
}

size_t ndgi_pages_fp8_dump_size(const ndgi_pages_plan* plan) {
  if (!plan || plan->precision != NDGI_FP8_E4M3) return 0;
  return sizeof(uint32_t) * ((size_t)kLaneThreadsHost * fp8_dump_row_words(plan->hidden) + plan->ct + plan->hidden);
}

ndgi_status ndgi_pages_plan_set_fp8_dump(ndgi_pages_plan* plan, int32_t item, void* dump) {
  if (!plan || plan->precision != NDGI_FP8_E4M3)
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_pages_plan_set_fp8_dump: needs an FP8 plan");
  if (dump && (item < 0 || !aligned(dump, 16)))
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_pages_plan_set_fp8_dump: bad item or unaligned buffer");
  struct {
    int flags, item;
    void* ptr;
  } w = {dump ? kDbgDumpFp8 : 0, dump ? item : -1, dump};
  static_assert(sizeof(w) == 16, "debug block layout");
  return cuda_status(cudaMemcpy(const_cast<int*>(plan->ctx.debug_word), &w, sizeof(w), cudaMemcpyHostToDevice),
                     "ndgi_pages_plan_set_fp8_dump");
}

ndgi_status ndgi_pages_plan_info(const ndgi_pages_plan* plan, int32_t info[4]) {
  if (!plan || !info) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_pages_plan_info: NULL argument");
  info[0] = plan->precision;
  if (plan->precision == NDGI_FP32) {
    info[1] = plan->simt_grid;
    info[2] = info[3] = 0;
  } else {
    info[1] = plan->shape.ctas_per_sm;
    info[2] = plan->shape.lanes;
    info[3] = plan->shape.slots;
  }
  return NDGI_OK;
}

ndgi_status ndgi_pages_plan_set_shape(ndgi_pages_plan* plan, int32_t ctas_per_sm, int32_t lanes, int32_t slots) {
  if (!plan || plan->precision == NDGI_FP32)
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_pages_plan_set_shape: needs a tensor-core plan");
  if (ctas_per_sm != 1)   // each CTA holds most of its SM's tensor memory for the whole launch
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_pages_plan_set_shape: ctas_per_sm must be 1");
  bool built = false;
  for (const TcPagesShape& c : tc_pages_candidates(num_sms()))
    built = built || (c.lanes == lanes && c.slots == slots);
  if (!built) return set_error(NDGI_ERR_UNSUPPORTED, "ndgi_pages_plan_set_shape: %d lanes x %d slots not built", lanes, slots);
  plan->shape = TcPagesShape{ctas_per_sm, lanes, slots};
  return NDGI_OK;
}

ndgi_status ndgi_pages_plan_destroy(ndgi_pages_plan* plan) {
  if (!plan) return NDGI_OK;
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  if (plan->cap_stream) cudaStreamDestroy(plan->cap_stream);
  cudaError_t e = cudaFree(plan->dblock);
  delete plan;
  return cuda_status(e, "ndgi_pages_plan_destroy");
}

}  // extern "C"
