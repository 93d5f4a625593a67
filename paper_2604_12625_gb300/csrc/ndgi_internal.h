// Internal declarations shared by the CUDA translation units of libndgi.so.
// Not part of the ABI (that is include/ndgi.h).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>

#include "../../include/ndgi.h"

namespace ndgi {

// Launch-time copy of a model descriptor (passed to kernels by value).
struct DevModel {
  int lm_w, lm_h, feat_w, feat_h, cs, bw;
  const uint8_t* bc4;
  int t_count, ct;
  const void* temporal;
  int temporal_f16;
  int hidden;
  const float *w1, *b1, *w2, *b2, *w3, *b3;
  int address_mode;
  float sx, sy;        // feat_w / lm_w, feat_h / lm_h (page texel -> feature coordinate)
  const float* key_t;  // keyframe times [t_count] or null (j / t_count)
};

inline DevModel to_dev(const ndgi_model_desc& d) {
  DevModel m;
  m.lm_w = d.lm_w; m.lm_h = d.lm_h; m.feat_w = d.feat_w; m.feat_h = d.feat_h; m.cs = d.cs;
  m.bw = d.feat_w / 4; m.bc4 = d.bc4; m.t_count = d.t_count; m.ct = d.ct; m.temporal = d.temporal;
  m.temporal_f16 = d.temporal_dtype == NDGI_FP16; m.hidden = d.hidden;
  m.w1 = d.w1; m.b1 = d.b1; m.w2 = d.w2; m.b2 = d.b2; m.w3 = d.w3; m.b3 = d.b3;
  m.address_mode = d.address_mode;
  m.sx = (float)d.feat_w / (float)d.lm_w;
  m.sy = (float)d.feat_h / (float)d.lm_h;
  m.key_t = d.key_t;
  return m;
}

// Error reporting (thread-local message + status).
ndgi_status set_error(ndgi_status s, const char* fmt, ...);
ndgi_status cuda_status(cudaError_t e, const char* what);

int num_sms();

// Host-side checks of a model descriptor common to every decode (NDGI_OK or the status it set).
ndgi_status check_model(const ndgi_model_desc* m, const char* who);

// The point decode with an explicit gather policy (a kPoints* value of tc_decode.h).
ndgi_status decode_points_mode(const ndgi_model_desc* model, ndgi_precision precision, const void* ws,
                               const float* uvt, int64_t n, float* rgb, void* stream, int mode);

// ---- FP32 CUDA-core decode (decode_simt.cu) ----
bool simt_supported(int cs, int ct, int hidden);
cudaError_t launch_points_f32(const DevModel& m, const float* uvt, int64_t n, float* rgb, cudaStream_t s);
cudaError_t launch_fp8_calibrate(const DevModel& m, const float* uvt, int64_t n, float* act_max, cudaStream_t s);
cudaError_t launch_debug_features(const DevModel& m, const float* uvt, int64_t n, float* x, int32_t* p35,
                                  cudaStream_t s);

// Device-side page-decode context (shared by the SIMT and tensor-core page kernels).
struct PagesCtx {
  const DevModel* models;       // device array [n_models]
  const void* const* ws;        // device array of prepared workspaces
  int n_models;
  int max_reqs;
  int out_format;
  void* phys;
  int64_t phys_w, phys_h;
  unsigned int* work_counter;   // device
  int* error_word;              // device: bits 0-3 rejected requests, kErrTimeout a timed-out wait
  const int* debug_word;        // device or NULL: bit 0 makes the tensor-core kernels' first wait run out
};

// Error-word bit latched by a tensor-core kernel whose bounded wait ran out
// (pages: in the plan's error word; points: in the prepared workspace's word).
constexpr int kErrTimeout = 16;
// Debug-word bit: each lane's first wait uses a short limit on a barrier that
// nothing arrives at, before any MMA is issued or tensor memory is touched by
// an MMA, so the kernel takes its timeout path (test of that path).
constexpr int kDbgInjectTimeout = 1;
// Debug-word bit: the FP8 4x1 page kernel copies the operands and accumulators
// of one tile (request debug_word[1], its first 2 x 64 texels) to the device
// buffer whose address is stored at debug_word + 2 (layout: ndgi_pages_plan_set_fp8_dump).
constexpr int kDbgDumpFp8 = 2;
// Words per texel row of that dump: A1 (8), D1 (H), A2 ((H+32)/4), D2 (H), A3 ((H+32)/4), D3 (4).
constexpr int fp8_dump_row_words(int H) { return 8 + 2 * H + 2 * ((H + 32) / 4) + 4; }
constexpr int kLaneThreadsHost = 128;   // texel rows of one tile (the dump's row count)
cudaError_t launch_pages_f32(const PagesCtx& c, int cs, int ct, int hidden, const ndgi_page_req* reqs,
                             const int32_t* n_dev, int grid, cudaStream_t s);

// ---- BC pack (pack.cu) ----
cudaError_t launch_bc_pack(const float* ea, const float* eb, const float* w, int cs, int feat_w, int feat_h,
                           uint8_t* out, cudaStream_t s);

}  // namespace ndgi
