// Tensor-core (tcgen05) decode: declarations used by the C ABI layer.
#pragma once

#include <vector>
#include "ndgi_internal.h"

namespace ndgi {

// Launch shape of the persistent page-decode kernel (picked by the autotuner).
struct TcPagesShape {
  int ctas_per_sm;     // CTAs per SM in the persistent grid
  int lanes;           // warpgroup lanes per CTA; the lanes split a request's 64x64 quadrants
                       // (8: four MMA lanes, each with a producer warpgroup for its layer-1 rows)
  int slots;           // 128-row tiles in flight per lane (at most 4 per CTA: tensor-memory bound)
};

bool tc_supported(int cs, int ct, int hidden);
bool tc_pages_supported(int cs, int ct, int hidden);
// The tensor-core point decode's gather alone, from a prepared FP16/BF16 workspace.
cudaError_t launch_debug_features_tc(const DevModel& m, const void* ws, const float* uvt, int64_t n, float* x,
                                     cudaStream_t s);
// FP16/BF16 workspace: the weight image, then the texel-sliced copy of the
// feature planes the point decode reads.
size_t tc_workspace_bytes(int cs, int ct, int hidden, int feat_w, int feat_h);
cudaError_t launch_tc_prepare(const DevModel& m, bool bf16, void* ws, cudaStream_t s);
// Point decode gather policy: kPointsAuto decodes through the decoded-texel
// cache (built first, in the same call) when the workspace has one and the
// call has at least feat_w * feat_h / 2 queries, else directly;
// kPointsBuild / kPointsReuse force the cache path, building the cache or
// reusing the one an earlier call on the same stream built from the same
// workspace; kPointsDirect forces the direct gather.
enum { kPointsAuto = 0, kPointsBuild = 1, kPointsReuse = 2, kPointsDirect = 3 };
bool tc_points_cache_path(const DevModel& m, int64_t n, int mode);
// The cache path runs the warp-specialised point kernel for this shape (else the four-lane one).
bool tc_points_ws_built(int cs, int ct, int hidden);
cudaError_t launch_tc_points(const DevModel& m, bool bf16, const void* ws, const float* uvt, int64_t n, float* rgb,
                             cudaStream_t s, int mode);
// The cache path's gather alone (builds the cache, then x [n][cs+ct]).
cudaError_t launch_debug_features_cache(const DevModel& m, const void* ws, const float* uvt, int64_t n, float* x,
                                        cudaStream_t s);
// staged: every model's features are at most half its lightmap resolution.
// prec: 0 FP16, 1 BF16, 2 E4M3 (the workspace then comes from launch_tc_prepare8).
cudaError_t launch_tc_pages(const PagesCtx& c, int prec, int cs, int ct, int hidden, const TcPagesShape& shape,
                            bool staged, const ndgi_page_req* reqs, const int32_t* n_dev, cudaStream_t s);
// FP8 (E4M3) page decode: supported shapes, image size, image builder from the
// calibration maxima (host array of 3), and the byte offset of the image's
// status word (bit 0: a bias out of the representable range; bit 1: 1/a1 too large).
bool tc_fp8_pages_supported(int cs, int ct, int hidden);
size_t tc_fp8_workspace_bytes(int cs, int ct, int hidden, int feat_w, int feat_h);
cudaError_t launch_tc_prepare8(const DevModel& m, const float act_max[3], void* ws, cudaStream_t s);
uint32_t tc_fp8_status_offset(int cs, int ct, int hidden);
// Stored FP8 parameters of a host copy of the image as FP32 (see ndgi_fp8_unpack);
// returns the number of floats (written only if len is enough).
size_t tc_fp8_unpack(int cs, int ct, int hidden, const unsigned char* image, float* out, size_t len);
TcPagesShape tc_default_pages_shape();
// Byte offset of the error word (then the debug word) in an FP16/BF16 workspace.
uint32_t tc_error_offset(int cs, int ct, int hidden);
std::vector<TcPagesShape> tc_pages_candidates(int sms);

}  // namespace ndgi
