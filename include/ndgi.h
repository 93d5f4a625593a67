/*
 * ndgi.h -- C ABI of libndgi.so: random-access neural decode of temporal
 * lightmap sets (Neural Dynamic GI, arXiv 2604.12625) on NVIDIA GB300 (sm_103a).
 *
 * The library evaluates the compact model of Sec. 3.1, Eq. 3,
 *     I(u, v, t) = H_Theta(u, v, t),
 * in the form fixed for this library: one spatial feature map of `cs`
 * single-channel BC4 planes (4x4 blocks of two 8-bit endpoints and sixteen
 * 3-bit indices; the endpoint/weight block form of Sec. 3.4, Eq. 6-7 and
 * supplement S2) sampled bilinearly at (u, v); one temporal feature line of
 * `t_count` x `ct` values sampled linearly at t (the linear operator of
 * Sec. 3.1, Eq. 2, applied to features); their concatenation fed to an MLP
 * with two hidden ReLU layers and a linear RGB output (Sec. 4).
 *
 * Conventions for every call
 *   - Every buffer argument is caller-owned DEVICE memory unless the comment
 *     says "host".  The library never frees caller memory and keeps no
 *     pointer to it after the call returns, except a pages plan, which
 *     records the model descriptors, workspaces and physical texture given
 *     to ndgi_pages_plan_create until it is destroyed.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     enqueue work on it and return without synchronising; results are
 *     valid once the stream has reached that point.
 *   - Every call returns an ndgi_status.  Argument errors are detected on the
 *     host before anything is enqueued.  No call traps, asserts or aborts;
 *     ndgi_last_error() gives a message for the most recent failure on the
 *     calling thread.
 *   - Feature coordinates use the texel-centre convention x = u*feat_w - 0.5;
 *     keyframes sit at t_j = j/t_count and the temporal axis is periodic
 *     (the segment after the last keyframe interpolates back to row 0).
 */
#ifndef NDGI_H_
#define NDGI_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NDGI_OK = 0,
  NDGI_ERR_INVALID_ARG = 1,   /* a pointer, size or enum is out of range   */
  NDGI_ERR_UNSUPPORTED = 2,   /* valid, but this shape/precision not built */
  NDGI_ERR_CUDA = 3,          /* a CUDA runtime call failed                */
  NDGI_ERR_OOM = 4,           /* a library-owned allocation failed         */
  NDGI_ERR_TIMEOUT = 5,       /* a bounded device wait ran out             */
  NDGI_ERR_DEVICE_CHECK = 6   /* a device-side argument check failed       */
} ndgi_status;

typedef enum {
  NDGI_FP32 = 0,              /* plain FP32 CUDA-core decode               */
  NDGI_FP16 = 1,              /* tcgen05 tensor cores, FP16 operands, FP32 accumulate */
  NDGI_BF16 = 2,              /* tcgen05 tensor cores, BF16 operands, FP32 accumulate */
  NDGI_FP8_E4M3 = 3           /* tcgen05 kind::f8f6f4, E4M3 weights and activations, FP32 accumulate
                                 (page decode only; prepared with ndgi_prepare_fp8) */
} ndgi_precision;

/*
 * A decodable model (Sec. 3.3, Eq. 5 restricted to one BC feature map, one
 * temporal line and the decoder parameters Phi).  A view: every pointer is
 * device memory owned by the caller.
 *   lm_w, lm_h       lightmap size; used to turn page texels into (u, v)
 *   feat_w, feat_h   feature-plane size, multiples of 4
 *   cs               number of BC4 planes (spatial feature channels)
 *   bc4              [feat_h/4][feat_w/4][cs][8] bytes: per block, per plane,
 *                    byte0 = r0, byte1 = r1, then 48 index bits little-endian,
 *                    texel p = 4*row + col at bit 16 + 3p of the 64-bit block
 *   t_count, ct      temporal line: t_count keyframes of ct channels
 *   temporal         [t_count][ct] of temporal_dtype (NDGI_FP32 or NDGI_FP16)
 *   hidden           width of both hidden layers
 *   w1 [cs+ct][hidden], b1 [hidden], w2 [hidden][hidden], b2 [hidden],
 *   w3 [hidden][3], b3 [3]: FP32, row-major [in][out]
 *   address_mode     0 = clamp to edge, 1 = mirrored repeat (spatial axes)
 *   key_t            NULL: keyframes at t_j = j/t_count; else [t_count] FP32
 *                    keyframe times 0 <= t_0 < ... < t_(T-1) < 1 (Sec. 3.1:
 *                    non-uniform, e.g. denser around a light-switch event):
 *                    t (periodic, period 1) interpolates the two rows of the
 *                    segment holding it, the last segment running from
 *                    t_(T-1) to t_0 + 1.  Times that break the order give
 *                    unspecified (but in-bounds) results.
 */
typedef struct {
  int32_t lm_w, lm_h;
  int32_t feat_w, feat_h, cs;
  const uint8_t *bc4;
  int32_t t_count, ct;
  const void *temporal;
  int32_t temporal_dtype;
  int32_t hidden;
  const float *w1, *b1, *w2, *b2, *w3, *b3;
  int32_t address_mode;
  const float *key_t;
} ndgi_model_desc;

/* Library version string (static storage). */
const char *ndgi_version(void);

/*
 * Copies the message of the calling thread's most recent failed call into
 * buf (host, NUL-terminated, truncated to buf_len).  Returns the status of
 * that failure, NDGI_OK if none.
 */
ndgi_status ndgi_last_error(char *buf, size_t buf_len);

/*
 * Synchronises `stream` and reports any asynchronous CUDA error raised by
 * work enqueued on it (NDGI_ERR_CUDA).  Device-side failures are latched per
 * call in caller-owned error words instead: a tensor-core kernel whose
 * bounded barrier wait runs out unwinds, frees its tensor memory and sets
 * bit 4 (16) of the error word of its workspace (point decodes; read with
 * ndgi_workspace_check) or of its plan (page decodes; ndgi_pages_check).
 */
ndgi_status ndgi_check(void *stream);

/*
 * Synchronises `stream`, then reads and clears the error word held in a
 * prepared FP16/BF16 workspace `ws` (device): every point decode that used
 * this workspace latches into it.  *device_error (host, may be NULL)
 * receives the word; bit 4 (16) = a bounded barrier wait ran out
 * (NDGI_ERR_TIMEOUT is returned).  Decodes that share a workspace share the
 * word; decodes with different workspaces never see each other's errors.
 * ndgi_prepare clears the word.  The paper has no counterpart (a library
 * service).
 */
ndgi_status ndgi_workspace_check(const ndgi_model_desc *model, ndgi_precision precision, const void *ws,
                                 int32_t *device_error, void *stream);

/*
 * Test hook for the timeout path (no paper counterpart).  flags = 1 makes
 * every later tensor-core point decode with this workspace wait, with a
 * short limit, for a barrier phase that nothing completes, before it issues
 * any MMA; the decode then takes its real timeout path (lanes stop at
 * their next barrier, tensor memory is freed, bit 4 of the workspace's
 * error word is set) and its output is unspecified.  flags = 0 restores
 * normal decodes.  Enqueued on `stream`.
 */
ndgi_status ndgi_debug_workspace_inject(const ndgi_model_desc *model, ndgi_precision precision, void *ws,
                                        int32_t flags, void *stream);

/*
 * Bytes of device workspace that ndgi_prepare needs for `precision`: the
 * MLP weights re-packed for the tensor-core decode, the texel-sliced copy of
 * the planes, and (FP16/BF16, maps with feat_w * feat_h * cs * 2 <= 64 MiB)
 * room for the point decode's decoded-texel cache.  0 for NDGI_FP32.
 */
size_t ndgi_prepare_workspace_size(const ndgi_model_desc *model, ndgi_precision precision);

/*
 * Packs the model's MLP into `ws` (device, caller-owned, ws_bytes >=
 * ndgi_prepare_workspace_size, 256-byte aligned) for decodes of
 * `precision`: weights rounded once to FP16/BF16 (round to nearest even),
 * laid out as the tensor-core operand tiles, followed by a texel-sliced copy
 * of the BC4 planes for the tensor-core decodes (the same information
 * regrouped so that a texel of every plane is two short reads: per block the
 * cs endpoint pairs, then per texel one 8-byte word holding, per plane, its
 * 3-bit index and the block's palette mode (r0 <= r1) as a 4-bit nibble;
 * 1.25x the planes' size for cs = 16).  The packed weights are the parameters such a
 * decode evaluates.  Re-run it whenever the weights or the planes change.
 */
ndgi_status ndgi_prepare(const ndgi_model_desc *model, ndgi_precision precision, void *ws, size_t ws_bytes,
                         void *stream);

/*
 * FP8 calibration for ndgi_prepare_fp8: runs the FP32 decode at the n
 * queries uvt [n][3] (device) and writes act_max[0..2] (device, 3 floats) =
 * the maxima of |layer-1 input| (spatial and temporal features), relu(z1) and
 * relu(z2) over them.  Asynchronous on `stream`.
 */
ndgi_status ndgi_calibrate_fp8(const ndgi_model_desc *model, const float *uvt, int64_t n, float *act_max,
                               void *stream);

/*
 * Packs the model for the FP8 (E4M3) page decode.  The paper names FP8
 * weights with per-layer scales but not their choice; this library uses
 * powers of two throughout, so that each layer's FP32 accumulator is already
 * in the next layer's activation unit.  With act_max = (m1, m2, m3) (host
 * array, e.g. copied from ndgi_calibrate_fp8) and p2(y) the smallest power
 * of two P with y <= 448 P:
 *   a1 = p2(m1), s1 = p2(max(max|W1|, m2/a1)), a2 = a1 s1,
 *   s2 = p2(max(max|W2|, m3/a2)), a3 = a2 s2, s3 = p2(max|W3|).
 * Stored weights are s_l e4m3(W_l / s_l) (round to nearest even,
 * saturating); layer inputs are quantised as a_l e4m3(x / a_l); a bias b of
 * a layer with output unit u (a2, a3, a3 s3) is stored as u v (t1 + t2 + t3),
 * three E4M3 terms of b/(u v) with v = max(1, p2(max|b/u|)).  For pages the
 * layer-1 temporal term (quantised v_t) is folded per request into b1'.
 * ws: device, >= ndgi_prepare_workspace_size(model, NDGI_FP8_E4M3) bytes,
 * 256-byte aligned.  Synchronises `stream` to read the image's status:
 * NDGI_ERR_UNSUPPORTED if a bias needs v > 256 or 1/a1 > 2^14.  Shapes:
 * cs = 16 and hidden a multiple of 32.
 */
ndgi_status ndgi_prepare_fp8(const ndgi_model_desc *model, const float act_max[3], void *ws, size_t ws_bytes,
                             void *stream);

/*
 * Validation helper: the parameters an FP8 image stores, as FP32 values in
 * out (host): [16] header {a1, a2, a3, out = a3 s3, s1, s2, s3, v2, v3,
 * status, 0...}, then W1 [cs+ct][hidden] (spatial rows s1 * E4M3; temporal
 * rows the stored FP32 values), W2 [hidden][hidden], W3 [hidden][3], b2
 * [hidden], b3 [3].  *needed (may be NULL) receives the float count; out ==
 * NULL only queries it.  Copies ws (device) synchronously.
 */
ndgi_status ndgi_fp8_unpack(const ndgi_model_desc *model, const void *ws, float *out, size_t out_len,
                            size_t *needed);

/*
 * Random-access point decode (Sec. 3.1, Eq. 3; Sec. 5.5 decodes this way):
 * for each i < n, rgb[i] = H(u_i, v_i, t_i).
 *   uvt  [n][3] FP32 (u, v, t); rgb [n][3] FP32 output.
 *   ws   the prepared workspace for `precision` (ignored for NDGI_FP32); the
 *        decode writes nothing to it but its error word (see
 *        ndgi_workspace_check) and its decoded-texel cache.
 * FP16/BF16 gather: when the workspace has room for the cache and n >=
 * feat_w * feat_h / 2 (many queries per feature texel), the call first
 * decodes every BC4 texel of the map once into the FP16 cache and then
 * blends each query's four taps from it in half2 arithmetic (the taps and
 * fractions are those of the direct gather); otherwise each query decodes
 * its taps' palette entries directly.  ndgi_decode_points_path tells which.
 * Decodes that share a workspace and may overlap on the GPU race on its
 * cache: serialise them on one stream, or give each stream its own
 * workspace.
 * n == 0 is a no-op.  Non-finite coordinates give unspecified but in-bounds
 * results.
 */
ndgi_status ndgi_decode_points(const ndgi_model_desc *model, ndgi_precision precision, const void *ws,
                               const float *uvt, int64_t n, float *rgb, void *stream);

/*
 * How ndgi_decode_points of n queries with this model and precision gathers:
 * 0 directly (and for FP32), 1 through the decoded-texel cache with four
 * lanes per SM that each gather and run their MMA chain, 2 through the cache
 * with the warp-specialised kernel (per lane, a producer warpgroup gathers
 * the next tile while a consumer warpgroup runs the MMA chain).
 */
int32_t ndgi_decode_points_path(const ndgi_model_desc *model, ndgi_precision precision, int64_t n);

/*
 * Point decode from HOST buffers (the paper decodes on the device only;
 * this is a serving service around ndgi_decode_points).  A pipe overlaps,
 * chunk by chunk, the copy of queries to the device, the decode, and the
 * copy of results back to the host: while chunk k is decoded on the
 * caller's stream, chunk k + 1 is copied in and chunk k - 1 copied out on
 * the pipe's two copy streams.
 *
 * ndgi_host_pipe_staging_size: bytes of device staging a pipe with this
 *   chunk (queries per chunk, >= 1) needs: three chunk buffers of queries and
 *   results (24 bytes per query each, rounded up to 256-byte boundaries).
 * ndgi_host_pipe_create: makes a pipe on the current device.  `staging` is
 *   caller-owned device memory of at least that size, 256-byte aligned, used
 *   by the pipe until it is destroyed.  The pipe creates its two copy
 *   streams and its events here (never during a decode).
 *   NDGI_ERR_INVALID_ARG for chunk < 1, a NULL, short or unaligned staging.
 * ndgi_decode_points_host: the decode of ndgi_decode_points with
 *   uvt_host [n][3] and rgb_host [n][3] FP32 in host memory.  Enqueues all
 *   work and returns: the results are in rgb_host once `stream` has reached
 *   this point (synchronise it).  uvt_host must stay unchanged and rgb_host
 *   untouched until then.  Page-locked (pinned) host buffers give the
 *   overlap; pageable ones still decode correctly but the copies then
 *   serialise.  Call on the pipe's device; one host thread at a time per
 *   pipe; successive calls on a pipe are ordered (a call's first copy waits
 *   for the previous call's last one).  n == 0 is a no-op.  Errors as for
 *   ndgi_decode_points, and NDGI_ERR_INVALID_ARG for a pipe of another
 *   device or NULL host buffers.
 * ndgi_host_pipe_destroy: synchronises the pipe's streams and frees them and
 *   its events (not the staging).  NULL is a no-op.
 */
typedef struct ndgi_host_pipe ndgi_host_pipe;
size_t ndgi_host_pipe_staging_size(int64_t chunk);
ndgi_status ndgi_host_pipe_create(int64_t chunk, void *staging, size_t staging_bytes, ndgi_host_pipe **pipe);
ndgi_status ndgi_decode_points_host(ndgi_host_pipe *pipe, const ndgi_model_desc *model, ndgi_precision precision,
                                    const void *ws, const float *uvt_host, int64_t n, float *rgb_host,
                                    void *stream);
ndgi_status ndgi_host_pipe_destroy(ndgi_host_pipe *pipe);

/*
 * The gather stage alone (Sec. 3.3 sampling of the feature map and temporal
 * line), for validation: x [n][cs+ct] FP32 receives [v_s, v_t]; p35
 * [n][4][cs] int32 (may be NULL) receives, for the taps (x0,y0), (x1,y0),
 * (x0,y1), (x1,y1), the BC4 palette numerator P35 (value = P35/8925) of each
 * plane: the exact integer the decode used.
 */
ndgi_status ndgi_debug_features(const ndgi_model_desc *model, const float *uvt, int64_t n, float *x,
                                int32_t *p35, void *stream);

/*
 * The gather of the FP16/BF16 point decode alone, for validation: the same
 * x [n][cs+ct] as ndgi_debug_features (identical taps, fractions and
 * palette integers; FP32 arithmetic reassociated), computed from the
 * texel-sliced copy of the planes that ndgi_prepare keeps in `ws` (a
 * workspace prepared for NDGI_FP16 or NDGI_BF16; re-run ndgi_prepare after the
 * planes change).
 */
ndgi_status ndgi_debug_features_tc(const ndgi_model_desc *model, const void *ws, const float *uvt, int64_t n,
                                   float *x, void *stream);

/*
 * The gather of the point decode's cache path alone, for validation: builds
 * the decoded-texel cache in `ws` (FP16/BF16 workspace of a map whose cache
 * fits; NDGI_ERR_UNSUPPORTED otherwise), then writes x [n][cs+ct] FP32: the
 * half2 blend of the four cached taps (exactly the FP16 values the decode
 * feeds the MLP) and the FP32 temporal feature.
 */
ndgi_status ndgi_debug_features_cache(const ndgi_model_desc *model, const void *ws, const float *uvt, int64_t n,
                                      float *x, void *stream);

/* ---------------------------------------------------------------------- */
/* Batched virtual-texture page decode (Sec. 3.5, supplement S3)           */
/* ---------------------------------------------------------------------- */

/*
 * One page request: decode texels (x0+i, y0+j), 0 <= i < w, 0 <= j < h, of
 * lightmap `model` at time t into the physical texture at (dst_x+i, dst_y+j).
 * 1 <= w, h <= 128; the source rectangle lies inside the lightmap and the
 * destination inside the physical texture.  32 bytes.
 */
typedef struct {
  int32_t model, x0, y0, w, h;
  float t;
  int32_t dst_x, dst_y;
} ndgi_page_req;

typedef enum {
  NDGI_RGBA32F = 0,           /* 16 bytes per texel, A = 1                 */
  NDGI_RGBA16F = 1,           /* 8 bytes per texel, A = 1                  */
  NDGI_RGBA8 = 2              /* 4 bytes per texel, UNORM: round(255 clamp(y, 0, 1)), A = 255; hybrid
                                 tables only (the paper's 8-bit, 4-channel physical texture, which holds
                                 the model's normalised output) */
} ndgi_out_format;

typedef struct ndgi_pages_plan ndgi_pages_plan;

/*
 * Creates a reusable plan for page decodes: n_models model descriptors
 * (host array, copied), their prepared workspaces ws[i] (host array of
 * device pointers; NULL entries allowed for NDGI_FP32), the physical
 * texture phys (device, [phys_h][phys_w] texels of out_format) and the
 * maximum number of requests per call.  The plan owns a small device
 * block (model table, work counter, error word) and the CUDA graph of the
 * decode.  *plan receives the handle.
 */
ndgi_status ndgi_pages_plan_create(const ndgi_model_desc *models, const void *const *ws, int32_t n_models,
                                   ndgi_precision precision, int32_t max_reqs, int32_t out_format, void *phys,
                                   int64_t phys_w, int64_t phys_h, ndgi_pages_plan **plan);

/*
 * Decodes the requests reqs_dev[0 .. *n_dev) (both device memory, so a
 * frame's request list can be produced on the GPU) with one persistent
 * launch replayed from the plan's CUDA graph.  reqs_dev must hold at least
 * *n_dev entries.  Requests that fail the device-side checks (bad model id,
 * sizes outside 1..128, rectangles outside the lightmap or the physical
 * texture) are skipped; *n_dev < 0 or > max_reqs rejects the whole frame.
 * Both are latched in the plan's error word (bit 0: count, bit 1: model or
 * size, bit 2: rectangle; FP8 plans also bit 3: a request's folded bias
 * needed a ones value above 256 and was clamped), which ndgi_pages_check
 * reads.  The graph is
 * rebuilt when reqs_dev or n_dev differ from the previous call.  Requests
 * with overlapping destinations race.
 */
ndgi_status ndgi_decode_pages(ndgi_pages_plan *plan, const ndgi_page_req *reqs_dev, const int32_t *n_dev,
                              void *stream);

/*
 * Picks the plan's launch shape (CTAs per SM and texel-tile shape) by timing
 * each candidate on the given requests (n_host = *n_dev, for sizing) and
 * keeps the fastest.  The physical texture is overwritten.
 */
ndgi_status ndgi_pages_autotune(ndgi_pages_plan *plan, const ndgi_page_req *reqs_dev, const int32_t *n_dev,
                                int32_t n_host, void *stream);

/*
 * Synchronises `stream` and reads the plan's device error word into
 * *device_error (host; 0 = no request was rejected), then clears it.
 * Returns NDGI_ERR_TIMEOUT if bit 4 (16: a tensor-core kernel's bounded
 * barrier wait ran out) is set, else NDGI_ERR_DEVICE_CHECK if any bit is.
 */
ndgi_status ndgi_pages_check(ndgi_pages_plan *plan, int32_t *device_error, void *stream);

/*
 * The plan's current launch shape (host int32[4]): precision, CTAs per SM,
 * warpgroup lanes per CTA, tiles in flight per lane (the last three describe
 * the tensor-core kernel; for NDGI_FP32 plans info[1] is the grid size).
 * Built tensor-core shapes: 4 x 1 and 2 x 2 (every lane runs its own MMA
 * chain and writes its own layer-1 rows), and 8 x 1, the warp-specialised
 * kernel: four MMA lanes, each paired with a warpgroup that writes the
 * layer-1 rows of the lane's next tile (plans whose features are at most
 * half the lightmap resolution; other plans run 4 x 1 under that shape).
 */
ndgi_status ndgi_pages_plan_info(const ndgi_pages_plan *plan, int32_t info[4]);

/*
 * Pins the tensor-core plan's launch shape (CTAs per SM, warpgroup lanes per
 * CTA, tiles in flight per lane) instead of the autotuner's choice.  A CTA
 * holds most of its SM's tensor memory, so ctas_per_sm must be 1.
 * NDGI_ERR_UNSUPPORTED if that shape is not built for the plan's model
 * shape; NDGI_ERR_INVALID_ARG for NDGI_FP32 plans or other ctas_per_sm.
 */
ndgi_status ndgi_pages_plan_set_shape(ndgi_pages_plan *plan, int32_t ctas_per_sm, int32_t lanes, int32_t slots);

/*
 * Test hook for the timeout path (no paper counterpart): flags = 1 makes the
 * plan's tensor-core decodes take their timeout path from a short wait on a
 * barrier phase that nothing completes, before any MMA is issued (bit 4 of
 * the plan's error word is set; output unspecified); 0 restores normal
 * decodes.  Copies synchronously; FP32 plans ignore it.
 */
ndgi_status ndgi_pages_plan_set_debug(ndgi_pages_plan *plan, int32_t flags);

/*
 * Test hook for the FP8 page decode's rounding accounting (no paper
 * counterpart).  With dump != NULL (device, 16-byte aligned,
 * ndgi_pages_fp8_dump_size bytes), later decodes of this FP8 plan with the
 * 4 x 1 launch shape copy the operands of one tile into dump: the first 2 x 64
 * texels (rows y0, y0+1, columns x0..x0+63; thread t is texel (t mod 64,
 * t div 64)) of request number `item` of the frame.  Layout, 32-bit words:
 *   [128][R], R = 8 + 2H + 2Q + 4, Q = (H + 32) / 4, per texel row t:
 *     A1 (8 words: the 32 E4M3 codes of the layer-1 row: 16 features in
 *        units a1, the three ones codes of v1, zeros),
 *     D1 (H FP32: the layer-1 accumulator, in units a2),
 *     A2 (Q words: the layer-2 row, H codes then the ones codes),
 *     D2 (H FP32, units a3), A3 (Q words), D3 (4 FP32: RGB in units out, pad);
 *   then vt [ct] FP32 (the request's quantised temporal features) and
 *   b1t [H] (bytes 0..2: the three E4M3 terms of b1' / (a2 v1) per output).
 * dump = NULL turns it off.  This call and ndgi_pages_plan_set_debug each
 * set the whole debug state.
 */
size_t ndgi_pages_fp8_dump_size(const ndgi_pages_plan *plan);
ndgi_status ndgi_pages_plan_set_fp8_dump(ndgi_pages_plan *plan, int32_t item, void *dump);

/* Destroys the plan and its device block and graph.  NULL is a no-op. */
ndgi_status ndgi_pages_plan_destroy(ndgi_pages_plan *plan);

/*
 * Page decode that allocates nothing (the paper has no counterpart; this is
 * a library service).  For callers that cannot call cudaMalloc, such as code
 * that runs inside a fixed memory arena or a real-time frame loop where an
 * allocation could block on the driver: the same FP32 page decode as a plan
 * with NDGI_FP32, but the model table and error word live in a static
 * device array of the library instead of a plan's allocated block.
 *   models       host array of n_models descriptors, 1 <= n_models <= 64
 *                (more is rejected with NDGI_ERR_INVALID_ARG)
 *   reqs_dev, n_dev, max_reqs, out_format, phys, phys_w, phys_h
 *                as for ndgi_pages_plan_create / ndgi_decode_pages
 *   device_error device int32 (may be NULL) that receives the error word of
 *                this call (same bits as ndgi_pages_check reports)
 * The static array is shared by every call and keeps the last call's
 * contents; each call rewrites it on `stream` before its decode (a small
 * kernel that receives the descriptors by value and clears the error word),
 * so calls that overlap on the GPU race.  The call returns without waiting
 * for `stream`.  The first call on a device looks up the array's device
 * address (once per device); make that first call before any stream
 * capture.  Descriptors are checked like ndgi_pages_plan_create's; all must
 * share cs, ct and hidden (NDGI_ERR_UNSUPPORTED otherwise).
 */
ndgi_status ndgi_decode_pages_static(const ndgi_model_desc *models, int32_t n_models,
                                     const ndgi_page_req *reqs_dev, const int32_t *n_dev, int32_t max_reqs,
                                     int32_t out_format, void *phys, int64_t phys_w, int64_t phys_h,
                                     int32_t *device_error, void *stream);

/* ---------------------------------------------------------------------- */
/* BC simulation and packing (Sec. 3.4, Eq. 6-7)                          */
/* ---------------------------------------------------------------------- */

/*
 * Packs trained endpoints and weights into BC4 blocks whose decode equals
 * the straight-through simulated values exactly (end of Sec. 3.4: after
 * training, the feature map is rebuilt from E and W, quantised and block
 * compressed).  Per block and plane: A = q255(ea), B = q255(eb),
 * k_p = q7(w_p) with q_s(x) = floor(min(max(s*x + 0.5, 0), s)) in FP32;
 *   A > B : r0 = A, r1 = B, index = (k == 0 ? 0 : k == 7 ? 1 : k + 1)
 *   A < B : r0 = B, r1 = A, the same map applied to 7 - k
 *   A == B: r0 = r1 = A, all indices 0.
 * ea, eb [feat_h/4][feat_w/4][cs] FP32, w [feat_h/4][feat_w/4][cs][16] FP32,
 * bc4_out [feat_h/4][feat_w/4][cs][8] bytes.
 */
ndgi_status ndgi_bc_pack(const float *ea, const float *eb, const float *w, int32_t cs, int32_t feat_w,
                         int32_t feat_h, uint8_t *bc4_out, void *stream);

/* ---------------------------------------------------------------------- */
/* BC7 (Sec. 3.4: F_uv and F3D quantised to 8 bits and BC7-compressed)     */
/* ---------------------------------------------------------------------- */

/*
 * BC7 compression of an RGBA8 image rgba [h][w][4] (w, h multiples of 4;
 * several images of one width may be stacked along h, e.g. the F3D slices)
 * into blocks [h/4][w/4][16].  The encoder is deterministic and integer-only:
 * per block it tries, in order, mode 6; mode 5 with rotation 0..3; mode 4
 * with rotation 0..3 and index selector 0..1; mode 7 with partitions 0..63;
 * and, when every alpha of the block is 255, modes 3, 1, 2 (partitions
 * 0..63) and mode 0 (partitions 0..15), keeping the first candidate with the
 * smallest squared error.  A candidate takes per subset (and per colour /
 * alpha group in modes 4, 5) the per-channel minimum and maximum as
 * endpoints, a channel swapped between them when its integer covariance
 * with the widest channel is negative, each coded by its nearest code (lowest code on ties; a p-bit
 * minimises the summed squared error, 0 on ties), and gives every texel its
 * nearest palette entry (lowest index on ties).  If sq_err is not NULL the
 * total squared error (over all texels and channels, in 8-bit units) is
 * added to the device uint64 it points to (8-byte aligned).  The other
 * buffers are device memory, 16-byte aligned.  Errors: NDGI_ERR_INVALID_ARG
 * (sizes, NULL, alignment).
 */
ndgi_status ndgi_bc7_encode(const uint8_t *rgba, int32_t w, int32_t h, uint8_t *blocks, uint64_t *sq_err,
                            void *stream);

/*
 * BC7 decode of blocks [h/4][w/4][16] to rgba [h][w][4] (the BPTC UNORM
 * format: all eight modes, two- and three-subset partitions, rotation and
 * index selector; the reserved mode decodes to 0).  Device buffers, 16-byte
 * aligned.
 */
ndgi_status ndgi_bc7_decode(const uint8_t *blocks, int32_t w, int32_t h, uint8_t *rgba, void *stream);

/*
 * 8-bit quantisation of four BC4 planes (a fit's F_uv or F3D slice packed by
 * ndgi_bc_pack with cs = 4): rgba [h][w][4] = round(255 * P35 / 8925) per
 * texel and plane, the input of ndgi_bc7_encode.  bc4 [h/4][w/4][4][8].
 */
ndgi_status ndgi_bc4x4_to_rgba8(const uint8_t *bc4, int32_t w, int32_t h, uint8_t *rgba, void *stream);

/*
 * 8-bit export of a map fitted with the shared-weight BC simulation
 * (ndgi_hybrid_fit_params.shared_w = 1): rgba [height][width][4], texel p of
 * block b = ((64 - W) A + W B + 32) >> 6 per channel with A, B the mode-6
 * endpoints of ea[b], eb[b] (ndgi_hybrid_fit_params, shared_w), W the 4-bit
 * BC7 weight of index q15(w[b][p]).  ea, eb
 * [height/4][width/4][4], w [height/4][width/4][16] FP32 (F3D slices stacked
 * along height); device buffers, 16-byte aligned.  The input of
 * ndgi_bc7_encode.
 */
ndgi_status ndgi_bc_sim7_to_rgba8(const float *ea, const float *eb, const float *w, int32_t width, int32_t height,
                                  uint8_t *rgba, void *stream);

/*
 * Exact BC7 mode-6 blocks [n_blocks][16] of a shared-weight BC simulation
 * (ea, eb [n_blocks][4], w [n_blocks][16] FP32): endpoint codes and p-bits of
 * the mode-6 endpoints, indices q15(w); where texel 0's index is 8 or more
 * the endpoints swap and index k becomes 15 - k.  The blocks decode to
 * ndgi_bc_sim7_to_rgba8's texels.  Device buffers, 16-byte aligned.
 */
ndgi_status ndgi_bc7_pack_sim(const float *ea, const float *eb, const float *w, int64_t n_blocks, uint8_t *blocks,
                              void *stream);

/*
 * Test reference: the same decode done by the GPU's texture unit (a BC7
 * view of the blocks, point-sampled at texel centres).  Allocates a CUDA
 * array and synchronises the stream; not for the decode path.
 */
ndgi_status ndgi_debug_bc7_hw_decode(const uint8_t *blocks, int32_t w, int32_t h, uint8_t *rgba, void *stream);

/* ---------------------------------------------------------------------- */
/* Differentiable fit (Sec. 3.4 BC simulation, Sec. 4 training)           */
/* ---------------------------------------------------------------------- */

/*
 * Trainable parameters, FP32 device memory owned by the caller.  The BC
 * planes are held as the simulation's endpoints and weights (Eq. 6):
 *   ea, eb [feat_h/4][feat_w/4][cs] in [0,1], w [feat_h/4][feat_w/4][cs][16]
 *   in [0,1]; temporal [t_count][ct]; MLP as in ndgi_model_desc.
 * A fit sample is a query (u, v, t), three FP32 values exactly as for
 * ndgi_decode_points (texel (ix, iy) of the lm_w x lm_h target is u =
 * (ix + 0.5) / lm_w, v = (iy + 0.5) / lm_h); t is continuous, so the
 * temporal feature is the linear interpolation (Sec. 3.1, Eq. 2) of the two
 * keyframe rows j0, j1 around t with weight alpha, as in the decode.
 */
typedef struct {
  int32_t lm_w, lm_h, feat_w, feat_h, cs, t_count, ct, hidden;
  float *ea, *eb, *w, *temporal, *w1, *b1, *w2, *b2, *w3, *b3;
  int32_t address_mode;
  const float *key_t;           /* keyframe times as in ndgi_model_desc, or NULL */
} ndgi_fit_params;

/* Gradient buffers shaped like ndgi_fit_params' tensors (FP32, device). */
typedef struct {
  float *ea, *eb, *w, *temporal, *w1, *b1, *w2, *b2, *w3, *b3;
} ndgi_fit_grads;

/*
 * Forward of the fit at n queries uvt [n][3]: rgb [n][3] FP32.  relaxed = 0 uses
 * the straight-through BC simulation (features quantised exactly as the
 * packed decode would see them); relaxed = 1 uses the continuous Eq. 7 with
 * unquantised E and W (for finite-difference checks).
 */
ndgi_status ndgi_fit_forward(const ndgi_fit_params *params, const float *uvt, int64_t n, int32_t relaxed,
                             float *rgb, void *stream);

/*
 * Backward of the fit: given dL/drgb [n][3], ADDS dL/dparam into *grads
 * (caller zeroes them).  Activations are recomputed, not stored.  The
 * straight-through estimator treats the quantisers as identity and uses
 * the quantised values as chain-rule factors:
 *   dL/dea += (1 - q(w)) g_f, dL/deb += q(w) g_f, dL/dw += (q(eb) - q(ea)) g_f.
 * The temporal feature's gradient g_t splits between the keyframe rows
 * around t: dL/dK[j0] += (1 - alpha) g_t, dL/dK[j1] += alpha g_t.
 * Accumulation uses FP32 atomics, so results vary in the last bits.
 */
ndgi_status ndgi_fit_backward(const ndgi_fit_params *params, const float *uvt, int64_t n, int32_t relaxed,
                              const float *grad_rgb, const ndgi_fit_grads *grads, void *stream);

/* Fit loop settings (Sec. 4: Adam, L2 loss; final stage freezes features). */
typedef struct {
  int32_t steps;              /* Adam steps                                 */
  int32_t batch;              /* samples per step                           */
  float lr, beta1, beta2, eps;
  int32_t freeze_steps;       /* last steps update the MLP only             */
  int32_t loss_every;         /* FP64 loss logged every k steps (0 = never) */
  uint64_t seed;              /* sample stream (counter-based SplitMix64)   */
  int32_t relaxed;            /* 1 = no BC quantisation in the forward      */
  float noise_alpha;          /* hybrid fit: V' = V + U(-1/2, 1/2) alpha on the 12 sampled map inputs (the
                                 training-time quantisation noise; 1/256 for 8-bit maps; 0 = off).  The
                                 draws are counter-based: for sample i of global step s and input k,
                                 z = splitmix64(b + k g), b = (seed ^ 0x6E6F697365) + 12 ((s << 32) + i) g,
                                 g = 0x9E3779B97F4A7C15, noise = alpha ((z >> 40) 2^-24 - 1/2).  The simple
                                 fit ignores it.                                                          */
} ndgi_fit_config;

/* Bytes of device workspace ndgi_encode_fit needs. */
size_t ndgi_encode_fit_workspace_size(const ndgi_fit_params *params, const ndgi_fit_config *cfg);

/*
 * Runs cfg->steps Adam steps of the L2 fit on device.  Each step draws
 * cfg->batch samples (texel ix, iy and time t) with the counter-based
 * generator
 *   ctr = step * 2^32 + i, z1 = SplitMix64(seed + (2 ctr + 1) g),
 *   z2 = SplitMix64(seed + (2 ctr + 2) g), g = 0x9E3779B97F4A7C15,
 *   ix = lo32(z1) mod lm_w, iy = hi32(z1) mod lm_h, t = (z2 >> 40) 2^-24,
 * evaluates the straight-through forward at ((ix + 0.5) / lm_w,
 * (iy + 0.5) / lm_h, t), the MSE against the target at t, which is the
 * keyframe targets [t_count][lm_h][lm_w][3] FP16 (device; keyframe j at
 * t = j / t_count) of that texel interpolated linearly between the two
 * keyframes around t, exactly as the temporal features are (Sec. 3.1,
 * Eq. 2: the lightmap between keyframes is their linear interpolation),
 * the backward, and Adam (endpoints
 * and weights projected onto [0,1]).  step_offset continues a previous run
 * (Adam step numbering and sample stream).  Every loss_every steps the FP64
 * batch loss is written to loss_log[k] (device, double,
 * ceil(steps/loss_every) entries, 8-byte aligned; targets 2-byte aligned;
 * NDGI_ERR_INVALID_ARG otherwise).  ws: device workspace of
 * ndgi_encode_fit_workspace_size bytes, holding the Adam moments (keep it
 * between calls to resume).  Pack the result with ndgi_bc_pack.
 */
ndgi_status ndgi_encode_fit(const ndgi_fit_params *params, const uint16_t *targets, const ndgi_fit_config *cfg,
                            int32_t step_offset, void *ws, size_t ws_bytes, double *loss_log, void *stream);

/*
 * Batched per-tile fit (Sec. 3.5 trains one model per virtual-texture tile;
 * Sec. 4 fits thousands of them side by side): ndgi_encode_fit for n_models
 * models of the same shape in one launch per step.  Each of params' ten
 * tensors holds the n_models models one after another (model m's tensor at
 * m times its single-model size), as do targets ([n_models][t_count][lm_h]
 * [lm_w][3] FP16); params' sizes are those of one model, and all models share
 * key_t.  Model m draws its samples as ndgi_encode_fit does with seed + m.
 * cfg->batch samples per model and step; loss_log holds the mean over all
 * models' samples.  ws: ndgi_encode_fit_batch_workspace_size bytes.
 * 1 <= n_models <= 65535 (one row of CTAs per model); NDGI_ERR_INVALID_ARG
 * otherwise.
 */
size_t ndgi_encode_fit_batch_workspace_size(const ndgi_fit_params *params, int32_t n_models,
                                            const ndgi_fit_config *cfg);
ndgi_status ndgi_encode_fit_batch(const ndgi_fit_params *params, int32_t n_models, const uint16_t *targets,
                                  const ndgi_fit_config *cfg, int32_t step_offset, void *ws, size_t ws_bytes,
                                  double *loss_log, void *stream);


/* ======================================================================
 * Hybrid feature map decoder: the paper's full decoder (Sec. 3.3, Eq. 4-5;
 * Sec. 4).  Four feature maps per model (Eq. 5): a low-resolution 3D map
 * F3D over (u, v, t) with 4 channels, sampled trilinearly (V_uvt), and the
 * tri-plane F_uv (4 channels), F_ut and F_vt (2 channels each), each sampled
 * bilinearly at the projection of (u, v, t) onto its plane.  The decoder
 * G_Phi takes [V_uvt, V_uv, V_ut, V_vt, gamma(t)] (16 inputs; Eq. 4,
 * gamma(t) = [sin pi t, cos pi t, sin 2 pi t, cos 2 pi t]) through two GELU
 * hidden layers (GELU(x) = x Phi(x), the exact erf form) to linear RGB.
 * Storage (this library's readings of what the paper leaves open):
 *   - F_uv and each t-slice of F3D are either four BC4 planes
 *     (NDGI_FEAT_BC4X4: block layout as ndgi_model_desc's bc4 with cs = 4,
 *     value P35 / 8925) or the paper's four-channel BC7 (NDGI_FEAT_BC7: one
 *     16-byte block per 4x4 texels, value byte / 255); F3D slices follow one
 *     another;
 *   - F_ut and F_vt are UNORM8 (value byte / 255), layout [t][x][2];
 *   - texel-centre convention on every axis; u and v follow address_mode,
 *     the t axis (t in [0, 1]) clamps to its edge texels.
 * ====================================================================== */

/*
 * A hybrid model; a view, every pointer device memory owned by the caller.
 *   lm_w, lm_h              lightmap (tile) size: page texels -> (u, v)
 *   uv_w, uv_h, uv_bc4      F_uv: sizes multiples of 4, [uv_h/4][uv_w/4][4][8]
 *                           (BC7: [uv_h/4][uv_w/4][16])
 *   vol_w, vol_h, vol_t     F3D: slice sizes multiples of 4, vol_t slices,
 *   vol_bc4                 [vol_t][vol_h/4][vol_w/4][4][8] (BC7: [..][16])
 *   ut_w, ut_t, ut          F_ut: [ut_t][ut_w][2] bytes
 *   vt_h, vt_t, vt          F_vt: [vt_t][vt_h][2] bytes
 *   hidden                  16, 32 or 64 (both hidden layers)
 *   w1 [16][hidden], b1, w2 [hidden][hidden], b2, w3 [hidden][3], b3: FP32 [in][out]
 *   address_mode            0 clamp, 1 mirrored repeat (u and v axes)
 *   feat_format             NDGI_FEAT_BC4X4 (0) or NDGI_FEAT_BC7 (1): the
 *                           block format of F_uv and F3D
 * uv_bc4 and vol_bc4 must be 16-byte aligned, ut and vt 2-byte aligned.
 */
enum { NDGI_FEAT_BC4X4 = 0, NDGI_FEAT_BC7 = 1 };
typedef struct {
  int32_t lm_w, lm_h;
  int32_t uv_w, uv_h;
  const uint8_t *uv_bc4;
  int32_t vol_w, vol_h, vol_t;
  const uint8_t *vol_bc4;
  int32_t ut_w, ut_t;
  const uint8_t *ut;
  int32_t vt_h, vt_t;
  const uint8_t *vt;
  int32_t hidden;
  const float *w1, *b1, *w2, *b2, *w3, *b3;
  int32_t address_mode;
  int32_t feat_format;
} ndgi_hybrid_desc;

/*
 * Bytes of device workspace ndgi_hybrid_prepare needs for `precision`: the
 * MLP weights re-packed for the tensor-core decode plus the decode's error
 * and debug words.  0 for NDGI_FP32 (which needs none).
 */
size_t ndgi_hybrid_workspace_size(const ndgi_hybrid_desc *model, ndgi_precision precision);

/*
 * Writes the tensor-core image of the model's MLP (NDGI_FP16 or NDGI_BF16)
 * into ws (device, 256-byte aligned, ndgi_hybrid_workspace_size bytes) and
 * clears its error word.  Re-run after changing the weights.
 */
ndgi_status ndgi_hybrid_prepare(const ndgi_hybrid_desc *model, ndgi_precision precision, void *ws, void *stream);

/*
 * Random-access decode at n queries: rgb[i] = G_Phi(features(u_i, v_i, t_i))
 * (Eq. 4).  uvt: [n][3] FP32 (device); rgb: [n][3] FP32 (device).
 * NDGI_FP32 runs the FP32 CUDA-core decode (ws unused, may be NULL);
 * NDGI_FP16 / NDGI_BF16 the tensor-core decode with the prepared ws (features
 * and hidden activations rounded to the operand type, FP32 accumulation).
 * A timed-out tensor-core wait latches bit 4 in ws's error word
 * (ndgi_hybrid_workspace_check).
 */
ndgi_status ndgi_hybrid_decode_points(const ndgi_hybrid_desc *model, ndgi_precision precision, const void *ws,
                                      const float *uvt, int64_t n, float *rgb, void *stream);

/* Reads and clears the error word of a prepared hybrid workspace (as ndgi_workspace_check). */
ndgi_status ndgi_hybrid_workspace_check(const ndgi_hybrid_desc *model, ndgi_precision precision, const void *ws,
                                        int32_t *device_error, void *stream);

/*
 * A device table of hybrid models for the page decode (Sec. 3.5: one model
 * per tile, each request names its tile's model).  Created from n_models
 * host descriptors that share `hidden`; ws[i] (host array of device
 * pointers) is model i's prepared workspace for an FP16/BF16 table, NULL for
 * NDGI_FP32.  The table copies the descriptors (the arrays they point to
 * must outlive it) and owns a device block with its error and debug words.
 */
typedef struct ndgi_hybrid_table ndgi_hybrid_table;
ndgi_status ndgi_hybrid_table_create(const ndgi_hybrid_desc *models, const void *const *ws, int32_t n_models,
                                     ndgi_precision precision, ndgi_hybrid_table **out);
ndgi_status ndgi_hybrid_table_destroy(ndgi_hybrid_table *table);

/*
 * Page decode with hybrid models: texel (x0+i, y0+j) of each request is
 * decoded at ((x0+i+0.5)/lm_w, (y0+j+0.5)/lm_h, t) with the request's model
 * and t, and written as RGBA (A = 1) to phys (device, [phys_h][phys_w][4] of
 * RGBA32F, RGBA16F or RGBA8 UNORM) at (dst_x+i, dst_y+j).  reqs: n requests
 * (device).
 * The host checks n, phys and format; the device checks each request
 * (model index, rectangle inside the lightmap and the physical texture)
 * and skips a bad one, latching bit 0 of the table's error word.
 */
ndgi_status ndgi_hybrid_decode_pages(ndgi_hybrid_table *table, const ndgi_page_req *reqs, int32_t n, void *phys,
                                     int64_t phys_w, int64_t phys_h, ndgi_out_format format, void *stream);

/*
 * Test hook for the timeout path (no paper counterpart): flags = 1 makes the
 * later tensor-core decodes that use ws (point decodes; with `model` and
 * `precision` describing it) and/or `table` (page decodes) take their real
 * timeout path before any MMA, as ndgi_debug_workspace_inject does; 0
 * restores normal decodes.  Either of ws and table may be NULL.
 */
ndgi_status ndgi_hybrid_debug_inject(const ndgi_hybrid_desc *model, ndgi_precision precision, void *ws,
                                     ndgi_hybrid_table *table, int32_t flags, void *stream);

/*
 * Mirrored tile border (supplement S3: each tile is stored with a small
 * border, e.g. 4 texels per edge, with the same mirrored padding used in
 * training, so that hardware filtering is seamless): later page decodes with
 * this table write (w + 2 border) x (h + 2 border) texels per request, at
 * (dst_x - border, dst_y - border); padded texel i of a row or column of n
 * texels decodes tile texel i - border reflected into [0, n) with the edge
 * texel repeated (-1 -> 0, n -> n - 1).  border 0..8 (default 0); a request
 * needs border <= w, h and its padded destination inside the texture.
 */
ndgi_status ndgi_hybrid_table_set_border(ndgi_hybrid_table *table, int32_t border);

/* Synchronises, reads and clears the table's error word (bit 0 bad request, bit 4 timeout). */
ndgi_status ndgi_hybrid_table_check(ndgi_hybrid_table *table, int32_t *device_error, void *stream);

/*
 * Test hook: y[i] = GELU(x[i]) on the device (x, y: n FP32, device) as the
 * FP32 decodes evaluate it (fast = 0: CUDA's erff), in the erfc form of
 * Abramowitz & Stegun 7.1.28 with one approximate reciprocal (|error| <=
 * 2e-6 (1 + |x|)): fast = 1 scalar, fast = 2 packed FP32 pairs; or fast = 3:
 * the polynomial form the FP16 / BF16 tensor-core epilogues use,
 * x/2 (1 + t P(t^2)), t = clamp(x, -4.5, 4.5), |error| <= 4.5e-5 + 4e-6 |x|.
 */
ndgi_status ndgi_debug_gelu(const float *x, int64_t n, float *y, int32_t fast, void *stream);

/*
 * Storage of a hybrid model in bits per lightmap texel, the paper's accounting
 * (Table "compression" and Table "config"): the BC-compressed maps F_uv and
 * F3D at bc_bits_per_texel bits per texel of all four channels (8 for BC7,
 * the paper's format; 16 for four BC4 planes; <= 0: the model's
 * feat_format decides), F_ut and F_vt
 * at 8 bits per value, and the MLP's parameters at mlp_bits (16 for FP16),
 * divided by lm_w * lm_h * n_lightmaps texels.  Host only; -1 on a bad
 * argument.
 */
double ndgi_model_bpp(const ndgi_hybrid_desc *model, int32_t n_lightmaps, int32_t bc_bits_per_texel,
                      int32_t mlp_bits);

/* ======================================================================
 * Fit of the hybrid decoder (Sec. 3.4's BC simulation applied to the
 * decoder of Sec. 3.3; Sec. 4 training)
 * ====================================================================== */

/*
 * Trainable parameters of one hybrid model (FP32, device, row-major):
 *   uv_ea, uv_eb [uv_h/4][uv_w/4][4], uv_wt [uv_h/4][uv_w/4][4][16]   F_uv as BC
 *       endpoints per block and channel and a weight per texel (Eq. 6-7);
 *   vol_ea, vol_eb [vol_t][vol_h/4][vol_w/4][4], vol_wt [..][4][16]    F3D likewise;
 *   ut [ut_t][ut_w][2], vt [vt_t][vt_h][2]                             F_ut, F_vt values;
 *   w1 [16][hidden], b1, w2 [hidden][hidden], b2, w3 [hidden][3], b3   the MLP.
 * The forward is the hybrid decode with F_uv and F3D read through the
 * straight-through quantisers of ndgi_fit_forward (A = q255(ea), B =
 * q255(eb), k = q7(w), value P35 / 8925; relaxed = 1: (1 - w) ea + w eb) and
 * F_ut / F_vt used as given; GELU(x) = x Phi(x) in FP32 (CUDA's erff).
 * Pack a result with ndgi_bc_pack (cs = 4; per F3D slice) and round F_ut /
 * F_vt to UNORM8.  hidden 16, 32 or 64.
 * shared_w = 1 follows Eq. 7 literally: one weight per texel shared by the
 * four channels (uv_wt [uv_h/4][uv_w/4][16], vol_wt [vol_t][..][16]), read as
 * BC7 mode 6: the mode-6 endpoints A, B of ea, eb (each channel q255, then
 * the endpoint's p-bit = the majority parity of its four channels, 0 on a
 * 2-2 tie, and each channel the nearest value of that parity, the lower on a
 * tie), W = the 4-bit BC7 weight of index q15(w), value ((64 - W) A + W B +
 * 32) >> 6 over 255 (relaxed: (1 - w) ea + w eb).  Export exactly with
 * ndgi_bc7_pack_sim, or as the paper does (8-bit maps re-encoded) with
 * ndgi_bc_sim7_to_rgba8 and ndgi_bc7_encode.
 */
typedef struct {
  int32_t lm_w, lm_h;
  int32_t uv_w, uv_h, vol_w, vol_h, vol_t, ut_w, ut_t, vt_h, vt_t;
  int32_t hidden, address_mode;
  float *uv_ea, *uv_eb, *uv_wt, *vol_ea, *vol_eb, *vol_wt, *ut, *vt, *w1, *b1, *w2, *b2, *w3, *b3;
  int32_t shared_w;
} ndgi_hybrid_fit_params;

/* Gradient buffers in ndgi_hybrid_fit_params' tensor order (FP32, device). */
typedef struct {
  float *g[14];
} ndgi_hybrid_fit_grads;

/* rgb [n][3] of the forward at queries uvt [n][3] (device). */
ndgi_status ndgi_hybrid_fit_forward(const ndgi_hybrid_fit_params *params, const float *uvt, int64_t n,
                                    int32_t relaxed, float *rgb, void *stream);

/*
 * Given dL/drgb [n][3], ADDS dL/dparam into *grads (caller zeroes them):
 * through the MLP (GELU'(z) = Phi(z) + z phi(z)), the trilinear F3D, the
 * bilinear F_uv / F_ut / F_vt samples and the straight-through quantisers
 * (dL/dea += (1 - q(w)) g, dL/deb += q(w) g, dL/dw += (q(eb) - q(ea)) g).
 * FP32 atomics: results vary in the last bits.
 */
ndgi_status ndgi_hybrid_fit_backward(const ndgi_hybrid_fit_params *params, const float *uvt, int64_t n,
                                     int32_t relaxed, const float *grad_rgb, const ndgi_hybrid_fit_grads *grads,
                                     void *stream);

/*
 * Runs cfg->steps Adam steps of the L2 fit of a hybrid model on device, as
 * ndgi_encode_fit: cfg->batch samples per step drawn with the same
 * counter-based generator (texel and t), targets [t_count][lm_h][lm_w][3]
 * FP16 (device) at the keyframe times (key_t, device, or NULL for j /
 * t_count) interpolated linearly at t, the feature maps projected onto
 * [0, 1] and frozen for the last cfg->freeze_steps steps (the final stage
 * fine-tunes the MLP alone, Sec. 4).  ws: ndgi_hybrid_encode_fit_workspace_size
 * bytes (Adam moments; keep it to resume with step_offset).  targets must be
 * 2-byte and loss_log 8-byte aligned (NDGI_ERR_INVALID_ARG otherwise).
 */
size_t ndgi_hybrid_encode_fit_workspace_size(const ndgi_hybrid_fit_params *params, const ndgi_fit_config *cfg);
ndgi_status ndgi_hybrid_encode_fit(const ndgi_hybrid_fit_params *params, const uint16_t *targets, int32_t t_count,
                                   const float *key_t, const ndgi_fit_config *cfg, int32_t step_offset, void *ws,
                                   size_t ws_bytes, double *loss_log, void *stream);

/*
 * Batched per-tile fit of hybrid models (Sec. 4 trains thousands of per-tile
 * models side by side): ndgi_hybrid_encode_fit for n_models models of one
 * shape in one launch per step.  Each of params' fourteen tensors holds the
 * n_models models one after another (model m at m times its single-model
 * size), as do targets ([n_models][t_count][lm_h][lm_w][3] FP16); params'
 * sizes are those of one model, and all models share key_t.  Model m draws
 * its samples (and training noise) as ndgi_hybrid_encode_fit does with
 * seed + m.  cfg->batch samples per model and step; loss_log holds the mean
 * over all models' samples.  ws: ndgi_hybrid_encode_fit_batch_workspace_size
 * bytes (the Adam moments of all models).  1 <= n_models <= 65535 (one row
 * of CTAs per model); NDGI_ERR_INVALID_ARG otherwise.
 */
size_t ndgi_hybrid_encode_fit_batch_workspace_size(const ndgi_hybrid_fit_params *params, int32_t n_models,
                                                   const ndgi_fit_config *cfg);
ndgi_status ndgi_hybrid_encode_fit_batch(const ndgi_hybrid_fit_params *params, int32_t n_models,
                                         const uint16_t *targets, int32_t t_count, const float *key_t,
                                         const ndgi_fit_config *cfg, int32_t step_offset, void *ws, size_t ws_bytes,
                                         double *loss_log, void *stream);

/* ======================================================================
 * Quality metrics (supplement S4.2)
 * ====================================================================== */

/*
 * Tiled, mask-aware PSNR and SSIM of n_maps decoded lightmaps against their
 * references: pred, ref [n_maps][h][w][channels] FP32 (device); mask
 * [n_maps][h][w] bytes (device; non-zero = valid texel) or NULL (all valid).
 * Each map is cut into tile x tile tiles (partial tiles at the right and
 * bottom keep their own size).  Per tile, over its valid texels: L = max -
 * min of the reference (all channels); PSNR = 10 log10(L^2 / MSE); SSIM =
 * Wang et al.'s index with an 11 x 11 Gaussian window (sigma 1.5, weights
 * normalised, biased covariances), C1 = (0.01 L)^2, C2 = (0.03 L)^2, at every
 * valid texel whose window lies inside the tile, averaged over those texels
 * and the channels.  psnr, ssim: [n_maps][ceil(h/tile)][ceil(w/tile)] FP64
 * (device); a tile with no valid texel (for SSIM: no valid centre) gets NaN,
 * a tile with zero error PSNR = +inf.  channels 1..4.  pred and ref must be
 * 4-byte and psnr, ssim 8-byte aligned (NDGI_ERR_INVALID_ARG otherwise).
 */
ndgi_status ndgi_tile_metrics(const float *pred, const float *ref, const uint8_t *mask, int32_t n_maps, int32_t h,
                              int32_t w, int32_t channels, int32_t tile, double *psnr, double *ssim, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* NDGI_H_ */
