// Point decode from host buffers: ndgi_decode_points_host and its pipe.
//
// A serving caller holds its queries and wants its results in host memory.
// Copying the whole batch in, decoding and copying the results out in turn
// leaves the copy engines idle during the decode and the SMs idle during the
// copies.  The pipe splits the batch into chunks and runs three stages at
// once on three streams: the copy of chunk k + 1 to the device (copy-in
// stream), the decode of chunk k (the caller's stream), the copy of chunk
// k - 1's results to the host (copy-out stream).  Each of the three staging
// buffers holds one chunk of queries and results; events order the stages
// of a buffer and free it for chunk k + 3.  The first and last chunks of a
// call are smaller (see piece) so that the stages start and end together.
#include <cstdint>

#include "ndgi_internal.h"
#include "tc_decode.h"

namespace {
constexpr int kBufs = 3;

size_t part_bytes(int64_t chunk) { return ((size_t)chunk * 12 + 255) / 256 * 256; }

// Length of piece k of a call, given the queries still to go: the pieces
// ramp up (c/8, c/4, c/2, then c) and, over the last 2c queries, halve down
// to c/8, so the pipeline fills and drains on small pieces.
int64_t piece(int64_t k, int64_t remaining, int64_t c) {
  const int64_t lo = (c >> 3) > 0 ? (c >> 3) : 1;
  int64_t len = k < 3 ? (c >> (3 - k)) : c;
  if (len < lo) len = lo;
  if (remaining <= 2 * c && remaining > lo) {
    const int64_t half = (remaining + 1) / 2;
    len = len < half ? len : (half > lo ? half : lo);
  }
  return len < remaining ? len : remaining;
}
}  // namespace

struct ndgi_host_pipe {
  int device;
  int64_t chunk;
  unsigned char* staging;   // kBufs x (queries, results), caller-owned
  cudaStream_t in, out;     // copy-in and copy-out streams
  cudaEvent_t start, fin;   // call boundaries
  cudaEvent_t loaded[kBufs], decoded[kBufs], stored[kBufs];
  bool used;                // a previous call's work may still be in flight
};

using namespace ndgi;

static void destroy_pipe(ndgi_host_pipe* p) {
  if (p->in) cudaStreamSynchronize(p->in);
  if (p->out) cudaStreamSynchronize(p->out);
  cudaEvent_t* evs[] = {&p->start, &p->fin};
  for (cudaEvent_t* e : evs)
    if (*e) cudaEventDestroy(*e);
  for (int b = 0; b < kBufs; ++b) {
    if (p->loaded[b]) cudaEventDestroy(p->loaded[b]);
    if (p->decoded[b]) cudaEventDestroy(p->decoded[b]);
    if (p->stored[b]) cudaEventDestroy(p->stored[b]);
  }
  if (p->in) cudaStreamDestroy(p->in);
  if (p->out) cudaStreamDestroy(p->out);
  delete p;
}

extern "C" {

size_t ndgi_host_pipe_staging_size(int64_t chunk) {
  if (chunk < 1) return 0;
  return (size_t)kBufs * 2 * part_bytes(chunk);
}

ndgi_status ndgi_host_pipe_create(int64_t chunk, void* staging, size_t staging_bytes, ndgi_host_pipe** pipe) {
  if (!pipe) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_host_pipe_create: pipe is NULL");
  *pipe = nullptr;
  if (chunk < 1 || chunk > ((int64_t)1 << 40))
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_host_pipe_create: chunk must be >= 1");
  if (!staging || ((uintptr_t)staging % 256) != 0 || staging_bytes < ndgi_host_pipe_staging_size(chunk))
    return set_error(NDGI_ERR_INVALID_ARG,
                     "ndgi_host_pipe_create: staging must be 256-byte aligned device memory of >= %zu bytes",
                     ndgi_host_pipe_staging_size(chunk));
  ndgi_host_pipe* p = new ndgi_host_pipe{};
  p->chunk = chunk;
  p->staging = static_cast<unsigned char*>(staging);
  cudaError_t e = cudaGetDevice(&p->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->out, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->start, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->fin, cudaEventDisableTiming);
  for (int b = 0; b < kBufs && e == cudaSuccess; ++b) {
    e = cudaEventCreateWithFlags(&p->loaded[b], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->decoded[b], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->stored[b], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    destroy_pipe(p);
    return cuda_status(e, "ndgi_host_pipe_create");
  }
  *pipe = p;
  return NDGI_OK;
}

ndgi_status ndgi_decode_points_host(ndgi_host_pipe* p, const ndgi_model_desc* model, ndgi_precision precision,
                                    const void* ws, const float* uvt_host, int64_t n, float* rgb_host,
                                    void* stream) {
  if (!p) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_decode_points_host: pipe is NULL");
  if (n < 0) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_decode_points_host: n < 0");
  if (n == 0) return NDGI_OK;
  if (!uvt_host || !rgb_host) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_decode_points_host: host buffer is NULL");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device)
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_decode_points_host: the pipe belongs to device %d", p->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t part = part_bytes(p->chunk);
  // On a failure after work was enqueued, the call still closes with the
  // fin event, so the next call's first copy waits for what did go out.
  auto fail = [&](ndgi_status st) {
    if (cudaEventRecord(p->fin, p->out) == cudaSuccess) p->used = true;
    return st;
  };
#define NDGI_TRY(call)                                                           \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess) return fail(cuda_status(e_, "ndgi_decode_points_host")); \
  } while (0)
  // everything enqueued before this call on `stream`, and the previous
  // call's last copy, comes first
  NDGI_TRY(cudaEventRecord(p->start, s));
  NDGI_TRY(cudaStreamWaitEvent(p->in, p->start, 0));
  NDGI_TRY(cudaStreamWaitEvent(p->out, p->start, 0));
  if (p->used) NDGI_TRY(cudaStreamWaitEvent(p->in, p->fin, 0));
  // the decoded-texel cache (when the whole call qualifies) is built once, by
  // the first chunk's decode, and reused by the others on the same stream
  const bool cached = (precision == NDGI_FP16 || precision == NDGI_BF16) && model &&
                      tc_supported(model->cs, model->ct, model->hidden) &&
                      tc_points_cache_path(to_dev(*model), n, kPointsAuto);
  int64_t off = 0;
  for (int64_t k = 0; off < n; ++k) {
    const int b = (int)(k % kBufs);
    const int64_t len = piece(k, n - off, p->chunk);
    float* q_dev = reinterpret_cast<float*>(p->staging + (size_t)b * 2 * part);
    float* r_dev = reinterpret_cast<float*>(p->staging + (size_t)b * 2 * part + part);
    // buffer b is free once chunk k - 3's results have left it (its decode came before)
    if (k >= kBufs) NDGI_TRY(cudaStreamWaitEvent(p->in, p->stored[b], 0));
    NDGI_TRY(cudaMemcpyAsync(q_dev, uvt_host + 3 * off, (size_t)len * 12, cudaMemcpyHostToDevice, p->in));
    NDGI_TRY(cudaEventRecord(p->loaded[b], p->in));
    NDGI_TRY(cudaStreamWaitEvent(s, p->loaded[b], 0));
    const int mode = cached ? (k == 0 ? kPointsBuild : kPointsReuse) : kPointsDirect;
    const ndgi_status st = decode_points_mode(model, precision, ws, q_dev, len, r_dev, stream, mode);
    if (st != NDGI_OK) return fail(st);
    NDGI_TRY(cudaEventRecord(p->decoded[b], s));
    NDGI_TRY(cudaStreamWaitEvent(p->out, p->decoded[b], 0));
    NDGI_TRY(cudaMemcpyAsync(rgb_host + 3 * off, r_dev, (size_t)len * 12, cudaMemcpyDeviceToHost, p->out));
    NDGI_TRY(cudaEventRecord(p->stored[b], p->out));
    off += len;
  }
  // `stream` reaches this point only after the last result is in host memory
  NDGI_TRY(cudaEventRecord(p->fin, p->out));
  NDGI_TRY(cudaStreamWaitEvent(s, p->fin, 0));
  p->used = true;
#undef NDGI_TRY
  return NDGI_OK;
}

ndgi_status ndgi_host_pipe_destroy(ndgi_host_pipe* p) {
  if (!p) return NDGI_OK;
  destroy_pipe(p);
  return NDGI_OK;
}

}  // extern "C"
