// Plain FP32 CUDA-core decode: one thread per query or page texel.
//
// This is the baseline the tensor-core decode is measured against, and the
// accurate (FP32, <= 1e-5 of range) decode.  Per query: texel-centre taps on
// the BC4 planes (block lines [by][bx][cs][8] read as 16-byte pairs of
// planes), exact integer palette decode, FP32 bilinear blend and temporal
// lerp, then the MLP from shared memory (W2 stored transposed so each output
// unit reads one contiguous row; layers 2 and 3 are fused so the second
// hidden vector never needs registers of its own).
#include "ndgi_internal.h"
#include "bc4.cuh"
#include "gather.cuh"

namespace ndgi {

constexpr int kSimtThreads = 128;

// Shared-memory image of the MLP: w1 [CIN][H], b1 [H], w2t [H][H] (out-major),
// b2 [H], w3 [H][4] (padded), b3 [4].
template <int CIN, int H>
struct SimtMlp {
  static constexpr int kW1 = 0;
  static constexpr int kB1 = kW1 + CIN * H;
  static constexpr int kW2t = kB1 + H;
  static constexpr int kB2 = kW2t + H * H;
  static constexpr int kW3 = kB2 + H;
  static constexpr int kB3 = kW3 + H * 4;
  static constexpr int kFloats = kB3 + 4;
  static constexpr size_t kBytes = kFloats * sizeof(float);

  static __device__ void load(float* s, const DevModel& m) {
    for (int i = threadIdx.x; i < CIN * H; i += blockDim.x) s[kW1 + i] = m.w1[i];
    for (int i = threadIdx.x; i < H; i += blockDim.x) {
      s[kB1 + i] = m.b1[i];
      s[kB2 + i] = m.b2[i];
    }
    for (int i = threadIdx.x; i < H * H; i += blockDim.x) {
      const int in = i / H, out = i % H;
      s[kW2t + out * H + in] = m.w2[i];
    }
    for (int i = threadIdx.x; i < H * 4; i += blockDim.x) {
      const int r = i / 4, c = i % 4;
      s[kW3 + i] = c < 3 ? m.w3[r * 3 + c] : 0.0f;
    }
    if (threadIdx.x < 4) s[kB3 + threadIdx.x] = threadIdx.x < 3 ? m.b3[threadIdx.x] : 0.0f;
  }

  static __device__ __forceinline__ void eval(const float* s, const float (&x)[CIN], float& y0, float& y1,
                                              float& y2) {
    float h1[H];
#pragma unroll
    for (int o = 0; o < H; ++o) h1[o] = s[kB1 + o];
#pragma unroll
    for (int i = 0; i < CIN; ++i) {
      const float4* row = reinterpret_cast<const float4*>(s + kW1 + i * H);
#pragma unroll
      for (int o4 = 0; o4 < H / 4; ++o4) {
        const float4 w = row[o4];
        h1[4 * o4 + 0] = fmaf(x[i], w.x, h1[4 * o4 + 0]);
        h1[4 * o4 + 1] = fmaf(x[i], w.y, h1[4 * o4 + 1]);
        h1[4 * o4 + 2] = fmaf(x[i], w.z, h1[4 * o4 + 2]);
        h1[4 * o4 + 3] = fmaf(x[i], w.w, h1[4 * o4 + 3]);
      }
    }
#pragma unroll
    for (int o = 0; o < H; ++o) h1[o] = fmaxf(h1[o], 0.0f);
    const float4 b3 = *reinterpret_cast<const float4*>(s + kB3);
    y0 = b3.x;
    y1 = b3.y;
    y2 = b3.z;
#pragma unroll 4
    for (int o = 0; o < H; ++o) {
      const float4* row = reinterpret_cast<const float4*>(s + kW2t + o * H);
      float z0 = s[kB2 + o], z1 = 0.0f;
#pragma unroll
      for (int i4 = 0; i4 < H / 4; i4 += 2) {
        const float4 a = row[i4];
        z0 = fmaf(h1[4 * i4 + 0], a.x, z0);
        z0 = fmaf(h1[4 * i4 + 1], a.y, z0);
        z0 = fmaf(h1[4 * i4 + 2], a.z, z0);
        z0 = fmaf(h1[4 * i4 + 3], a.w, z0);
        if (i4 + 1 < H / 4) {
          const float4 b = row[i4 + 1];
          z1 = fmaf(h1[4 * i4 + 4], b.x, z1);
          z1 = fmaf(h1[4 * i4 + 5], b.y, z1);
          z1 = fmaf(h1[4 * i4 + 6], b.z, z1);
          z1 = fmaf(h1[4 * i4 + 7], b.w, z1);
        }
      }
      const float h2 = fmaxf(z0 + z1, 0.0f);
      const float4 w3 = *reinterpret_cast<const float4*>(s + kW3 + o * 4);
      y0 = fmaf(h2, w3.x, y0);
      y1 = fmaf(h2, w3.y, y1);
      y2 = fmaf(h2, w3.z, y2);
    }
  }
};

template <int CS, int CT, int H>
__global__ void __launch_bounds__(kSimtThreads) k_points_f32(DevModel m, const float* __restrict__ uvt, int64_t n,
                                                             float* __restrict__ rgb) {
  using Mlp = SimtMlp<CS + CT, H>;
  extern __shared__ __align__(16) float s_mlp[];
  __shared__ uint2 lut[16];
  init_p35_lut(lut, threadIdx.x);
  Mlp::load(s_mlp, m);
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float u = uvt[3 * i], v = uvt[3 * i + 1], t = uvt[3 * i + 2];
    float x[CS + CT];
    gather_f32<CS, CT>(m, u, v, t, x, nullptr, lut);
    float y0, y1, y2;
    Mlp::eval(s_mlp, x, y0, y1, y2);
    rgb[3 * i] = y0;
    rgb[3 * i + 1] = y1;
    rgb[3 * i + 2] = y2;
  }
}

template <int CS, int CT>
__global__ void __launch_bounds__(kSimtThreads) k_debug_features(DevModel m, const float* __restrict__ uvt, int64_t n,
                                                                 float* __restrict__ xo, int32_t* __restrict__ p35) {
  __shared__ uint2 lut[16];
  init_p35_lut(lut, threadIdx.x);
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float x[CS + CT];
    gather_f32<CS, CT>(m, uvt[3 * i], uvt[3 * i + 1], uvt[3 * i + 2], x, p35 ? p35 + i * 4 * CS : nullptr, lut);
#pragma unroll
    for (int c = 0; c < CS + CT; ++c) xo[i * (CS + CT) + c] = x[c];
  }
}

// Page decode, FP32: work item = (request, chunk of 128 texels); one thread per texel.
// The request count is read on the device, so the launch can be replayed from a graph.
template <int CS, int CT, int H>
__global__ void __launch_bounds__(kSimtThreads) k_pages_f32(PagesCtx c, const ndgi_page_req* __restrict__ reqs,
                                                            const int32_t* __restrict__ n_dev) {
  using Mlp = SimtMlp<CS + CT, H>;
  extern __shared__ __align__(16) float s_mlp[];
  __shared__ uint2 lut[16];
  init_p35_lut(lut, threadIdx.x);
  __syncthreads();
  int n = *n_dev;
  if (n > c.max_reqs || n < 0) {   // reject the whole frame: the request buffer may be shorter
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(c.error_word, 1);
    n = 0;
  }
  const int64_t items = (int64_t)n * 128;
  int loaded = -1;
  for (int64_t w = blockIdx.x; w < items; w += gridDim.x) {
    const ndgi_page_req r = reqs[w >> 7];
    const int chunk = (int)(w & 127);
    const bool valid = r.model >= 0 && r.model < c.n_models && r.w >= 1 && r.w <= 128 && r.h >= 1 && r.h <= 128;
    if (!valid) {
      if (chunk == 0 && threadIdx.x == 0) atomicOr(c.error_word, 2);
      continue;
    }
    const DevModel& m = c.models[r.model];
    const bool inside = r.x0 >= 0 && r.y0 >= 0 && (int64_t)r.x0 + r.w <= m.lm_w && (int64_t)r.y0 + r.h <= m.lm_h &&
                        r.dst_x >= 0 && r.dst_y >= 0 && (int64_t)r.dst_x + r.w <= c.phys_w &&
                        (int64_t)r.dst_y + r.h <= c.phys_h;
    if (!inside) {
      if (chunk == 0 && threadIdx.x == 0) atomicOr(c.error_word, 4);
      continue;
    }
    if (chunk * 128 >= r.w * r.h) continue;
    if (loaded != r.model) {   // block-uniform: reload the MLP when the model changes
      __syncthreads();
      Mlp::load(s_mlp, m);
      __syncthreads();
      loaded = r.model;
    }
    const int k = chunk * 128 + threadIdx.x;
    if (k >= r.w * r.h) continue;
    const int i = k % r.w, j = k / r.w;
    // texel centre of lightmap texel (x0+i, y0+j) in feature coordinates is
    // (x0+i+0.5)*sx - 0.5; pass it as a normalised coordinate u = (x0+i+0.5)/lm_w.
    const float u = ((float)(r.x0 + i) + 0.5f) / (float)m.lm_w;
    const float v = ((float)(r.y0 + j) + 0.5f) / (float)m.lm_h;
    float x[CS + CT];
    gather_f32<CS, CT>(m, u, v, r.t, x, nullptr, lut);
    float y0, y1, y2;
    Mlp::eval(s_mlp, x, y0, y1, y2);
    const int64_t o = (int64_t)(r.dst_y + j) * c.phys_w + (r.dst_x + i);
    if (c.out_format == NDGI_RGBA32F) {
      reinterpret_cast<float4*>(c.phys)[o] = make_float4(y0, y1, y2, 1.0f);
    } else {
      __half2 a = __floats2half2_rn(y0, y1), b = __floats2half2_rn(y2, 1.0f);
      uint2 p;
      p.x = *reinterpret_cast<uint32_t*>(&a);
      p.y = *reinterpret_cast<uint32_t*>(&b);
      reinterpret_cast<uint2*>(c.phys)[o] = p;
    }
  }
}

// ---------------------------------------------------------------------------
// Dispatch over the built (cs, ct, hidden) shapes.
// FP8 calibration: the maxima of |layer-1 input|, relu(z1) and relu(z2) of the
// FP32 decode over the given queries (act_max must hold zeros on entry; the
// values are non-negative, so their float bits order like the floats).
template <int CS, int CT, int H>
__global__ void __launch_bounds__(kSimtThreads) k_fp8_calibrate(DevModel m, const float* __restrict__ uvt, int64_t n,
                                                                float* __restrict__ act_max) {
  using Mlp = SimtMlp<CS + CT, H>;
  extern __shared__ __align__(16) float s_mlp[];
  __shared__ uint2 lut[16];
  init_p35_lut(lut, threadIdx.x);
  Mlp::load(s_mlp, m);
  __syncthreads();
  float m1 = 0.0f, m2 = 0.0f, m3 = 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float x[CS + CT];
    gather_f32<CS, CT>(m, uvt[3 * i], uvt[3 * i + 1], uvt[3 * i + 2], x, nullptr, lut);
    float h1[H];
#pragma unroll
    for (int o = 0; o < H; ++o) h1[o] = s_mlp[Mlp::kB1 + o];
#pragma unroll
    for (int k = 0; k < CS + CT; ++k) {
      m1 = fmaxf(m1, fabsf(x[k]));
#pragma unroll
      for (int o = 0; o < H; ++o) h1[o] = fmaf(x[k], s_mlp[Mlp::kW1 + k * H + o], h1[o]);
    }
#pragma unroll
    for (int o = 0; o < H; ++o) {
      h1[o] = fmaxf(h1[o], 0.0f);
      m2 = fmaxf(m2, h1[o]);
    }
    for (int o = 0; o < H; ++o) {
      float z = s_mlp[Mlp::kB2 + o];
#pragma unroll
      for (int k = 0; k < H; ++k) z = fmaf(h1[k], s_mlp[Mlp::kW2t + o * H + k], z);
      m3 = fmaxf(m3, z);
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, off));
    m2 = fmaxf(m2, __shfl_xor_sync(0xffffffffu, m2, off));
    m3 = fmaxf(m3, __shfl_xor_sync(0xffffffffu, m3, off));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(reinterpret_cast<unsigned int*>(act_max), __float_as_uint(m1));
    atomicMax(reinterpret_cast<unsigned int*>(act_max) + 1, __float_as_uint(m2));
    atomicMax(reinterpret_cast<unsigned int*>(act_max) + 2, __float_as_uint(m3));
  }
}

// ---------------------------------------------------------------------------
#define NDGI_SIMT_SHAPES(X) \
  X(4, 4, 16)               \
  X(8, 8, 16)               \
  X(8, 8, 32)               \
  X(16, 8, 16)              \
  X(16, 8, 32)              \
  X(16, 8, 64)              \
  X(16, 16, 64)

bool simt_supported(int cs, int ct, int hidden) {
#define X(A, B, C) if (cs == A && ct == B && hidden == C) return true;
  NDGI_SIMT_SHAPES(X)
#undef X
  return false;
}

static int grid_for(int64_t work, int per_block, int blocks_per_sm) {
  const int64_t need = (work + per_block - 1) / per_block;
  const int64_t cap = (int64_t)num_sms() * blocks_per_sm;
  return (int)(need < cap ? (need > 0 ? need : 1) : cap);
}

cudaError_t launch_points_f32(const DevModel& m, const float* uvt, int64_t n, float* rgb, cudaStream_t s) {
  const int grid = grid_for(n, kSimtThreads, 16);
#define X(A, B, C)                                                                              \
  if (m.cs == A && m.ct == B && m.hidden == C) {                                                \
    constexpr size_t smem = SimtMlp<A + B, C>::kBytes;                                          \
    if (smem > 48 * 1024) {                                                                     \
      cudaError_t e = cudaFuncSetAttribute(k_points_f32<A, B, C>,                               \
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem);  \
      if (e != cudaSuccess) return e;                                                           \
    }                                                                                           \
    k_points_f32<A, B, C><<<grid, kSimtThreads, smem, s>>>(m, uvt, n, rgb);                     \
    return cudaGetLastError();                                                                  \
  }
  NDGI_SIMT_SHAPES(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t launch_fp8_calibrate(const DevModel& m, const float* uvt, int64_t n, float* act_max, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(act_max, 0, 3 * sizeof(float), s);
  if (e != cudaSuccess) return e;
  const int grid = grid_for(n, kSimtThreads, 8);
#define X(A, B, C)                                                                              \
  if (m.cs == A && m.ct == B && m.hidden == C) {                                                \
    constexpr size_t smem = SimtMlp<A + B, C>::kBytes;                                          \
    if (smem > 48 * 1024) {                                                                     \
      e = cudaFuncSetAttribute(k_fp8_calibrate<A, B, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); \
      if (e != cudaSuccess) return e;                                                           \
    }                                                                                           \
    k_fp8_calibrate<A, B, C><<<grid, kSimtThreads, smem, s>>>(m, uvt, n, act_max);              \
    return cudaGetLastError();                                                                  \
  }
  NDGI_SIMT_SHAPES(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t launch_debug_features(const DevModel& m, const float* uvt, int64_t n, float* x, int32_t* p35,
                                  cudaStream_t s) {
  const int grid = grid_for(n, kSimtThreads, 16);
#define X(A, B, C)                                                            \
  if (m.cs == A && m.ct == B) {                                               \
    k_debug_features<A, B><<<grid, kSimtThreads, 0, s>>>(m, uvt, n, x, p35);  \
    return cudaGetLastError();                                                \
  }
  NDGI_SIMT_SHAPES(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t launch_pages_f32(const PagesCtx& c, int cs, int ct, int hidden, const ndgi_page_req* reqs,
                             const int32_t* n_dev, int grid, cudaStream_t s) {
#define X(A, B, C)                                                                              \
  if (cs == A && ct == B && hidden == C) {                                                      \
    constexpr size_t smem = SimtMlp<A + B, C>::kBytes;                                          \
    if (smem > 48 * 1024) {                                                                     \
      cudaError_t e = cudaFuncSetAttribute(k_pages_f32<A, B, C>,                                \
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem);  \
      if (e != cudaSuccess) return e;                                                           \
    }                                                                                           \
    k_pages_f32<A, B, C><<<grid, kSimtThreads, smem, s>>>(c, reqs, n_dev);                      \
    return cudaGetLastError();                                                                  \
  }
  NDGI_SIMT_SHAPES(X)
#undef X
  return cudaErrorInvalidValue;
}

}  // namespace ndgi
