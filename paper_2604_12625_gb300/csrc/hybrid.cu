// Hybrid feature map decoder: the paper's full decoder (Sec. 3.3, Eq. 4-5;
// Sec. 4).  Per query (u, v, t):
//   V_uvt  trilinear sample of F3D (4 BC4 planes per t-slice): the two
//          slices around t, each bilinear at (u, v), then linear in t;
//   V_uv   bilinear sample of F_uv (4 BC4 planes);
//   V_ut   bilinear sample of the UNORM8 plane F_ut at (u, t), 2 channels;
//   V_vt   bilinear sample of F_vt at (v, t), 2 channels;
//   gamma  [sin pi t, cos pi t, sin 2 pi t, cos 2 pi t];
// x = [V_uvt, V_uv, V_ut, V_vt, gamma] (16 values) -> GELU(x W1 + b1) ->
// GELU(. W2 + b2) -> . W3 + b3.
//
// Two decodes share the FP32 feature gather:
//   - CUDA cores, FP32 throughout (k_hybrid_points_f32 / k_hybrid_pages_f32);
//   - tensor cores (k_hybrid_tc): the 16 features and the ones column that
//     carries b1 are one K = 32 FP16/BF16 row of tensor memory per query, and
//     the three layers run on the per-lane engine of tc_engine.cuh with the
//     GELU epilogue; the next tile's gather overlaps this tile's layer 2, and
//     layer 3 goes out with the next tile's layer 1 (two MMA round trips per
//     tile).  For pages each request's model image is staged in shared memory
//     once per request and the CTA's four lanes split the request's tiles.
#include <vector>

#include "bc7.cuh"
#include "hybrid.h"
#include "tc_engine.cuh"

namespace ndgi {

// GELU(x) = x Phi(x) = x (1 + erf(x / sqrt 2)) / 2, the exact form, with the
// CUDA math library's erff (the FP32 decodes).
__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }

// The same for the tensor-core epilogues, whose results are rounded to
// FP16/BF16 right after: Phi from the complementary-error-function form of
// Abramowitz & Stegun 7.1.28, erf(z) = 1 - (1 + a1 z + ... + a6 z^6)^-16 for
// z >= 0 with |error| <= 3e-7.  Then 1 - Phi(|x|) = erfc(z) / 2 =
// (2^(1/16) P(z))^-16, z = |x| / sqrt 2, so the 2^(1/16) goes into the
// coefficients and the rest is one approximate reciprocal and four squarings;
// GELU(x) = x - x erfc/2 for x >= 0 and x erfc/2 below.
__device__ __forceinline__ float gelu_fast(float x) {
  constexpr float k = 1.0442737824274138f;   // 2^(1/16)
  const float z = fabsf(x) * 0.70710678118654752f;
  float p = fmaf(k * 0.0000430638f, z, k * 0.0002765672f);
  p = fmaf(p, z, k * 0.0001520143f);
  p = fmaf(p, z, k * 0.0092705272f);
  p = fmaf(p, z, k * 0.0422820123f);
  p = fmaf(p, z, k * 0.0705230784f);
  p = fmaf(p, z, k);
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(p));
  r *= r;
  r *= r;
  r *= r;
  r *= r;   // erfc(z) / 2
  return x >= 0.0f ? fmaf(-x, r, x) : x * r;
}

// ---------------------------------------------------------------------------
// Feature gather (FP32)
// ---------------------------------------------------------------------------

// Bilinear sample of four BC4 planes [h/4][bw][4][8] at taps (x0|x1, y0|y1):
// a tap's four planes are one 32-byte block line (two 16-byte loads).
__device__ __forceinline__ void bc4x4_bilinear(const uint8_t* __restrict__ bc4, int bw, int x0, int x1, int y0,
                                               int y1, float fx, float fy, const uint2* lut, float* out) {
  const int tx[4] = {x0, x1, x0, x1}, ty[4] = {y0, y0, y1, y1};
  float f[4][4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint4* line = reinterpret_cast<const uint4*>(bc4 + ((size_t)(ty[q] >> 2) * bw + (tx[q] >> 2)) * 32);
    const uint4 a = __ldg(line), b = __ldg(line + 1);
    const uint32_t shift = 16u + 3u * (uint32_t)(((ty[q] & 3) << 2) | (tx[q] & 3));
    f[q][0] = p35_value(bc4_p35_lut(a.x, a.y, shift, lut));
    f[q][1] = p35_value(bc4_p35_lut(a.z, a.w, shift, lut));
    f[q][2] = p35_value(bc4_p35_lut(b.x, b.y, shift, lut));
    f[q][3] = p35_value(bc4_p35_lut(b.z, b.w, shift, lut));
  }
  const float gx = 1.0f - fx, gy = 1.0f - fy;
#pragma unroll
  for (int c = 0; c < 4; ++c) out[c] = gy * (gx * f[0][c] + fx * f[1][c]) + fy * (gx * f[2][c] + fx * f[3][c]);
}

// Bilinear sample of a BC7 map [h/4][bw][16] at taps (x0|x1, y0|y1): each tap
// one texel decode of its block, value byte / 255.
__device__ __forceinline__ void u8x4_unpack(uint32_t v, float* out) {
#pragma unroll
  for (int c = 0; c < 4; ++c) out[c] = (float)((v >> (8 * c)) & 255u) * (1.0f / 255.0f);
}

__device__ __forceinline__ void bc7_bilinear(const uint8_t* __restrict__ blocks, int bw, int x0, int x1, int y0,
                                             int y1, float fx, float fy, float* out) {
  const int tx[4] = {x0, x1, x0, x1}, ty[4] = {y0, y0, y1, y1};
  float f[4][4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint4 b = __ldg(reinterpret_cast<const uint4*>(blocks + ((size_t)(ty[q] >> 2) * bw + (tx[q] >> 2)) * 16));
    u8x4_unpack(bc7_texel(b, ((ty[q] & 3) << 2) | (tx[q] & 3)), f[q]);
  }
  const float gx = 1.0f - fx, gy = 1.0f - fy;
#pragma unroll
  for (int c = 0; c < 4; ++c) out[c] = gy * (gx * f[0][c] + fx * f[1][c]) + fy * (gx * f[2][c] + fx * f[3][c]);
}

// A four-channel map (F_uv or an F3D slice) in the model's block format.
__device__ __forceinline__ void map4_bilinear(const DevHybrid& m, const uint8_t* __restrict__ base, int bw, int x0,
                                              int x1, int y0, int y1, float fx, float fy, const uint2* lut,
                                              float* out) {
  if (m.bc7) bc7_bilinear(base, bw, x0, x1, y0, y1, fx, fy, out);
  else bc4x4_bilinear(base, bw, x0, x1, y0, y1, fx, fy, lut, out);
}

__device__ __forceinline__ size_t vol_slice_bytes(const DevHybrid& m) {
  return (size_t)(m.vol_h / 4) * (size_t)(m.vol_w / 4) * (m.bc7 ? 16 : 32);
}

// Bilinear sample of a two-channel UNORM8 plane [ny][nx][2] (one 16-bit load per tap).
__device__ __forceinline__ void u8x2_bilinear(const uint8_t* __restrict__ p, int nx, int x0, int x1, int y0, int y1,
                                              float fx, float fy, float* out) {
  const unsigned short* w = reinterpret_cast<const unsigned short*>(p);
  const uint32_t q00 = __ldg(w + (size_t)y0 * nx + x0), q10 = __ldg(w + (size_t)y0 * nx + x1);
  const uint32_t q01 = __ldg(w + (size_t)y1 * nx + x0), q11 = __ldg(w + (size_t)y1 * nx + x1);
  const float gx = 1.0f - fx, gy = 1.0f - fy, s = 1.0f / 255.0f;
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const int sh = 8 * c;
    const float f00 = (float)((q00 >> sh) & 255u) * s, f10 = (float)((q10 >> sh) & 255u) * s;
    const float f01 = (float)((q01 >> sh) & 255u) * s, f11 = (float)((q11 >> sh) & 255u) * s;
    out[c] = gy * (gx * f00 + fx * f10) + fy * (gx * f01 + fx * f11);
  }
}

// The decoder input x[16] at (u, v, t) (Eq. 4); lut: init_p35_lut's table.
__device__ __forceinline__ void hybrid_features(const DevHybrid& m, float u, float v, float t, float (&x)[16],
                                                const uint2* lut) {
  const int mode = m.address_mode;
  int x0, x1, y0, y1, z0, z1;
  float fx, fy, fz;
  axis_setup(u, m.vol_w, mode, x0, x1, fx);
  axis_setup(v, m.vol_h, mode, y0, y1, fy);
  axis_setup(t, m.vol_t, 0, z0, z1, fz);
  const size_t slice = vol_slice_bytes(m);
  float a[4], b[4];
  map4_bilinear(m, m.vol + (size_t)z0 * slice, m.vol_w / 4, x0, x1, y0, y1, fx, fy, lut, a);
  map4_bilinear(m, m.vol + (size_t)z1 * slice, m.vol_w / 4, x0, x1, y0, y1, fx, fy, lut, b);
  const float gz = 1.0f - fz;
#pragma unroll
  for (int c = 0; c < 4; ++c) x[c] = gz * a[c] + fz * b[c];
  axis_setup(u, m.uv_w, mode, x0, x1, fx);
  axis_setup(v, m.uv_h, mode, y0, y1, fy);
  map4_bilinear(m, m.uv, m.uv_w / 4, x0, x1, y0, y1, fx, fy, lut, x + 4);
  axis_setup(u, m.ut_w, mode, x0, x1, fx);
  axis_setup(t, m.ut_t, 0, y0, y1, fy);
  u8x2_bilinear(m.ut, m.ut_w, x0, x1, y0, y1, fx, fy, x + 8);
  axis_setup(v, m.vt_h, mode, x0, x1, fx);
  axis_setup(t, m.vt_t, 0, y0, y1, fy);
  u8x2_bilinear(m.vt, m.vt_h, x0, x1, y0, y1, fx, fy, x + 10);
  sincospif(t, &x[12], &x[13]);
  sincospif(2.0f * t, &x[14], &x[15]);
}

// ---------------------------------------------------------------------------
// FP32 CUDA-core decode
// ---------------------------------------------------------------------------

// Shared-memory copy of one model's MLP: w1 [16][H], b1, w2 [H][H], b2, w3 [H][3], b3.
template <int H>
struct HybridMlp32 {
  static constexpr int kW1 = 0, kB1 = 16 * H, kW2 = kB1 + H, kB2 = kW2 + H * H, kW3 = kB2 + H, kB3 = kW3 + 3 * H;
  static constexpr int kFloats = kB3 + 3;
};

template <int H>
__device__ __forceinline__ void load_mlp32(const DevHybrid& m, float* sw, int tid, int nt) {
  using M = HybridMlp32<H>;
  for (int i = tid; i < 16 * H; i += nt) sw[M::kW1 + i] = m.w1[i];
  for (int i = tid; i < H * H; i += nt) sw[M::kW2 + i] = m.w2[i];
  for (int i = tid; i < 3 * H; i += nt) sw[M::kW3 + i] = m.w3[i];
  for (int i = tid; i < H; i += nt) {
    sw[M::kB1 + i] = m.b1[i];
    sw[M::kB2 + i] = m.b2[i];
  }
  if (tid < 3) sw[M::kB3 + tid] = m.b3[tid];
}

// Layer 1 one hidden unit at a time, each folded into the layer-2
// accumulators as soon as it is known (H + 16 live values, not 2H).
template <int H>
__device__ __forceinline__ void mlp32(const float* sw, const float (&x)[16], float& r0, float& r1, float& r2) {
  using M = HybridMlp32<H>;
  float z2[H];
#pragma unroll
  for (int o = 0; o < H; ++o) z2[o] = sw[M::kB2 + o];
#pragma unroll 1
  for (int i = 0; i < H; ++i) {
    float z = sw[M::kB1 + i];
#pragma unroll
    for (int k = 0; k < 16; ++k) z = fmaf(x[k], sw[M::kW1 + k * H + i], z);
    const float h = gelu(z);
#pragma unroll
    for (int o = 0; o < H; ++o) z2[o] = fmaf(h, sw[M::kW2 + i * H + o], z2[o]);
  }
  r0 = sw[M::kB3 + 0];
  r1 = sw[M::kB3 + 1];
  r2 = sw[M::kB3 + 2];
#pragma unroll
  for (int o = 0; o < H; ++o) {
    const float h = gelu(z2[o]);
    r0 = fmaf(h, sw[M::kW3 + 3 * o + 0], r0);
    r1 = fmaf(h, sw[M::kW3 + 3 * o + 1], r1);
    r2 = fmaf(h, sw[M::kW3 + 3 * o + 2], r2);
  }
}

template <int H>
__global__ void __launch_bounds__(256) k_hybrid_points_f32(DevHybrid m, const float* __restrict__ uvt, int64_t n,
                                                           float* __restrict__ rgb) {
  __shared__ float sw[HybridMlp32<H>::kFloats];
  __shared__ uint2 lut[16];
  load_mlp32<H>(m, sw, threadIdx.x, blockDim.x);
  init_p35_lut(lut, threadIdx.x);
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float x[16];
    hybrid_features(m, __ldcs(uvt + 3 * i), __ldcs(uvt + 3 * i + 1), __ldcs(uvt + 3 * i + 2), x, lut);
    float r0, r1, r2;
    mlp32<H>(sw, x, r0, r1, r2);
    __stcs(rgb + 3 * i, r0);
    __stcs(rgb + 3 * i + 1, r1);
    __stcs(rgb + 3 * i + 2, r2);
  }
}

// A request is decoded only if its model index and both rectangles are valid
// (the destination including the border b on every side, b <= w, h).
__device__ __forceinline__ bool hybrid_req_ok(const ndgi_page_req& r, const DevHybrid* models, int n_models,
                                              int64_t phys_w, int64_t phys_h, int b) {
  if (r.model < 0 || r.model >= n_models) return false;
  const DevHybrid& m = models[r.model];
  return r.w >= 1 && r.w <= 128 && r.h >= 1 && r.h <= 128 && b <= r.w && b <= r.h && r.x0 >= 0 && r.y0 >= 0 &&
         r.x0 + r.w <= m.lm_w && r.y0 + r.h <= m.lm_h && r.dst_x - b >= 0 && r.dst_y - b >= 0 &&
         r.dst_x + r.w + b <= phys_w && r.dst_y + r.h + b <= phys_h;
}

// Mirrored tile border (supplement S3): texel i of a request's padded row or
// column, i in [0, n + 2b), is tile texel i - b reflected into [0, n) with
// the edge texel repeated (-1 -> 0, n -> n - 1).
__device__ __forceinline__ int border_mirror(int i, int n, int b) {
  const int k = i - b;
  return k < 0 ? -1 - k : (k >= n ? 2 * n - 1 - k : k);
}

__device__ __forceinline__ uint32_t unorm8(float y) {
  return (uint32_t)__float2int_rn(__saturatef(y) * 255.0f);
}

__device__ __forceinline__ void put_texel(void* phys, int fmt, int64_t o, float y0, float y1, float y2) {
  if (fmt == NDGI_RGBA32F) {
    __stcs(reinterpret_cast<float4*>(phys) + o, make_float4(y0, y1, y2, 1.0f));
  } else if (fmt == NDGI_RGBA8) {
    __stcs(reinterpret_cast<unsigned int*>(phys) + o, unorm8(y0) | (unorm8(y1) << 8) | (unorm8(y2) << 16) | 0xFF000000u);
  } else {
    __stcs(reinterpret_cast<uint2*>(phys) + o, make_uint2(pack2<false>(y0, y1), pack2<false>(y2, 1.0f)));
  }
}

// One request per CTA at a time (its model's MLP staged in shared memory).
template <int H>
__global__ void __launch_bounds__(256) k_hybrid_pages_f32(HybridPagesCtx c, const ndgi_page_req* __restrict__ reqs,
                                                          int n) {
  __shared__ float sw[HybridMlp32<H>::kFloats];
  __shared__ uint2 lut[16];
  init_p35_lut(lut, threadIdx.x);
  for (int ri = blockIdx.x; ri < n; ri += gridDim.x) {
    const ndgi_page_req r = reqs[ri];
    const bool ok = hybrid_req_ok(r, c.models, c.n_models, c.phys_w, c.phys_h, c.border);
    __syncthreads();   // the previous request's texels are done with sw
    if (!ok) {
      if (threadIdx.x == 0) atomicOr(c.error_word, 1);
      continue;
    }
    const DevHybrid m = c.models[r.model];
    load_mlp32<H>(m, sw, threadIdx.x, blockDim.x);
    __syncthreads();
    const int b = c.border, pw = r.w + 2 * b, ph = r.h + 2 * b;
    for (int i = threadIdx.x; i < pw * ph; i += blockDim.x) {
      const int ix = i % pw, iy = i / pw;
      const float u = ((float)(r.x0 + border_mirror(ix, r.w, b)) + 0.5f) / (float)m.lm_w;
      const float v = ((float)(r.y0 + border_mirror(iy, r.h, b)) + 0.5f) / (float)m.lm_h;
      float x[16];
      hybrid_features(m, u, v, r.t, x, lut);
      float y0, y1, y2;
      mlp32<H>(sw, x, y0, y1, y2);
      put_texel(c.phys, c.fmt, (int64_t)(r.dst_y - b + iy) * c.phys_w + (r.dst_x - b + ix), y0, y1, y2);
    }
  }
}

// ---------------------------------------------------------------------------
// Tensor-core decode (FP16/BF16 operands, FP32 accumulation)
// ---------------------------------------------------------------------------
// The model image is the point-decode layout of tc_engine.cuh with 16 inputs
// and no temporal line: B2 [H][H+16] (column H = b2), B3 [16][H+16] (rows 0..2
// = W3^T, column H = b3), B1 [H][32] (columns 0..15 = W1^T, column 16 = b1),
// then the error and debug words.
template <int H>
using HybridLayout = TcLayout<16, 0, H>;

// One column (u) or row (v) of a page request: its F3D and F_uv taps and
// fractions along that axis, and its V_ut (columns) or V_vt (rows).
struct HybAxis {
  int v0, v1;   // F3D taps
  float vf;
  int u0, u1;   // F_uv taps
  float uf;
  float p0, p1;
};
constexpr int kHybVolSide = 48;   // largest F3D footprint side staged in shared memory
constexpr int kHybBorderMax = 8;  // largest mirrored tile border
constexpr int kHybAxisMax = 128 + 2 * kHybBorderMax;   // entries of a per-axis table
constexpr int kHybUvSide = kHybAxisMax + 1;   // largest BC7 F_uv footprint side staged (decoded) in shared memory

template <int H>
struct HybridSmem {
  using L = HybridLayout<H>;
  static constexpr uint32_t kW = 0;                    // B2, B3
  static constexpr uint32_t kB1 = L::kShared;          // B1
  static constexpr uint32_t kPoints = kB1 + H * L::K1P * 2;   // end of the point kernel's part
  static constexpr uint32_t kCols = (kPoints + 15) / 16 * 16;  // pages: HybAxis [128] per column
  static constexpr uint32_t kRows = kCols + kHybAxisMax * sizeof(HybAxis);
  static constexpr uint32_t kVol = kRows + kHybAxisMax * sizeof(HybAxis);   // float4 [footprint] of F3D at t
  static constexpr uint32_t kUv = kVol + kHybVolSide * kHybVolSide * 16;     // RGBA8 [footprint] of a BC7 F_uv
  static constexpr uint32_t kPages = kUv;                                     // tables with BC4 maps only
  static constexpr uint32_t kPagesBc7 = kUv + kHybUvSide * kHybUvSide * 4;
};

constexpr int kHybLanes = 4;

template <int H, bool BF16>
__global__ void k_hybrid_prepare(DevHybrid m, unsigned char* __restrict__ ws) {
  using L = HybridLayout<H>;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
  for (int i = tid; i < H * L::K2; i += nt) {
    const int n = i / L::K2, k = i % L::K2;
    const float v = k < H ? m.w2[k * H + n] : (k == H ? m.b2[n] : 0.0f);
    *reinterpret_cast<uint16_t*>(ws + L::kB2 + kmajor_offset(n, k, L::K2)) = to_bits<BF16>(v);
  }
  for (int i = tid; i < L::N3 * L::K2; i += nt) {
    const int n = i / L::K2, k = i % L::K2;
    const float v = n >= 3 ? 0.0f : (k < H ? m.w3[k * 3 + n] : (k == H ? m.b3[n] : 0.0f));
    *reinterpret_cast<uint16_t*>(ws + L::kB3 + kmajor_offset(n, k, L::K2)) = to_bits<BF16>(v);
  }
  for (int i = tid; i < H * L::K1P; i += nt) {
    const int n = i / L::K1P, k = i % L::K1P;
    const float v = k < 16 ? m.w1[k * H + n] : (k == 16 ? m.b1[n] : 0.0f);
    *reinterpret_cast<uint16_t*>(ws + L::kB1P + kmajor_offset(n, k, L::K1P)) = to_bits<BF16>(v);
  }
  if (tid == 0) {
    *reinterpret_cast<int*>(ws + L::kErrOff) = 0;
    *reinterpret_cast<int*>(ws + L::kDbgOff) = 0;
  }
}

// Layer-1 row: the 16 features, then 1 (column 16, carries b1), then zeros.
template <bool BF16>
__device__ __forceinline__ void hybrid_pack_a1(const float (&x)[16], uint32_t (&w)[16]) {
#pragma unroll
  for (int k = 0; k < 8; ++k) w[k] = pack2<BF16>(x[2 * k], x[2 * k + 1]);
  w[8] = BF16 ? 0x3F80u : 0x3C00u;
#pragma unroll
  for (int k = 9; k < 16; ++k) w[k] = 0u;
}

// Two GELUs with the packed FP32 pair instructions of sm_100+ (fma.rn.f32x2,
// mul.rn.f32x2): the arithmetic of gelu_fast element for element, in half
// the FMA-pipe instructions (the reciprocals stay scalar).
__device__ __forceinline__ uint64_t f2_pack(float lo, float hi) {
  uint64_t d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
  return d;
}
__device__ __forceinline__ void f2_unpack(uint64_t v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ float2 gelu_fast2(float a, float b) {
  constexpr float k = 1.0442737824274138f;   // 2^(1/16), as in gelu_fast
  const uint64_t z = f2_pack(fabsf(a) * 0.70710678118654752f, fabsf(b) * 0.70710678118654752f);
  uint64_t p = f2_fma(f2_pack(k * 0.0000430638f, k * 0.0000430638f), z,
                      f2_pack(k * 0.0002765672f, k * 0.0002765672f));
  p = f2_fma(p, z, f2_pack(k * 0.0001520143f, k * 0.0001520143f));
  p = f2_fma(p, z, f2_pack(k * 0.0092705272f, k * 0.0092705272f));
  p = f2_fma(p, z, f2_pack(k * 0.0422820123f, k * 0.0422820123f));
  p = f2_fma(p, z, f2_pack(k * 0.0705230784f, k * 0.0705230784f));
  p = f2_fma(p, z, f2_pack(k, k));
  float pa, pb, ra, rb;
  f2_unpack(p, pa, pb);
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(ra) : "f"(pa));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rb) : "f"(pb));
  uint64_t r = f2_pack(ra, rb);
  r = f2_mul(r, r);
  r = f2_mul(r, r);
  r = f2_mul(r, r);
  r = f2_mul(r, r);   // erfc(z) / 2
  f2_unpack(r, ra, rb);
  // x >= 0: x - x r = fma(x, -r, x); x < 0: x r = fma(x, r, 0)
  const float sa = __uint_as_float(__float_as_uint(ra) ^ (~__float_as_uint(a) & 0x80000000u));
  const float sb = __uint_as_float(__float_as_uint(rb) ^ (~__float_as_uint(b) & 0x80000000u));
  float ya, yb;
  f2_unpack(f2_fma(f2_pack(a, b), f2_pack(sa, sb), f2_pack(fmaxf(a, 0.0f), fmaxf(b, 0.0f))), ya, yb);
  return make_float2(ya, yb);
}

// GELU of two values for the FP16 / BF16 epilogues: x (1 + t P(t^2)) / 2 with
// t = clamp(x, -4.5, 4.5) and P of degree 8 in t^2 approximating
// erf(t / sqrt 2) / t (weighted least squares towards minimax; the
// coefficients and their check come from csrc/gelu_poly_fit.py), in the
// packed FP32-pair instructions.  |error| <= 4.5e-5 + 4e-6 |x| (beyond the
// clamp Phi is held at its polynomial value at +-4.5, 1.4e-6 past 1 or 0,
// i.e. within 4.9e-6 of Phi(x)), far below the FP16 rounding of the result
// (|x| 2^-12).
__device__ __forceinline__ float2 gelu_poly2(float a, float b) {
  constexpr float c0 = 0.7974528670310974f, c1 = -0.13199074566364288f, c2 = 0.019172420725226402f;
  constexpr float c3 = -0.002073553390800953f, c4 = 0.00016233573842328042f, c5 = -8.838639587338548e-06f;
  constexpr float c6 = 3.1406239031639416e-07f, c7 = -6.496896798324769e-09f, c8 = 5.903861427514201e-11f;
  const uint64_t t = f2_pack(fminf(fmaxf(a, -4.5f), 4.5f), fminf(fmaxf(b, -4.5f), 4.5f));
  // Horner on the halved coefficients (exact: powers of two), so that
  // 1/2 + t P(t^2) / 2 = Phi(x) takes one FMA and x Phi(x) one multiply.
  const uint64_t s = f2_mul(t, t);
  uint64_t p = f2_fma(f2_pack(0.5f * c8, 0.5f * c8), s, f2_pack(0.5f * c7, 0.5f * c7));
  p = f2_fma(p, s, f2_pack(0.5f * c6, 0.5f * c6));
  p = f2_fma(p, s, f2_pack(0.5f * c5, 0.5f * c5));
  p = f2_fma(p, s, f2_pack(0.5f * c4, 0.5f * c4));
  p = f2_fma(p, s, f2_pack(0.5f * c3, 0.5f * c3));
  p = f2_fma(p, s, f2_pack(0.5f * c2, 0.5f * c2));
  p = f2_fma(p, s, f2_pack(0.5f * c1, 0.5f * c1));
  p = f2_fma(p, s, f2_pack(0.5f * c0, 0.5f * c0));
  const uint64_t phi = f2_fma(t, p, f2_pack(0.5f, 0.5f));   // Phi(x)
  float ya, yb;
  f2_unpack(f2_mul(f2_pack(a, b), phi), ya, yb);
  return make_float2(ya, yb);
}

// Slot s of a lane's engine: this thread's layer-1/2 accumulator row -> GELU ->
// FP16/BF16 -> the hidden A tile, 16 columns at a time; with ONES also the
// ones column that carries the next layer's bias (the engine's ReLU epilogue
// with GELU in its place).
template <bool ONES, typename E>
__device__ __forceinline__ void epilogue_gelu(E& e, int s) {
  static_assert(!E::F8 && E::kACol % 16 == 0, "16-column FP16/BF16 epilogue");
  constexpr int H = (int)E::kACol;
  const uint32_t d = e.tmem[s] + e.lane_off, a = d + E::kACol;
#pragma unroll
  for (int c = 0; c < H; c += 16) {
    uint32_t r[16], w[8];
    tmem_ld16(d + c, r);
    tmem_ld_wait();
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float2 g = gelu_poly2(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1]));
      w[j] = pack2<E::BF16>(g.x, g.y);
    }
    tmem_st8(a + c / 2, w);
  }
  if constexpr (ONES) {
    const uint32_t one = E::BF16 ? 0x3F80u : 0x3C00u;
    const uint32_t ow[8] = {one, 0, 0, 0, 0, 0, 0, 0};
    tmem_st8(a + H / 2, ow);
  }
}

// One lane's tiles first, first + step, ... (< tiles) through the three
// layers, software-pipelined: the next tile's gather runs while this tile's
// layer 2 is on the tensor core, and its layer 1 is issued with this tile's
// layer 3.  gather(tile, w) gives this thread's layer-1 row, emit(tile, rgb)
// takes its result.  Returns false once a wait of the lane has timed out.
template <typename E, typename G, typename O>
__device__ __forceinline__ bool hybrid_lane_run(E& e, int64_t first, int64_t step, int64_t tiles, G&& gather,
                                                O&& emit, bool& inflight) {
  static_assert(E::kMerge, "layer 3 and the next layer 1 share one commit");
  if (first >= tiles) return true;
  {
    uint32_t w[E::kA1Words];
    gather(first, w);
    e.write_a1(0, w);
  }
  if (!e.layer1(0)) return false;
  inflight = true;
  int64_t cur = first, prev = -1, next = first + step;
  for (;;) {
    inflight = !e.wait(0);   // layer 1 of cur (and layer 3 of prev)
    if (prev >= 0) {         // lane-uniform: false on the first tile only
      float y0, y1, y2;
      e.output(0, y0, y1, y2);   // D3 is read before the layer-2 rows overwrite its columns
      emit(prev, y0, y1, y2);
    }
    epilogue_gelu<true>(e, 0);
    if (!e.layer2(0)) return false;
    inflight = true;
    const bool more = next < tiles;
    if (more) {
      uint32_t w[E::kA1Words];
      gather(next, w);
      e.write_a1(0, w);
    }
    inflight = !e.wait(0);   // layer 2
    epilogue_gelu<false>(e, 0);
    if (!e.layer3(0, more)) return false;
    inflight = true;
    if (!more) break;
    prev = cur;
    cur = next;
    next += step;
  }
  inflight = !e.wait(0);     // the last layer 3
  float y0, y1, y2;
  e.output(0, y0, y1, y2);
  emit(cur, y0, y1, y2);
  return true;
}

template <int H, bool BF16>
__global__ void __launch_bounds__(kLaneThreads* kHybLanes, 1)
    k_hybrid_points_tc(DevHybrid m, const float* __restrict__ uvt, int64_t n, float* __restrict__ rgb) {
  using L = HybridLayout<H>;
  using S = HybridSmem<H>;
  constexpr int P = BF16 ? kBF16 : kF16;
  using E = Engine<H, P, L::K1P, 1>;
  static_assert(kHybLanes * E::kSlotCols <= 512, "slots exceed the SM's tensor memory");
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ uint64_t bars[kHybLanes];
  __shared__ uint32_t slot;
  __shared__ uint2 lut[16];
  __shared__ float s_b3[3];
  const int tid = threadIdx.x;
  copy16(sm + S::kW, m.ws, L::kShared, tid, blockDim.x);
  copy16(sm + S::kB1, m.ws + L::kB1P, H * L::K1P * 2, tid, blockDim.x);
  init_p35_lut(lut, tid);
  if (tid < 3) s_b3[tid] = stored_b3<BF16>(m.ws + L::kB3, tid, H, L::K2);
  const uint32_t tbase = cta_setup<kHybLanes, E::kSlotCols>(bars, &slot, tid);
  const uint32_t base = smem_addr(sm);
  E e;
  engine_init<H, P, L::K1P, 1>(e, tbase, bars, tid, base + S::kB1, base + S::kW + L::kB2, base + S::kW + L::kB3);
  e.b3 = s_b3;
  int* err = reinterpret_cast<int*>(m.ws + L::kErrOff);
  if (*reinterpret_cast<const int*>(m.ws + L::kDbgOff) & kDbgInjectTimeout) inject_timeout(e);
  const int t = e.t;
  auto gather = [&](int64_t tl, uint32_t (&w)[16]) {
    const int64_t q = tl * 128 + t;
    float x[16];
    if (q < n) {
      hybrid_features(m, __ldcs(uvt + 3 * q), __ldcs(uvt + 3 * q + 1), __ldcs(uvt + 3 * q + 2), x, lut);
    } else {
#pragma unroll
      for (int k = 0; k < 16; ++k) x[k] = 0.0f;
    }
    hybrid_pack_a1<BF16>(x, w);
  };
  auto emit = [&](int64_t tl, float y0, float y1, float y2) {
    const int64_t q = tl * 128 + t;
    if (q < n) {
      __stcs(rgb + 3 * q, y0);
      __stcs(rgb + 3 * q + 1, y1);
      __stcs(rgb + 3 * q + 2, y2);
    }
  };
  bool inflight[1] = {false};
  const bool ok = hybrid_lane_run(e, (int64_t)blockIdx.x * kHybLanes + e.wg, (int64_t)gridDim.x * kHybLanes,
                                  (n + 127) / 128, gather, emit, inflight[0]);
  cta_teardown<kHybLanes, E::kSlotCols, E, 1>(tbase, e, inflight, !ok, tid, err);
}

// F3D texel (x, y) of slices z0 and z1 blended at fz, all four channels.
__device__ __forceinline__ float4 vol_texel(const DevHybrid& m, int x, int y, int z0, int z1, float fz,
                                            const uint2* lut) {
  if (m.bc7) {
    const size_t slice = vol_slice_bytes(m), off = ((size_t)(y >> 2) * (m.vol_w / 4) + (x >> 2)) * 16;
    const int p = ((y & 3) << 2) | (x & 3);
    float a[4], b[4];
    u8x4_unpack(bc7_texel(__ldg(reinterpret_cast<const uint4*>(m.vol + (size_t)z0 * slice + off)), p), a);
    u8x4_unpack(bc7_texel(__ldg(reinterpret_cast<const uint4*>(m.vol + (size_t)z1 * slice + off)), p), b);
    const float gz = 1.0f - fz;
    return make_float4(gz * a[0] + fz * b[0], gz * a[1] + fz * b[1], gz * a[2] + fz * b[2], gz * a[3] + fz * b[3]);
  }
  const size_t slice = (size_t)(m.vol_h / 4) * (size_t)(m.vol_w / 4) * 32;
  const size_t off = ((size_t)(y >> 2) * (m.vol_w / 4) + (x >> 2)) * 32;
  const uint32_t shift = 16u + 3u * (uint32_t)(((y & 3) << 2) | (x & 3));
  const uint4* la = reinterpret_cast<const uint4*>(m.vol + (size_t)z0 * slice + off);
  const uint4* lb = reinterpret_cast<const uint4*>(m.vol + (size_t)z1 * slice + off);
  const uint4 a0 = __ldg(la), a1 = __ldg(la + 1), b0 = __ldg(lb), b1 = __ldg(lb + 1);
  const float gz = 1.0f - fz;
  float4 v;
  v.x = gz * p35_value(bc4_p35_lut(a0.x, a0.y, shift, lut)) + fz * p35_value(bc4_p35_lut(b0.x, b0.y, shift, lut));
  v.y = gz * p35_value(bc4_p35_lut(a0.z, a0.w, shift, lut)) + fz * p35_value(bc4_p35_lut(b0.z, b0.w, shift, lut));
  v.z = gz * p35_value(bc4_p35_lut(a1.x, a1.y, shift, lut)) + fz * p35_value(bc4_p35_lut(b1.x, b1.y, shift, lut));
  v.w = gz * p35_value(bc4_p35_lut(a1.z, a1.w, shift, lut)) + fz * p35_value(bc4_p35_lut(b1.z, b1.w, shift, lut));
  return v;
}

// Pages: one request per CTA at a time.  Per request the CTA stages its
// model's image in shared memory and, once for the whole page, everything
// that depends on one axis only: per column the F3D and F_uv taps along u and
// V_ut, per row the same along v and V_vt, gamma(t), and (when the page's F3D
// footprint is at most 48 x 48 texels) the F3D texels it touches, already
// blended between the two slices around t.  A texel then costs one bilinear
// step over staged F3D values and one BC4 bilinear sample of F_uv (one tap
// where both fractions are zero, as at texel centres of an F_uv of the
// lightmap's size).  The four lanes take the page's 128-texel tiles in turn
// (texel k of the request is (k mod w, k div w)).
template <int H, bool BF16, bool BC7>
__global__ void __launch_bounds__(kLaneThreads* kHybLanes, 1)
    k_hybrid_pages_tc(HybridPagesCtx c, const ndgi_page_req* __restrict__ reqs, int n) {
  using L = HybridLayout<H>;
  using S = HybridSmem<H>;
  constexpr int P = BF16 ? kBF16 : kF16;
  using E = Engine<H, P, L::K1P, 1>;
  static_assert(kHybLanes * E::kSlotCols <= 512, "slots exceed the SM's tensor memory");
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ uint64_t bars[kHybLanes];
  __shared__ uint32_t slot;
  __shared__ uint2 lut[16];
  __shared__ float s_b3[3], s_gamma[4], s_fz;
  __shared__ int s_z[2], s_lo[2], s_hi[2], s_ulo[2], s_uhi[2];
  uint32_t* uvs = reinterpret_cast<uint32_t*>(sm + S::kUv);
  HybAxis* cols = reinterpret_cast<HybAxis*>(sm + S::kCols);
  HybAxis* rows = reinterpret_cast<HybAxis*>(sm + S::kRows);
  float4* vol = reinterpret_cast<float4*>(sm + S::kVol);
  const int tid = threadIdx.x;
  init_p35_lut(lut, tid);
  const uint32_t tbase = cta_setup<kHybLanes, E::kSlotCols>(bars, &slot, tid);
  const uint32_t base = smem_addr(sm);
  E e;
  engine_init<H, P, L::K1P, 1>(e, tbase, bars, tid, base + S::kB1, base + S::kW + L::kB2, base + S::kW + L::kB3);
  e.b3 = s_b3;
  if (c.debug_word && (*c.debug_word & kDbgInjectTimeout)) inject_timeout(e);
  const int t = e.t;
  bool inflight[1] = {false}, stopped = false;
  for (int ri = blockIdx.x; ri < n; ri += gridDim.x) {
    const ndgi_page_req r = reqs[ri];
    const bool ok = hybrid_req_ok(r, c.models, c.n_models, c.phys_w, c.phys_h, c.border);
    tc_fence_before();
    __syncthreads();   // every lane is done with the previous request's image and tables
    if (!ok) {
      if (tid == 0) atomicOr(c.error_word, 1);
      continue;
    }
    const DevHybrid& m = c.models[r.model];
    copy16(sm + S::kW, m.ws, L::kShared, tid, blockDim.x);
    copy16(sm + S::kB1, m.ws + L::kB1P, H * L::K1P * 2, tid, blockDim.x);
    if (tid < 3) s_b3[tid] = stored_b3<BF16>(m.ws + L::kB3, tid, H, L::K2);
    if (tid == 0) {
      s_lo[0] = s_lo[1] = s_ulo[0] = s_ulo[1] = 0x7fffffff;
      s_hi[0] = s_hi[1] = s_uhi[0] = s_uhi[1] = -1;
    }
    __syncthreads();
    // ---- per-axis tables, gamma(t) and the F3D slice pair ----
    const int mode = m.address_mode;
    const int b = c.border, pw = r.w + 2 * b, ph = r.h + 2 * b;
    if (tid < pw || (tid >= kHybAxisMax && tid - kHybAxisMax < ph)) {
      const bool col = tid < kHybAxisMax;
      const int i = col ? tid : tid - kHybAxisMax;
      const float coord = col ? ((float)(r.x0 + border_mirror(i, r.w, b)) + 0.5f) / (float)m.lm_w
                              : ((float)(r.y0 + border_mirror(i, r.h, b)) + 0.5f) / (float)m.lm_h;
      HybAxis a;
      axis_setup(coord, col ? m.vol_w : m.vol_h, mode, a.v0, a.v1, a.vf);
      axis_setup(coord, col ? m.uv_w : m.uv_h, mode, a.u0, a.u1, a.uf);
      int x0, x1, y0, y1;
      float fx, fy, pv[2];
      axis_setup(coord, col ? m.ut_w : m.vt_h, mode, x0, x1, fx);
      axis_setup(r.t, col ? m.ut_t : m.vt_t, 0, y0, y1, fy);
      u8x2_bilinear(col ? m.ut : m.vt, col ? m.ut_w : m.vt_h, x0, x1, y0, y1, fx, fy, pv);
      a.p0 = pv[0];
      a.p1 = pv[1];
      (col ? cols : rows)[i] = a;
      atomicMin(&s_lo[col ? 0 : 1], min(a.v0, a.v1));
      atomicMax(&s_hi[col ? 0 : 1], max(a.v0, a.v1));
      if (BC7) {
        atomicMin(&s_ulo[col ? 0 : 1], min(a.u0, a.u1));
        atomicMax(&s_uhi[col ? 0 : 1], max(a.u0, a.u1));
      }
    } else if (tid == 2 * kHybAxisMax) {
      sincospif(r.t, &s_gamma[0], &s_gamma[1]);
      sincospif(2.0f * r.t, &s_gamma[2], &s_gamma[3]);
      axis_setup(r.t, m.vol_t, 0, s_z[0], s_z[1], s_fz);
    }
    __syncthreads();
    const int lx = s_lo[0], ly = s_lo[1], fw = s_hi[0] - lx + 1, fh = s_hi[1] - ly + 1;
    const bool staged = fw <= kHybVolSide && fh <= kHybVolSide;
    const int z0 = s_z[0], z1 = s_z[1];
    const float fz = s_fz;
    if (staged)
      for (int i = tid; i < fw * fh; i += blockDim.x) vol[i] = vol_texel(m, lx + i % fw, ly + i / fw, z0, z1, fz, lut);
    // a BC7 F_uv: the page's footprint decoded once, whole blocks at a time, as RGBA8
    const int ulx = s_ulo[0], uly = s_ulo[1], ufw = s_uhi[0] - ulx + 1, ufh = s_uhi[1] - uly + 1;
    const bool uv_staged = BC7 && m.bc7 && ufw <= kHybUvSide && ufh <= kHybUvSide;
    if (uv_staged) {
      const int bx0 = ulx >> 2, by0 = uly >> 2, nbx = (s_uhi[0] >> 2) - bx0 + 1;
      const int nb = nbx * ((s_uhi[1] >> 2) - by0 + 1);
      for (int i = tid; i < nb; i += blockDim.x) {
        const int bx = bx0 + i % nbx, by = by0 + i / nbx;
        uint32_t px[16];
        bc7_block(__ldg(reinterpret_cast<const uint4*>(m.uv + ((size_t)by * (m.uv_w / 4) + bx) * 16)), px);
#pragma unroll
        for (int p = 0; p < 16; ++p) {
          const int xx = 4 * bx + (p & 3) - ulx, yy = 4 * by + (p >> 2) - uly;
          if (xx >= 0 && xx < ufw && yy >= 0 && yy < ufh) uvs[yy * ufw + xx] = px[p];
        }
      }
    }
    fence_async_smem();
    __syncthreads();
    tc_fence_after();
    if (stopped) continue;
    const int texels = pw * ph;
    auto gather = [&](int64_t tl, uint32_t (&w)[16]) {
      const int k = (int)tl * 128 + t;
      float x[16];
      if (k < texels) {
        const HybAxis& cx = cols[k % pw];
        const HybAxis& cy = rows[k / pw];
        if (staged) {
          const float4 q00 = vol[(cy.v0 - ly) * fw + (cx.v0 - lx)], q10 = vol[(cy.v0 - ly) * fw + (cx.v1 - lx)];
          const float4 q01 = vol[(cy.v1 - ly) * fw + (cx.v0 - lx)], q11 = vol[(cy.v1 - ly) * fw + (cx.v1 - lx)];
          const float gx = 1.0f - cx.vf, gy = 1.0f - cy.vf, fx = cx.vf, fy = cy.vf;
          x[0] = gy * (gx * q00.x + fx * q10.x) + fy * (gx * q01.x + fx * q11.x);
          x[1] = gy * (gx * q00.y + fx * q10.y) + fy * (gx * q01.y + fx * q11.y);
          x[2] = gy * (gx * q00.z + fx * q10.z) + fy * (gx * q01.z + fx * q11.z);
          x[3] = gy * (gx * q00.w + fx * q10.w) + fy * (gx * q01.w + fx * q11.w);
        } else {
          const size_t slice = vol_slice_bytes(m);
          float a[4], b[4];
          map4_bilinear(m, m.vol + (size_t)z0 * slice, m.vol_w / 4, cx.v0, cx.v1, cy.v0, cy.v1, cx.vf, cy.vf, lut, a);
          map4_bilinear(m, m.vol + (size_t)z1 * slice, m.vol_w / 4, cx.v0, cx.v1, cy.v0, cy.v1, cx.vf, cy.vf, lut, b);
#pragma unroll
          for (int j = 0; j < 4; ++j) x[j] = (1.0f - fz) * a[j] + fz * b[j];
        }
        if (BC7 && uv_staged) {
          const uint32_t* r0 = uvs + (cy.u0 - uly) * ufw - ulx;
          if (cx.uf == 0.0f && cy.uf == 0.0f) {
            u8x4_unpack(r0[cx.u0], x + 4);
          } else {
            const uint32_t* r1 = uvs + (cy.u1 - uly) * ufw - ulx;
            float f[4][4];
            u8x4_unpack(r0[cx.u0], f[0]);
            u8x4_unpack(r0[cx.u1], f[1]);
            u8x4_unpack(r1[cx.u0], f[2]);
            u8x4_unpack(r1[cx.u1], f[3]);
            const float gx = 1.0f - cx.uf, gy = 1.0f - cy.uf;
#pragma unroll
            for (int c = 0; c < 4; ++c)
              x[4 + c] = gy * (gx * f[0][c] + cx.uf * f[1][c]) + cy.uf * (gx * f[2][c] + cx.uf * f[3][c]);
          }
        } else if (BC7 && m.bc7) {
          if (cx.uf == 0.0f && cy.uf == 0.0f) {
            const uint4 blk = __ldg(reinterpret_cast<const uint4*>(m.uv + ((size_t)(cy.u0 >> 2) * (m.uv_w / 4) +
                                                                         (cx.u0 >> 2)) * 16));
            u8x4_unpack(bc7_texel(blk, ((cy.u0 & 3) << 2) | (cx.u0 & 3)), x + 4);
          } else {
            bc7_bilinear(m.uv, m.uv_w / 4, cx.u0, cx.u1, cy.u0, cy.u1, cx.uf, cy.uf, x + 4);
          }
        } else if (cx.uf == 0.0f && cy.uf == 0.0f) {   // one tap (its weight is 1)
          const uint4* line = reinterpret_cast<const uint4*>(m.uv + ((size_t)(cy.u0 >> 2) * (m.uv_w / 4) +
                                                                     (cx.u0 >> 2)) * 32);
          const uint4 a = __ldg(line), b = __ldg(line + 1);
          const uint32_t shift = 16u + 3u * (uint32_t)(((cy.u0 & 3) << 2) | (cx.u0 & 3));
          x[4] = p35_value(bc4_p35_lut(a.x, a.y, shift, lut));
          x[5] = p35_value(bc4_p35_lut(a.z, a.w, shift, lut));
          x[6] = p35_value(bc4_p35_lut(b.x, b.y, shift, lut));
          x[7] = p35_value(bc4_p35_lut(b.z, b.w, shift, lut));
        } else {
          bc4x4_bilinear(m.uv, m.uv_w / 4, cx.u0, cx.u1, cy.u0, cy.u1, cx.uf, cy.uf, lut, x + 4);
        }
        x[8] = cx.p0;
        x[9] = cx.p1;
        x[10] = cy.p0;
        x[11] = cy.p1;
#pragma unroll
        for (int j = 0; j < 4; ++j) x[12 + j] = s_gamma[j];
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) x[j] = 0.0f;
      }
      hybrid_pack_a1<BF16>(x, w);
    };
    auto emit = [&](int64_t tl, float y0, float y1, float y2) {
      const int k = (int)tl * 128 + t;
      if (k < texels)
        put_texel(c.phys, c.fmt, (int64_t)(r.dst_y - b + k / pw) * c.phys_w + (r.dst_x - b + k % pw), y0, y1, y2);
    };
    stopped = !hybrid_lane_run(e, e.wg, kHybLanes, (texels + 127) / 128, gather, emit, inflight[0]);
  }
  cta_teardown<kHybLanes, E::kSlotCols, E, 1>(tbase, e, inflight, stopped, tid, c.error_word);
}

__global__ void k_debug_gelu(const float* __restrict__ x, int64_t n, float* __restrict__ y, int fast) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fast == 3 ? gelu_poly2(x[i], 0.0f).x
                     : fast == 2 ? gelu_fast2(x[i], 0.0f).x : (fast ? gelu_fast(x[i]) : gelu(x[i]));
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
#define NDGI_HYBRID_HIDDEN(X) X(16) X(32) X(64)

bool hybrid_hidden_ok(int hidden) {
#define X(H) if (hidden == H) return true;
  NDGI_HYBRID_HIDDEN(X)
#undef X
  return false;
}

size_t hybrid_ws_bytes(int hidden) {
#define X(H) if (hidden == H) return (HybridLayout<H>::kWsBytes + 16 + 255) / 256 * 256;
  NDGI_HYBRID_HIDDEN(X)
#undef X
  return 0;
}

int hybrid_err_offset(int hidden) {
#define X(H) if (hidden == H) return (int)HybridLayout<H>::kErrOff;
  NDGI_HYBRID_HIDDEN(X)
#undef X
  return -1;
}

cudaError_t launch_hybrid_prepare(const DevHybrid& m, bool bf16, cudaStream_t s) {
#define X(H)                                                                      \
  if (m.hidden == H) {                                                            \
    if (bf16) k_hybrid_prepare<H, true><<<8, 256, 0, s>>>(m, m.ws);               \
    else k_hybrid_prepare<H, false><<<8, 256, 0, s>>>(m, m.ws);                   \
    return cudaGetLastError();                                                    \
  }
  NDGI_HYBRID_HIDDEN(X)
#undef X
  return cudaErrorInvalidValue;
}

template <typename K>
static cudaError_t launch_tc_kernel(K kern, uint32_t smem, int grid, cudaStream_t s, void** args) {
  cudaError_t e = set_smem(kern, tc_smem(smem));
  if (e != cudaSuccess) return e;
  return cudaLaunchKernel((const void*)kern, dim3(grid), dim3(kLaneThreads * kHybLanes), args, tc_smem(smem), s);
}

// prec: 0 FP32, 1 FP16, 2 BF16.
cudaError_t launch_hybrid_points(const DevHybrid& m, int prec, const float* uvt, int64_t n, float* rgb,
                                 cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
#define X(H)                                                                                            \
  if (m.hidden == H) {                                                                                  \
    if (prec == 0) {                                                                                    \
      const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 8);                \
      k_hybrid_points_f32<H><<<grid, 256, 0, s>>>(m, uvt, n, rgb);                                      \
      return cudaGetLastError();                                                                        \
    }                                                                                                   \
    const int grid = (int)std::min<int64_t>(((n + 127) / 128 + kHybLanes - 1) / kHybLanes, num_sms()); \
    DevHybrid mm = m;                                                                                   \
    const float* a1 = uvt;                                                                              \
    int64_t a2 = n;                                                                                     \
    float* a3 = rgb;                                                                                    \
    void* args[] = {&mm, &a1, &a2, &a3};                                                                \
    return launch_tc_kernel(prec == 2 ? k_hybrid_points_tc<H, true> : k_hybrid_points_tc<H, false>,     \
                            HybridSmem<H>::kPoints, grid, s, args);                                     \
  }
  NDGI_HYBRID_HIDDEN(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t launch_hybrid_pages(const HybridPagesCtx& c, int hidden, int prec, const ndgi_page_req* reqs, int n,
                                cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
#define X(H)                                                                                       \
  if (hidden == H) {                                                                               \
    if (prec == 0) {                                                                               \
      const int grid = std::min(n, num_sms() * 8);                                                 \
      k_hybrid_pages_f32<H><<<grid, 256, 0, s>>>(c, reqs, n);                                      \
      return cudaGetLastError();                                                                   \
    }                                                                                              \
    HybridPagesCtx cc = c;                                                                         \
    const ndgi_page_req* a1 = reqs;                                                                \
    int a2 = n;                                                                                    \
    void* args[] = {&cc, &a1, &a2};                                                                \
    auto kern = c.uv_stage ? (prec == 2 ? k_hybrid_pages_tc<H, true, true> : k_hybrid_pages_tc<H, false, true>)   \
                           : (prec == 2 ? k_hybrid_pages_tc<H, true, false> : k_hybrid_pages_tc<H, false, false>); \
    return launch_tc_kernel(kern, c.uv_stage ? HybridSmem<H>::kPagesBc7 : HybridSmem<H>::kPages,             \
                            std::min(n, num_sms()), s, args);                                      \
  }
  NDGI_HYBRID_HIDDEN(X)
#undef X
  return cudaErrorInvalidValue;
}

}  // namespace ndgi

// ---------------------------------------------------------------------------
// C ABI (include/ndgi.h, hybrid feature map decoder)
// ---------------------------------------------------------------------------
using ndgi::DevHybrid;
using ndgi::HybridPagesCtx;
using ndgi::set_error;
using ndgi::cuda_status;

struct ndgi_hybrid_table {
  DevHybrid* d_models = nullptr;   // device copy of the descriptors
  int* d_words = nullptr;          // device: error word, debug word
  int n_models = 0, hidden = 0, prec = 0;
  int border = 0;                  // mirrored tile border of every page (texels per edge)
  int any_bc7 = 0;                 // some model holds BC7 maps
};

namespace {

bool is_aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

// The dimension checks shared by every hybrid call (device pointers unchecked).
ndgi_status check_hybrid_dims(const ndgi_hybrid_desc* m, const char* who) {
  if (!m) return set_error(NDGI_ERR_INVALID_ARG, "%s: model is NULL", who);
  if (m->lm_w <= 0 || m->lm_h <= 0) return set_error(NDGI_ERR_INVALID_ARG, "%s: lightmap size must be > 0", who);
  if (m->uv_w <= 0 || m->uv_h <= 0 || m->uv_w % 4 || m->uv_h % 4 || m->vol_w <= 0 || m->vol_h <= 0 ||
      m->vol_w % 4 || m->vol_h % 4 || m->vol_t <= 0)
    return set_error(NDGI_ERR_INVALID_ARG, "%s: F_uv and F3D slice sizes must be positive multiples of 4", who);
  if (m->ut_w <= 0 || m->ut_t <= 0 || m->vt_h <= 0 || m->vt_t <= 0)
    return set_error(NDGI_ERR_INVALID_ARG, "%s: F_ut / F_vt sizes must be > 0", who);
  if ((int64_t)m->uv_w * m->uv_h > ((int64_t)1 << 30) || (int64_t)m->vol_w * m->vol_h * m->vol_t > ((int64_t)1 << 30) ||
      (int64_t)m->ut_w * m->ut_t > ((int64_t)1 << 28) || (int64_t)m->vt_h * m->vt_t > ((int64_t)1 << 28))
    return set_error(NDGI_ERR_INVALID_ARG, "%s: a feature map is too large", who);
  if (!ndgi::hybrid_hidden_ok(m->hidden))
    return set_error(NDGI_ERR_UNSUPPORTED, "%s: hidden width %d not built (16, 32, 64)", who, m->hidden);
  if (m->address_mode != 0 && m->address_mode != 1)
    return set_error(NDGI_ERR_INVALID_ARG, "%s: address_mode must be 0 or 1", who);
  if (m->feat_format != NDGI_FEAT_BC4X4 && m->feat_format != NDGI_FEAT_BC7)
    return set_error(NDGI_ERR_INVALID_ARG, "%s: feat_format must be NDGI_FEAT_BC4X4 or NDGI_FEAT_BC7", who);
  return NDGI_OK;
}

ndgi_status check_hybrid(const ndgi_hybrid_desc* m, const char* who) {
  ndgi_status st = check_hybrid_dims(m, who);
  if (st != NDGI_OK) return st;
  if (!m->uv_bc4 || !m->vol_bc4 || !m->ut || !m->vt || !m->w1 || !m->b1 || !m->w2 || !m->b2 || !m->w3 || !m->b3)
    return set_error(NDGI_ERR_INVALID_ARG, "%s: a model array is NULL", who);
  if (!is_aligned(m->uv_bc4, 16) || !is_aligned(m->vol_bc4, 16) || !is_aligned(m->ut, 2) || !is_aligned(m->vt, 2))
    return set_error(NDGI_ERR_INVALID_ARG, "%s: BC arrays must be 16-byte and UNORM8 planes 2-byte aligned", who);
  return NDGI_OK;
}

DevHybrid to_dev_hybrid(const ndgi_hybrid_desc& d, const void* ws) {
  DevHybrid m;
  m.lm_w = d.lm_w;
  m.lm_h = d.lm_h;
  m.uv_w = d.uv_w;
  m.uv_h = d.uv_h;
  m.uv = d.uv_bc4;
  m.vol_w = d.vol_w;
  m.vol_h = d.vol_h;
  m.vol_t = d.vol_t;
  m.vol = d.vol_bc4;
  m.ut_w = d.ut_w;
  m.ut_t = d.ut_t;
  m.ut = d.ut;
  m.vt_h = d.vt_h;
  m.vt_t = d.vt_t;
  m.vt = d.vt;
  m.hidden = d.hidden;
  m.w1 = d.w1;
  m.b1 = d.b1;
  m.w2 = d.w2;
  m.b2 = d.b2;
  m.w3 = d.w3;
  m.b3 = d.b3;
  m.address_mode = d.address_mode;
  m.bc7 = d.feat_format == NDGI_FEAT_BC7;
  m.ws = static_cast<unsigned char*>(const_cast<void*>(ws));
  return m;
}

// 0 FP32, 1 FP16, 2 BF16, -1 not supported by the hybrid decode.
int hybrid_prec(ndgi_precision p) { return p == NDGI_FP32 ? 0 : p == NDGI_FP16 ? 1 : p == NDGI_BF16 ? 2 : -1; }

}  // namespace

extern "C" {

size_t ndgi_hybrid_workspace_size(const ndgi_hybrid_desc* model, ndgi_precision precision) {
  if (check_hybrid_dims(model, "ndgi_hybrid_workspace_size") != NDGI_OK) return 0;
  const int p = hybrid_prec(precision);
  return p > 0 ? ndgi::hybrid_ws_bytes(model->hidden) : 0;
}

ndgi_status ndgi_hybrid_prepare(const ndgi_hybrid_desc* model, ndgi_precision precision, void* ws, void* stream) {
  ndgi_status st = check_hybrid(model, "ndgi_hybrid_prepare");
  if (st != NDGI_OK) return st;
  const int p = hybrid_prec(precision);
  if (p < 0) return set_error(NDGI_ERR_UNSUPPORTED, "ndgi_hybrid_prepare: precision not built for hybrid models");
  if (p == 0) return NDGI_OK;
  if (!ws || !is_aligned(ws, 256))
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_hybrid_prepare: ws is NULL or not 256-byte aligned");
  return cuda_status(ndgi::launch_hybrid_prepare(to_dev_hybrid(*model, ws), p == 2, (cudaStream_t)stream),
                     "ndgi_hybrid_prepare");
}

ndgi_status ndgi_hybrid_decode_points(const ndgi_hybrid_desc* model, ndgi_precision precision, const void* ws,
                                      const float* uvt, int64_t n, float* rgb, void* stream) {
  ndgi_status st = check_hybrid(model, "ndgi_hybrid_decode_points");
  if (st != NDGI_OK) return st;
  if (n < 0) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_hybrid_decode_points: n < 0");
  if (n == 0) return NDGI_OK;
  if (!uvt || !rgb) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_hybrid_decode_points: uvt or rgb is NULL");
  if (!is_aligned(uvt, 4) || !is_aligned(rgb, 4))
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_hybrid_decode_points: uvt and rgb must be 4-byte aligned");
  const int p = hybrid_prec(precision);
  if (p < 0) return set_error(NDGI_ERR_UNSUPPORTED, "ndgi_hybrid_decode_points: precision not built for hybrid models");
  if (p > 0 && (!ws || !is_aligned(ws, 256)))
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_hybrid_decode_points: FP16/BF16 need the prepared workspace");
  return cuda_status(ndgi::launch_hybrid_points(to_dev_hybrid(*model, ws), p, uvt, n, rgb, (cudaStream_t)stream),
                     "ndgi_hybrid_decode_points");
}

ndgi_status ndgi_hybrid_workspace_check(const ndgi_hybrid_desc* model, ndgi_precision precision, const void* ws,
                                        int32_t* device_error, void* stream) {
  ndgi_status st = check_hybrid_dims(model, "ndgi_hybrid_workspace_check");
  if (st != NDGI_OK) return st;
  if (hybrid_prec(precision) <= 0 || !ws)
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_hybrid_workspace_check: needs an FP16/BF16 workspace");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_status(e, "ndgi_hybrid_workspace_check");
  int word = 0;
  unsigned char* w = static_cast<unsigned char*>(const_cast<void*>(ws)) + ndgi::hybrid_err_offset(model->hidden);
  e = cudaMemcpy(&word, w, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && word != 0) e = cudaMemset(w, 0, sizeof(int));
  if (e != cudaSuccess) return cuda_status(e, "ndgi_hybrid_workspace_check");
  if (device_error) *device_error = word;
  if (word & ndgi::kErrTimeout) return set_error(NDGI_ERR_TIMEOUT, "ndgi_hybrid_workspace_check: a wait timed out");
  return NDGI_OK;
}

ndgi_status ndgi_hybrid_debug_inject(const ndgi_hybrid_desc* model, ndgi_precision precision, void* ws,
                                     ndgi_hybrid_table* table, int32_t flags, void* stream) {
  if (ws) {
    ndgi_status st = check_hybrid_dims(model, "ndgi_hybrid_debug_inject");
    if (st != NDGI_OK) return st;
    if (hybrid_prec(precision) <= 0)
      return set_error(NDGI_ERR_INVALID_ARG, "ndgi_hybrid_debug_inject: needs an FP16/BF16 workspace");
    const int off = ndgi::hybrid_err_offset(model->hidden) + 4;
    cudaError_t e = cudaMemcpyAsync(static_cast<unsigned char*>(ws) + off, &flags, sizeof(int),
                                    cudaMemcpyHostToDevice, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_status(e, "ndgi_hybrid_debug_inject");
  }
  if (table) {
    cudaError_t e = cudaMemcpy(table->d_words + 1, &flags, sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_status(e, "ndgi_hybrid_debug_inject");
  }
  return NDGI_OK;
}

ndgi_status ndgi_hybrid_table_create(const ndgi_hybrid_desc* models, const void* const* ws, int32_t n_models,
                                     ndgi_precision precision, ndgi_hybrid_table** out) {
  if (!out) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_hybrid_table_create: out is NULL");
  *out = nullptr;
  if (!models || n_models <= 0) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_hybrid_table_create: no models");
  const int p = hybrid_prec(precision);
  if (p < 0) return set_error(NDGI_ERR_UNSUPPORTED, "ndgi_hybrid_table_create: precision not built for hybrid models");
  std::vector<DevHybrid> h(n_models);
  for (int i = 0; i < n_models; ++i) {
    ndgi_status st = check_hybrid(&models[i], "ndgi_hybrid_table_create");
    if (st != NDGI_OK) return st;
    if (models[i].hidden != models[0].hidden)
      return set_error(NDGI_ERR_INVALID_ARG, "ndgi_hybrid_table_create: models differ in hidden width");
    const void* w = nullptr;
    if (p > 0) {
      if (!ws || !ws[i] || !is_aligned(ws[i], 256))
        return set_error(NDGI_ERR_INVALID_ARG, "ndgi_hybrid_table_create: model %d has no prepared workspace", i);
      w = ws[i];
    }
    h[i] = to_dev_hybrid(models[i], w);
  }
  auto* t = new ndgi_hybrid_table;
  t->n_models = n_models;
  t->hidden = models[0].hidden;
  for (int i = 0; i < n_models; ++i) t->any_bc7 |= models[i].feat_format == NDGI_FEAT_BC7;
  t->prec = p;
  cudaError_t e = cudaMalloc(&t->d_models, sizeof(DevHybrid) * n_models);
  if (e == cudaSuccess) e = cudaMalloc(&t->d_words, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(t->d_models, h.data(), sizeof(DevHybrid) * n_models, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(t->d_words, 0, 2 * sizeof(int));
  if (e != cudaSuccess) {
    cudaFree(t->d_models);
    cudaFree(t->d_words);
    delete t;
    return cuda_status(e, "ndgi_hybrid_table_create");
  }
  *out = t;
  return NDGI_OK;
}

ndgi_status ndgi_hybrid_table_destroy(ndgi_hybrid_table* table) {
  if (!table) return NDGI_OK;
  cudaFree(table->d_models);
  cudaFree(table->d_words);
  delete table;
  return NDGI_OK;
}

ndgi_status ndgi_hybrid_decode_pages(ndgi_hybrid_table* table, const ndgi_page_req* reqs, int32_t n, void* phys,
                                     int64_t phys_w, int64_t phys_h, ndgi_out_format format, void* stream) {
  if (!table) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_hybrid_decode_pages: table is NULL");
  if (n < 0) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_hybrid_decode_pages: n < 0");
  if (n == 0) return NDGI_OK;
  if (!reqs || !phys) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_hybrid_decode_pages: reqs or phys is NULL");
  if (phys_w <= 0 || phys_h <= 0) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_hybrid_decode_pages: empty phys");
  if (format != NDGI_RGBA32F && format != NDGI_RGBA16F && format != NDGI_RGBA8)
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_hybrid_decode_pages: unknown output format");
  if (!is_aligned(phys, format == NDGI_RGBA32F ? 16 : format == NDGI_RGBA16F ? 8 : 4) || !is_aligned(reqs, 4))
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_hybrid_decode_pages: phys or reqs misaligned");
  HybridPagesCtx c;
  c.models = table->d_models;
  c.n_models = table->n_models;
  c.phys = phys;
  c.phys_w = phys_w;
  c.phys_h = phys_h;
  c.fmt = (int)format;
  c.error_word = table->d_words;
  c.debug_word = table->d_words + 1;
  c.border = table->border;
  c.uv_stage = table->any_bc7;
  return cuda_status(ndgi::launch_hybrid_pages(c, table->hidden, table->prec, reqs, n, (cudaStream_t)stream),
                     "ndgi_hybrid_decode_pages");
}

ndgi_status ndgi_hybrid_table_set_border(ndgi_hybrid_table* table, int32_t border) {
  if (!table || border < 0 || border > ndgi::kHybBorderMax)
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_hybrid_table_set_border: bad table or border (0..%d)",
                     ndgi::kHybBorderMax);
  table->border = border;
  return NDGI_OK;
}

ndgi_status ndgi_hybrid_table_check(ndgi_hybrid_table* table, int32_t* device_error, void* stream) {
  if (!table) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_hybrid_table_check: table is NULL");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  int word = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&word, table->d_words, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && word != 0) e = cudaMemset(table->d_words, 0, sizeof(int));
  if (e != cudaSuccess) return cuda_status(e, "ndgi_hybrid_table_check");
  if (device_error) *device_error = word;
  if (word & ndgi::kErrTimeout) return set_error(NDGI_ERR_TIMEOUT, "ndgi_hybrid_table_check: a wait timed out");
  if (word) return set_error(NDGI_ERR_DEVICE_CHECK, "ndgi_hybrid_table_check: a request was rejected (0x%x)", word);
  return NDGI_OK;
}

ndgi_status ndgi_debug_gelu(const float* x, int64_t n, float* y, int32_t fast, void* stream) {
  if (n < 0) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_debug_gelu: n < 0");
  if (n == 0) return NDGI_OK;
  if (!x || !y) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_debug_gelu: x or y is NULL");
  const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)ndgi::num_sms() * 8);
  ndgi::k_debug_gelu<<<grid, 256, 0, (cudaStream_t)stream>>>(x, n, y, fast);
  return cuda_status(cudaGetLastError(), "ndgi_debug_gelu");
}

double ndgi_model_bpp(const ndgi_hybrid_desc* model, int32_t n_lightmaps, int32_t bc_bits_per_texel,
                      int32_t mlp_bits) {
  if (!model || n_lightmaps <= 0 || mlp_bits <= 0) return -1.0;
  if (bc_bits_per_texel <= 0) bc_bits_per_texel = model->feat_format == NDGI_FEAT_BC7 ? 8 : 16;
  if (model->lm_w <= 0 || model->lm_h <= 0 || model->uv_w <= 0 || model->uv_h <= 0 || model->vol_w <= 0 ||
      model->vol_h <= 0 || model->vol_t <= 0 || model->ut_w <= 0 || model->ut_t <= 0 || model->vt_h <= 0 ||
      model->vt_t <= 0 || model->hidden <= 0)
    return -1.0;
  const double H = model->hidden;
  const double bc_texels = (double)model->uv_w * model->uv_h + (double)model->vol_w * model->vol_h * model->vol_t;
  const double u8_values = 2.0 * model->ut_w * model->ut_t + 2.0 * model->vt_h * model->vt_t;
  const double params = (16.0 * H + H) + (H * H + H) + (3.0 * H + 3.0);
  const double bits = bc_texels * bc_bits_per_texel + u8_values * 8.0 + params * mlp_bits;
  return bits / ((double)model->lm_w * model->lm_h * n_lightmaps);
}

}  // extern "C"
