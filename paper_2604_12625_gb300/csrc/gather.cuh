// FP32 feature gather shared by the CUDA-core and tensor-core decodes.
#pragma once

#include "ndgi_internal.h"
#include "bc4.cuh"

namespace ndgi {

// Feature gather at (u, v, t) in FP32: x = [v_s (CS), v_t (CT)].
// If p35 != nullptr, the tap numerators are written there ([4][CS]).  `lut`
// is the 16-entry palette table in shared memory (init_p35_lut).  Block lines
// are read 16 bytes (two planes) at a time.
// BATCHED = false reads one plane pair of the four taps at a time and never
// skips a load: fewer live registers, for kernels where the gather is a cold
// path and register pressure matters more.
template <int CS, int CT, bool BATCHED = true>
__device__ __forceinline__ void gather_f32(const DevModel& m, float u, float v, float t, float (&x)[CS + CT],
                                           int32_t* p35, const uint2* lut) {
  static_assert(CS % 2 == 0, "planes are read in pairs");
  int x0, x1, y0, y1;
  float fx, fy;
  axis_setup(u, m.feat_w, m.address_mode, x0, x1, fx);
  axis_setup(v, m.feat_h, m.address_mode, y0, y1, fy);
  const int tx[4] = {x0, x1, x0, x1};
  const int ty[4] = {y0, y0, y1, y1};
  const uint4* line[4];
  uint32_t shift[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    line[q] = reinterpret_cast<const uint4*>(m.bc4 + ((size_t)(ty[q] >> 2) * m.bw + (tx[q] >> 2)) * CS * 8);
    shift[q] = 16u + 3u * (uint32_t)(((ty[q] & 3) << 2) | (tx[q] & 3));
  }
  const float gx = 1.0f - fx, gy = 1.0f - fy;
  // Planes in groups of up to 8: all of a group's block loads (4 taps x 16
  // bytes per plane pair) are issued before any of them is decoded, so a
  // query waits on the memory system once per group rather than per pair.
  if (BATCHED) {
    // Taps that fall in a block already loaded reuse its line instead of
    // loading it again (the two x taps share a block 3 times in 4, likewise y),
    // which cuts the L1 requests of random queries from 4 lines to ~1.6; the
    // loads of a group of up to 8 planes are all issued before decoding.
    constexpr int G = CS < 8 ? CS : 8;
    const bool same_x = (x0 >> 2) == (x1 >> 2), same_y = (y0 >> 2) == (y1 >> 2);
#pragma unroll
    for (int c0 = 0; c0 < CS; c0 += G) {
      uint4 b[4][G / 2];
#pragma unroll
      for (int e = 0; e < G / 2; ++e) {
        b[0][e] = __ldg(line[0] + c0 / 2 + e);
        if (!same_x) b[1][e] = __ldg(line[1] + c0 / 2 + e);
        if (!same_y) b[2][e] = __ldg(line[2] + c0 / 2 + e);
        if (!same_x && !same_y) b[3][e] = __ldg(line[3] + c0 / 2 + e);
      }
#pragma unroll
      for (int e = 0; e < G / 2; ++e) {
        if (same_x) b[1][e] = b[0][e];
        if (same_y) b[2][e] = b[0][e];
        if (same_x || same_y) b[3][e] = same_x ? b[2][e] : b[1][e];
      }
#pragma unroll
      for (int e = 0; e < G / 2; ++e) {
        const int c = c0 + 2 * e;
        float f[2][4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int p0 = bc4_p35_lut(b[q][e].x, b[q][e].y, shift[q], lut);
          const int p1 = bc4_p35_lut(b[q][e].z, b[q][e].w, shift[q], lut);
          if (p35) {
            p35[q * CS + c] = p0;
            p35[q * CS + c + 1] = p1;
          }
          f[0][q] = p35_value(p0);
          f[1][q] = p35_value(p1);
        }
#pragma unroll
        for (int k = 0; k < 2; ++k)
          x[c + k] = gy * (gx * f[k][0] + fx * f[k][1]) + fy * (gx * f[k][2] + fx * f[k][3]);
      }
    }
  } else {
#pragma unroll
    for (int c = 0; c < CS; c += 2) {
      float f[2][4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint4 b = __ldg(line[q] + c / 2);
        const int p0 = bc4_p35_lut(b.x, b.y, shift[q], lut);
        const int p1 = bc4_p35_lut(b.z, b.w, shift[q], lut);
        if (p35) {
          p35[q * CS + c] = p0;
          p35[q * CS + c + 1] = p1;
        }
        f[0][q] = p35_value(p0);
        f[1][q] = p35_value(p1);
      }
#pragma unroll
      for (int k = 0; k < 2; ++k)
        x[c + k] = gy * (gx * f[k][0] + fx * f[k][1]) + fy * (gx * f[k][2] + fx * f[k][3]);
    }
  }
  int j0, j1;
  float a;
  temporal_setup(t, m.t_count, j0, j1, a);
  const float ga = 1.0f - a;
#pragma unroll
  for (int c = 0; c < CT; ++c) {
    const float k0 = load_temporal(m.temporal, m.temporal_f16, j0 * CT + c);
    const float k1 = load_temporal(m.temporal, m.temporal_f16, j1 * CT + c);
    x[CS + c] = ga * k0 + a * k1;
  }
}

// Palette table for gather_tc: as init_p35_lut, with the exponent bits of
// 2^23 added to the constant term, so the byte dot product's integer result
// read as a float is exactly 2^23 + P35 (P35 < 2^23 never carries into them).
__device__ __forceinline__ void init_p35_lut_f(uint2* lut, int tid) {
  init_p35_lut(lut, tid);
  if (tid < 16) lut[tid].y += 0x4B000000u;
}

__device__ __forceinline__ float p35_plus_2p23(uint32_t lo, uint32_t hi, uint32_t shift, const uint2* lutf) {
  const uint32_t k = bc4_index(lo, hi, shift);
  const uint32_t m8 = (lo & 0xffu) > ((lo >> 8) & 0xffu) ? 8u : 0u;
  const uint2 e = lutf[k | m8];
  return __uint_as_float(__dp2a_lo(e.x, lo, e.y));
}

// Feature gather for the tensor-core decode, whose features are rounded to
// FP16/BF16 right after: same taps and fractions as gather_f32, but the FP32
// arithmetic is reassociated.  P35 comes out of the dot product as the float
// 2^23 + P35 (lutf from init_p35_lut_f; one exact subtraction, no integer
// conversion), the 1/8925 scale is folded into the four bilinear weights, and
// the temporal rows are read 16 bytes at a time when the line is 16-byte
// aligned and its rows are whole 16-byte units.
template <int CS, int CT>
__device__ __forceinline__ void gather_tc(const DevModel& m, float u, float v, float t, float (&x)[CS + CT],
                                          const uint2* lutf) {
  static_assert(CS % 2 == 0, "planes are read in pairs");
  int x0, x1, y0, y1;
  float fx, fy;
  axis_setup(u, m.feat_w, m.address_mode, x0, x1, fx);
  axis_setup(v, m.feat_h, m.address_mode, y0, y1, fy);
  const int tx[4] = {x0, x1, x0, x1};
  const int ty[4] = {y0, y0, y1, y1};
  const uint4* line[4];
  uint32_t shift[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    line[q] = reinterpret_cast<const uint4*>(m.bc4 + ((size_t)(ty[q] >> 2) * m.bw + (tx[q] >> 2)) * CS * 8);
    shift[q] = 16u + 3u * (uint32_t)(((ty[q] & 3) << 2) | (tx[q] & 3));
  }
  const float gx = 1.0f - fx, gy = 1.0f - fy;
  const float wq[4] = {gx * gy * kInv8925, fx * gy * kInv8925, gx * fy * kInv8925, fx * fy * kInv8925};
  constexpr int G = CS < 8 ? CS : 8;
  const bool same_x = (x0 >> 2) == (x1 >> 2), same_y = (y0 >> 2) == (y1 >> 2);
#pragma unroll
  for (int c0 = 0; c0 < CS; c0 += G) {
    uint4 b[4][G / 2];
#pragma unroll
    for (int e = 0; e < G / 2; ++e) {
      b[0][e] = __ldg(line[0] + c0 / 2 + e);
      if (!same_x) b[1][e] = __ldg(line[1] + c0 / 2 + e);
      if (!same_y) b[2][e] = __ldg(line[2] + c0 / 2 + e);
      if (!same_x && !same_y) b[3][e] = __ldg(line[3] + c0 / 2 + e);
    }
#pragma unroll
    for (int e = 0; e < G / 2; ++e) {
      if (same_x) b[1][e] = b[0][e];
      if (same_y) b[2][e] = b[0][e];
      if (same_x || same_y) b[3][e] = same_x ? b[2][e] : b[1][e];
    }
#pragma unroll
    for (int e = 0; e < G / 2; ++e) {
      const int c = c0 + 2 * e;
      float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float p0 = p35_plus_2p23(b[q][e].x, b[q][e].y, shift[q], lutf) - 8388608.0f;
        const float p1 = p35_plus_2p23(b[q][e].z, b[q][e].w, shift[q], lutf) - 8388608.0f;
        a0 = fmaf(wq[q], p0, a0);
        a1 = fmaf(wq[q], p1, a1);
      }
      x[c] = a0;
      x[c + 1] = a1;
    }
  }
  int j0, j1;
  float a;
  temporal_setup(t, m.t_count, j0, j1, a);
  const float ga = 1.0f - a;
  const bool vec = (reinterpret_cast<uintptr_t>(m.temporal) & 15u) == 0u;
  if (CT % 8 == 0 && m.temporal_f16 && vec) {
    const uint4* r0 = reinterpret_cast<const uint4*>(static_cast<const __half*>(m.temporal) + (size_t)j0 * CT);
    const uint4* r1 = reinterpret_cast<const uint4*>(static_cast<const __half*>(m.temporal) + (size_t)j1 * CT);
#pragma unroll
    for (int g = 0; g < (CT % 8 == 0 ? CT / 8 : 0); ++g) {
      const uint4 k0 = __ldg(r0 + g), k1 = __ldg(r1 + g);
      const uint32_t w0[4] = {k0.x, k0.y, k0.z, k0.w}, w1[4] = {k1.x, k1.y, k1.z, k1.w};
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const float2 f0 = __half22float2(*reinterpret_cast<const __half2*>(&w0[h]));
        const float2 f1 = __half22float2(*reinterpret_cast<const __half2*>(&w1[h]));
        x[CS + 8 * g + 2 * h] = ga * f0.x + a * f1.x;
        x[CS + 8 * g + 2 * h + 1] = ga * f0.y + a * f1.y;
      }
    }
  } else if (CT % 4 == 0 && !m.temporal_f16 && vec) {
    const float4* r0 = reinterpret_cast<const float4*>(static_cast<const float*>(m.temporal) + (size_t)j0 * CT);
    const float4* r1 = reinterpret_cast<const float4*>(static_cast<const float*>(m.temporal) + (size_t)j1 * CT);
#pragma unroll
    for (int g = 0; g < (CT % 4 == 0 ? CT / 4 : 0); ++g) {
      const float4 k0 = __ldg(r0 + g), k1 = __ldg(r1 + g);
      x[CS + 4 * g] = ga * k0.x + a * k1.x;
      x[CS + 4 * g + 1] = ga * k0.y + a * k1.y;
      x[CS + 4 * g + 2] = ga * k0.z + a * k1.z;
      x[CS + 4 * g + 3] = ga * k0.w + a * k1.w;
    }
  } else {
#pragma unroll
    for (int c = 0; c < CT; ++c) {
      const float k0 = load_temporal(m.temporal, m.temporal_f16, j0 * CT + c);
      const float k1 = load_temporal(m.temporal, m.temporal_f16, j1 * CT + c);
      x[CS + c] = ga * k0 + a * k1;
    }
  }
}

}  // namespace ndgi
