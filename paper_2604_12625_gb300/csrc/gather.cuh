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
  temporal_setup_k(t, m.t_count, m.key_t, j0, j1, a);
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
  temporal_setup_k(t, m.t_count, m.key_t, j0, j1, a);
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

// ---------------------------------------------------------------------------
// Texel-sliced copy of the BC4 planes (built by ndgi_prepare for the tensor-
// core decodes).  The same information, regrouped per 4x4 block so that one
// texel of every plane is two short reads instead of a whole 128-byte line
// and a variable 64-bit shift per plane.  Block (by, bx) starts at
// (by * bw + bx) * BLOCK bytes:
//   [0, EP)          the (r0, r1) endpoint bytes of planes 0..CS-1 (plane c at
//                    bytes 2c, 2c+1), zero padded;
//   [EP, EP + 128)   16 words of 8 bytes: texel p's word holds, for plane c,
//                    the nibble (n8 << 3 | k) at bit 4c, k the texel's 3-bit
//                    index and n8 = 1 when r0 <= r1 (the block's palette mode,
//                    derived from its endpoints), i.e. the palette-table entry.
// ---------------------------------------------------------------------------
template <int CS>
struct Sliced {
  static_assert(CS <= 16, "at most 16 planes per sliced block");
  static constexpr int EP = CS <= 8 ? 16 : 32;
  static constexpr int BLOCK = EP + 128;
};

// Palette table for gather_sliced: entry (n8 << 3 | k) with n8 = 1 when
// r0 <= r1 (the six-value mode), constant term carrying 2^23's exponent bits
// as in init_p35_lut_f.
__device__ __forceinline__ void init_p35_lut_sliced(uint2* lut, int tid) {
  if (tid < 16) {
    const uint32_t k = tid & 7u;
    const bool m8 = tid < 8;   // n8 = 0: r0 > r1
    const uint32_t ca = __byte_perm(m8 ? kCa8Lo : kCa6Lo, m8 ? kCa8Hi : kCa6Hi, k) & 0xffu;
    const uint32_t cb = __byte_perm(m8 ? kCb8Lo : kCb6Lo, m8 ? kCb8Hi : kCb6Hi, k) & 0xffu;
    lut[tid] = make_uint2(ca | (cb << 16), ((!m8 && k == 7u) ? 8925u : 0u) + 0x4B000000u);
  }
}

// Plane c's palette-table entry (nibble at bit 4c of the texel word {lo, hi}).
template <int C>
__device__ __forceinline__ uint32_t nibble(uint2 w) {
  if constexpr (C < 8) return (w.x >> (4 * C)) & 15u;
  else return (w.y >> (4 * (C - 8))) & 15u;
}
__device__ __forceinline__ uint32_t nibble_at(uint2 w, int c) {
  return ((c < 8 ? w.x : w.y) >> (4 * (c & 7))) & 15u;
}

// Plane c's palette value at one tap, as the float 2^23 + P35: w is the
// endpoint word of planes 2*(c/2), 2*(c/2)+1, e its table entry.
template <int C>
__device__ __forceinline__ float sliced_value(uint32_t w, uint2 e) {
  if constexpr ((C & 1) == 0) return __uint_as_float(__dp2a_lo(e.x, w, e.y));
  else return __uint_as_float(__dp2a_hi(e.x, w, e.y));
}

template <int CS, int CT, int C>
__device__ __forceinline__ void sliced_plane(const uint32_t (&ew)[4][Sliced<CS>::EP / 4], const uint2 (&ix)[4],
                                             const float (&wq)[4], float (&x)[CS + CT], const uint2* lut) {
  if constexpr (C < CS) {
    float acc = 0.0f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float p = sliced_value<C>(ew[q][C / 2], lut[nibble<C>(ix[q])]) - 8388608.0f;
      acc = fmaf(wq[q], p, acc);
    }
    x[C] = acc;
    sliced_plane<CS, CT, C + 1>(ew, ix, wq, x, lut);
  }
}

// gather_tc on the texel-sliced copy `sl` (identical taps, fractions and P35).
template <int CS, int CT>
__device__ __forceinline__ void gather_sliced(const DevModel& m, const uint8_t* sl, float u, float v, float t,
                                              float (&x)[CS + CT], const uint2* lut) {
  using SL = Sliced<CS>;
  constexpr int EW = SL::EP / 16;   // uint4 endpoint words per block
  int x0, x1, y0, y1;
  float fx, fy;
  axis_setup(u, m.feat_w, m.address_mode, x0, x1, fx);
  axis_setup(v, m.feat_h, m.address_mode, y0, y1, fy);
  const int tx[4] = {x0, x1, x0, x1};
  const int ty[4] = {y0, y0, y1, y1};
  const float gx = 1.0f - fx, gy = 1.0f - fy;
  const float wq[4] = {gx * gy * kInv8925, fx * gy * kInv8925, gx * fy * kInv8925, fx * fy * kInv8925};
  const bool same_x = (x0 >> 2) == (x1 >> 2), same_y = (y0 >> 2) == (y1 >> 2);
  const uint8_t* base[4];
  uint2 ix[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    base[q] = sl + ((size_t)(ty[q] >> 2) * m.bw + (tx[q] >> 2)) * SL::BLOCK;
    const int p = ((ty[q] & 3) << 2) | (tx[q] & 3);
    ix[q] = __ldg(reinterpret_cast<const uint2*>(base[q] + SL::EP) + p);
  }
  uint4 e[4][EW];
#pragma unroll
  for (int h = 0; h < EW; ++h) {
    e[0][h] = __ldg(reinterpret_cast<const uint4*>(base[0]) + h);
    if (!same_x) e[1][h] = __ldg(reinterpret_cast<const uint4*>(base[1]) + h);
    if (!same_y) e[2][h] = __ldg(reinterpret_cast<const uint4*>(base[2]) + h);
    if (!same_x && !same_y) e[3][h] = __ldg(reinterpret_cast<const uint4*>(base[3]) + h);
  }
#pragma unroll
  for (int h = 0; h < EW; ++h) {
    if (same_x) e[1][h] = e[0][h];
    if (same_y) e[2][h] = e[0][h];
    if (same_x || same_y) e[3][h] = same_x ? e[2][h] : e[1][h];
  }
  uint32_t ew[4][SL::EP / 4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
#pragma unroll
    for (int h = 0; h < EW; ++h) {
      ew[q][4 * h] = e[q][h].x;
      ew[q][4 * h + 1] = e[q][h].y;
      ew[q][4 * h + 2] = e[q][h].z;
      ew[q][4 * h + 3] = e[q][h].w;
    }
  }
  sliced_plane<CS, CT, 0>(ew, ix, wq, x, lut);
  int j0, j1;
  float a;
  temporal_setup_k(t, m.t_count, m.key_t, j0, j1, a);
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
      for (int hh = 0; hh < 4; ++hh) {
        const float2 f0 = __half22float2(*reinterpret_cast<const __half2*>(&w0[hh]));
        const float2 f1 = __half22float2(*reinterpret_cast<const __half2*>(&w1[hh]));
        x[CS + 8 * g + 2 * hh] = ga * f0.x + a * f1.x;
        x[CS + 8 * g + 2 * hh + 1] = ga * f0.y + a * f1.y;
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

// Builds the texel-sliced copy of the BC4 planes (one thread per block).
template <int CS>
__global__ void k_slice_features(const uint8_t* __restrict__ bc4, int64_t nblocks, uint8_t* __restrict__ out) {
  using SL = Sliced<CS>;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nblocks; i += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t* src = bc4 + i * CS * 8;
    uint8_t* dst = out + i * SL::BLOCK;
    uint32_t ep[SL::EP / 4];
#pragma unroll
    for (int w = 0; w < SL::EP / 4; ++w) ep[w] = 0u;
    uint64_t idx[16];
#pragma unroll
    for (int p = 0; p < 16; ++p) idx[p] = 0u;
#pragma unroll
    for (int c = 0; c < CS; ++c) {
      uint64_t b = 0;
#pragma unroll
      for (int k = 0; k < 8; ++k) b |= (uint64_t)src[c * 8 + k] << (8 * k);
      ep[c / 2] |= (uint32_t)(b & 0xFFFFu) << (16 * (c & 1));
      const uint64_t n8 = (b & 0xFFu) <= ((b >> 8) & 0xFFu) ? 8u : 0u;   // r0 <= r1: six-value palette
#pragma unroll
      for (int p = 0; p < 16; ++p) idx[p] |= (((b >> (16 + 3 * p)) & 7u) | n8) << (4 * c);
    }
#pragma unroll
    for (int w = 0; w < SL::EP / 16; ++w)
      reinterpret_cast<uint4*>(dst)[w] = make_uint4(ep[4 * w], ep[4 * w + 1], ep[4 * w + 2], ep[4 * w + 3]);
#pragma unroll
    for (int p = 0; p < 16; ++p)
      reinterpret_cast<uint2*>(dst + SL::EP)[p] = make_uint2((uint32_t)idx[p], (uint32_t)(idx[p] >> 32));
  }
}

}  // namespace ndgi
