// Device helpers for the BC4 feature gather: block decode, texel-centre
// bilinear setup and the periodic temporal lerp setup.
//
// BC4 palette (the block form of Sec. 3.4, Eq. 7 / supplement S2 with the
// BC4 interpolant grid): a block holds r0, r1 and sixteen 3-bit indices.
// If r0 > r1 the palette is r0, r1 and ((8-k) r0 + (k-1) r1)/7 for k = 2..7;
// otherwise r0, r1, ((6-k) r0 + (k-1) r1)/5 for k = 2..5, then 0 and 255.
// Values are kept as the integer numerator P35 over 8925 = 35*255, so
// P35 = ca(k)*r0 + cb(k)*r1 + cc(k) with small integer coefficients; the
// coefficient of each index is fetched with a byte permute from packed
// tables (one table pair per mode).  The feature value is P35 * (1/8925)
// rounded once in FP32.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cstdint>

namespace ndgi {

// Coefficient tables, byte k = coefficient of index k.
//   eight-value mode: ca = 35,0,30,25,20,15,10,5   cb = 0,35,5,10,15,20,25,30
//   six-value mode:   ca = 35,0,28,21,14,7,0,0     cb = 0,35,7,14,21,28,0,0  (+8925 at k=7)
constexpr uint32_t kCa8Lo = 0x191E0023u, kCa8Hi = 0x050A0F14u;
constexpr uint32_t kCb8Lo = 0x0A052300u, kCb8Hi = 0x1E19140Fu;
constexpr uint32_t kCa6Lo = 0x151C0023u, kCa6Hi = 0x0000070Eu;
constexpr uint32_t kCb6Lo = 0x0E072300u, kCb6Hi = 0x00001C15u;
constexpr float kInv8925 = 1.0f / 8925.0f;

// 3-bit index at bit `shift` (= 16 + 3p) of the 64-bit block {lo, hi}.
__device__ __forceinline__ uint32_t bc4_index(uint32_t lo, uint32_t hi, uint32_t shift) {
  const uint64_t bits = ((uint64_t)hi << 32) | lo;
  return (uint32_t)(bits >> shift) & 7u;
}

// Palette numerator of texel p of block {lo, hi} (shift = 16 + 3p).
__device__ __forceinline__ int bc4_p35(uint32_t lo, uint32_t hi, uint32_t shift) {
  const uint32_t r0 = lo & 0xffu, r1 = (lo >> 8) & 0xffu;
  const uint32_t k = bc4_index(lo, hi, shift);
  const bool m8 = r0 > r1;
  const uint32_t ca = __byte_perm(m8 ? kCa8Lo : kCa6Lo, m8 ? kCa8Hi : kCa6Hi, k) & 0xffu;
  const uint32_t cb = __byte_perm(m8 ? kCb8Lo : kCb6Lo, m8 ? kCb8Hi : kCb6Hi, k) & 0xffu;
  const uint32_t cc = (!m8 && k == 7u) ? 8925u : 0u;
  return (int)(ca * r0 + cb * r1 + cc);
}

// Table form of the same palette for kernels that keep a 16-entry table in
// shared memory: entry (m8 << 3 | k) holds {ca | cb << 16, cc} (m8 = 1 when
// r0 > r1), so P35 = ca*r0 + cb*r1 + cc is one 2-way byte dot product of the
// block's low word (bytes r0, r1) with the packed coefficients.
__device__ __forceinline__ void init_p35_lut(uint2* lut, int tid) {
  if (tid < 16) {
    const uint32_t k = tid & 7u;
    const bool m8 = tid >= 8;
    const uint32_t ca = __byte_perm(m8 ? kCa8Lo : kCa6Lo, m8 ? kCa8Hi : kCa6Hi, k) & 0xffu;
    const uint32_t cb = __byte_perm(m8 ? kCb8Lo : kCb6Lo, m8 ? kCb8Hi : kCb6Hi, k) & 0xffu;
    lut[tid] = make_uint2(ca | (cb << 16), (!m8 && k == 7u) ? 8925u : 0u);
  }
}

__device__ __forceinline__ int bc4_p35_lut(uint32_t lo, uint32_t hi, uint32_t shift, const uint2* lut) {
  const uint32_t k = bc4_index(lo, hi, shift);
  const uint32_t m8 = (lo & 0xffu) > ((lo >> 8) & 0xffu) ? 8u : 0u;
  const uint2 e = lut[k | m8];
  return (int)__dp2a_lo(e.x, lo, e.y);
}

__device__ __forceinline__ float p35_value(int p35) {
  return __fmul_rn(__int2float_rn(p35), kInv8925);
}

// Maps a texel index into [0, n): clamp (mode 0) or mirrored repeat (mode 1).
__device__ __forceinline__ int address(int i, int n, int mode) {
  if (mode == 1) {
    const int period = 2 * n;
    int r = i % period;
    if (r < 0) r += period;
    return r < n ? r : period - 1 - r;
  }
  return min(max(i, 0), n - 1);
}

// Texel-centre sampling along one axis: x = coord*size - 0.5, taps floor(x)
// and floor(x)+1, fraction x - floor(x).  coord*size is split into a rounded
// product and its exact FMA residual, and the rounding error of the -0.5 is
// carried too, so the fraction is exact whenever the product is (always for
// power-of-two sizes) and within one rounding otherwise.
__device__ __forceinline__ void axis_setup(float coord, int size, int mode, int& t0, int& t1, float& frac) {
  const float fs = (float)size;
  const float hi = __fmul_rn(coord, fs);
  const float lo = __fmaf_rn(coord, fs, -hi);
  const float x = __fsub_rn(hi, 0.5f);
  const float xe = __fsub_rn(-0.5f, __fsub_rn(x, hi));   // rounding error of hi - 0.5 (0 when hi >= 0.25)
  float fl = floorf(x);
  float fr = __fadd_rn(__fsub_rn(x, fl), __fadd_rn(lo, xe));
  if (fr >= 1.0f) {
    fl = __fadd_rn(fl, 1.0f);
    fr = __fsub_rn(fr, 1.0f);
  } else if (fr < 0.0f) {
    fl = __fsub_rn(fl, 1.0f);
    fr = __fadd_rn(fr, 1.0f);
  }
  fl = fminf(fmaxf(fl, -1073741824.0f), 1073741824.0f);   // NaN -> lower bound, keeps ints finite
  if (!(fr >= 0.0f && fr <= 1.0f)) fr = 0.0f;
  const int i = (int)fl;
  t0 = address(i, size, mode);
  t1 = address(i + 1, size, mode);
  frac = fr;
}

// Periodic temporal setup: s = t*T, rows j = floor(s) mod T and (j+1) mod T,
// weight alpha = s - floor(s); the product is split as in axis_setup.
__device__ __forceinline__ void temporal_setup(float t, int T, int& j0, int& j1, float& alpha) {
  const float fT = (float)T;
  const float hi = __fmul_rn(t, fT);
  const float lo = __fmaf_rn(t, fT, -hi);
  float fl = floorf(hi);
  float fr = __fadd_rn(__fsub_rn(hi, fl), lo);
  if (fr >= 1.0f) {
    fl = __fadd_rn(fl, 1.0f);
    fr = __fsub_rn(fr, 1.0f);
  } else if (fr < 0.0f) {
    fl = __fsub_rn(fl, 1.0f);
    fr = __fadd_rn(fr, 1.0f);
  }
  fl = fminf(fmaxf(fl, -1073741824.0f), 1073741824.0f);
  if (!(fr >= 0.0f && fr <= 1.0f)) fr = 0.0f;
  int j = (int)fl % T;
  if (j < 0) j += T;
  j0 = j;
  j1 = (j + 1 == T) ? 0 : j + 1;
  alpha = fr;
}

// The same with keyframes at given times 0 <= key_t[0] < ... < key_t[T-1] < 1
// (Sec. 3.1 allows non-uniform times), periodic with period 1: t lies in the
// segment [key_t[j], key_t[j1]) (the last one runs from key_t[T-1] to
// key_t[0] + 1) and alpha is its position there.  key_t == nullptr: uniform
// keyframes j/T (temporal_setup).  The search takes at most log2(T) steps
// and stays in bounds whatever the times hold.
__device__ __forceinline__ void temporal_setup_k(float t, int T, const float* key_t, int& j0, int& j1, float& alpha) {
  if (key_t == nullptr) {
    temporal_setup(t, T, j0, j1, alpha);
    return;
  }
  float s = __fsub_rn(t, floorf(t));
  if (!(s >= 0.0f && s < 1.0f)) s = 0.0f;   // not finite, or t just below an integer (s rounds to 1)
  const float k0 = __ldg(key_t);
  int j = -1;
  if (s >= k0) {   // largest j with key_t[j] <= s
    int lo = 0, hi = T - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(key_t + mid) <= s) lo = mid;
      else hi = mid - 1;
    }
    j = lo;
  }
  float start, end;
  if (j < 0 || j == T - 1) {   // the wrap segment
    start = __ldg(key_t + T - 1);
    end = __fadd_rn(k0, 1.0f);
    if (j < 0) s = __fadd_rn(s, 1.0f);
    j = T - 1;
  } else {
    start = __ldg(key_t + j);
    end = __ldg(key_t + j + 1);
  }
  j0 = j;
  j1 = j + 1 == T ? 0 : j + 1;
  alpha = fminf(fmaxf(__fdiv_rn(__fsub_rn(s, start), __fsub_rn(end, start)), 0.0f), 1.0f);
}

__device__ __forceinline__ float load_temporal(const void* base, int f16, int idx) {
  if (f16) return __half2float(reinterpret_cast<const __half*>(base)[idx]);
  return reinterpret_cast<const float*>(base)[idx];
}

// Straight-through quantiser decision q_s(x) = floor(min(max(s*x + 0.5, 0), s)),
// each operation rounded once in FP32 (no contraction).
__device__ __forceinline__ int quant(float x, float s) {
  float y = __fmul_rn(s, x);
  y = __fadd_rn(y, 0.5f);
  y = fmaxf(y, 0.0f);
  y = fminf(y, s);
  return (int)floorf(y);
}

}  // namespace ndgi
