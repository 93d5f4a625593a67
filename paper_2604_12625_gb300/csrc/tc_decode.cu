// Tensor-core decode: the decoder MLP on tcgen05 (FP16 or BF16 operands,
// FP32 accumulation in tensor memory), for random points and for batched
// virtual-texture pages; the page decode also runs with FP8 (E4M3) weights
// and activations (kind::f8f6f4).
//
// Structure.  A CTA holds NWG independent "lanes" (warpgroups of 4 warps).
// A lane owns one 128-row MMA tile at a time in a slot of tensor memory: its
// 128 threads write the tile's layer-1 rows (one row each) into the slot's
// columns with tcgen05.st, one thread issues the layer's tcgen05.mma chain
// (A from tensor memory, the small weight tile B from shared memory) and
// commits to the slot's mbarrier, and the 128 threads read their rows of the
// FP32 accumulator back (tcgen05.ld), apply ReLU with the FP16/BF16
// conversion in one instruction, and write the next layer's A rows.  Layer 3
// of a tile is issued together with layer 1 of the lane's next tile, so a tile
// costs two dependent MMA round trips.  The MLP weights are shared by the
// lanes; the lanes of a CTA interleave, so one lane's gather and epilogues
// overlap the others' MMAs.
//
// Biases ride in the MMA: an A tile carries a ones column in its K padding
// and the matching B row holds the bias, so the MMA adds it.  The exception
// is b3 of the FP16/BF16 paths (the same stored value), added in FP32 when the
// layer-3 accumulator is read: it frees layer 3's last K step and the TMEM
// columns that let layer 3 share a commit with the next layer 1.
// For pages, t is constant per request, so the temporal part of layer 1 is
// folded into a per-request bias b1' = b1 + W1_t v_t (FP32), stored in B1 as
// a hi + lo pair of FP16/BF16 values against two ones columns; layer 1 then
// contracts only the 16 spatial channels plus those two columns (K = 32).
//
// Page features: a lane decodes each BC4 feature row of its page quadrant
// once (exact integer palette numerator from a 16-entry table and a byte dot
// product, scaled once in FP32, stored as FP16) into a 16-row ring in shared
// memory, in batches of up to 8 rows, and blends the four taps of each texel
// with packed half2 arithmetic from there.
//
// FP8 pages.  Every scale is a power of two (see k_tc_prepare8), chosen so that
// a layer's FP32 accumulator is already in the next layer's activation unit:
// the epilogue is then one ReLU + E4M3 conversion per pair of values, exactly
// like the FP16 one.  Biases ride in the K padding as three E4M3 terms against
// ones columns of value v (a power of two), which keeps about 12 significant
// bits of each bias.
//
// Every mbarrier wait is bounded; a timeout is latched in a device error word
// that ndgi_check reports, and the CTA unwinds and frees its tensor memory.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>
#include <type_traits>

#include "ndgi_internal.h"
#include "bc4.cuh"
#include "gather.cuh"
#include "tc_decode.h"
#include "umma.cuh"

namespace ndgi {

// Device error word of the tensor-core kernels (bit 0: an mbarrier wait timed out).
static __device__ int g_tc_error;

constexpr int kLaneThreads = 128;

// Operand kinds of the tensor-core decode.
constexpr int kF16 = 0, kBF16 = 1, kE4M3 = 2;

// ---------------------------------------------------------------------------
// Weight image (built by ndgi_prepare), identical layout in global and shared
// memory so a CTA copies it with 16-byte loads.
// ---------------------------------------------------------------------------
template <int CS, int CT, int H>
struct TcLayout {
  static constexpr int CIN = CS + CT;
  static constexpr int K1P = ((CIN + 1 + 15) / 16) * 16;   // points: inputs + ones column (b1)
  static constexpr int K1G = ((CS + 2 + 15) / 16) * 16;    // pages: spatial channels + two ones columns (b1' hi, lo)
  static constexpr int K2 = H + 16;                        // hidden + ones column (b2 / b3)
  static constexpr int N3 = 16;                            // output layer N (3 used)
  static constexpr uint32_t kB2 = 0;                       // [H][K2]     K-major, column H = b2
  static constexpr uint32_t kB3 = kB2 + H * K2 * 2;        // [16][K2]    rows 3..15 zero, column H = b3
  static constexpr uint32_t kShared = kB3 + N3 * K2 * 2;   // end of the part both kernels use
  static constexpr uint32_t kB1P = kShared;                // [H][K1P]    points layer 1, column CIN = b1
  static constexpr uint32_t kB1G = kB1P + H * K1P * 2;     // [H][K1G]    pages layer 1 (spatial; bias columns per request)
  static constexpr uint32_t kW1T = kB1G + H * K1G * 2;     // [CT][H] f32 stored temporal weights
  static constexpr uint32_t kB1 = kW1T + CT * H * 4;       // [H] f32 stored b1
  static constexpr uint32_t kWsBytes = kB1 + H * 4;
  static constexpr uint32_t kSliceOff = (kWsBytes + 255) / 256 * 256;   // then the texel-sliced BC4 copy (points)
  static constexpr int EB = 2;                             // bytes per operand element
  static constexpr uint32_t kTmemCols = H <= 32 ? 32 : (H <= 64 ? 64 : 128);
  static_assert(H % 16 == 0 && H <= 128, "hidden width must be a multiple of 16, at most 128");
  static_assert(kShared % 16 == 0 && kB1G % 16 == 0 && kW1T % 16 == 0, "16-byte granular image");
};

// FP8 scales of one model (the tail of its FP8 image), all powers of two:
// layer-1 inputs are quantised in units a1, layer-1 outputs (= layer-2
// inputs) are in units a2, the RGB accumulator in units `out`.
struct Fp8Scales {
  float a1, inv_a1, inv_a2, out;
  uint32_t ones2, ones3;   // A-side ones word of layers 2 / 3: E4M3 code of v in bytes 0..2, byte 3 zero
  float a2;
  uint32_t status;         // bit 0: a bias needs a ones value above 256; bit 1: 1/a1 too large for FP16
  float s1, s2, s3, a3;    // weight scales and the layer-2 output unit
  float v2, v3, pad0, pad1;
};
static_assert(sizeof(Fp8Scales) == 64, "FP8 scale block");

// FP8 (E4M3) image for the page decode: one-byte codes, a K step of 32.
// Layer 1 contracts the 16 spatial channels plus three ones columns that
// carry the per-request bias b1' (K = 32); layers 2 and 3 carry their biases
// the same way in K2 = H + 32.
template <int CS, int CT, int H>
struct TcLayout8 {
  static constexpr int EB = 1;
  static constexpr int K1G = 32;
  static constexpr int K2 = H + 32;
  static constexpr int N3 = 16;
  static constexpr uint32_t kB2 = 0;                       // [H][K2]  codes of W2^T / s2; columns H..H+2 = b2 terms
  static constexpr uint32_t kB3 = kB2 + H * K2;            // [16][K2] codes of W3^T / s3; columns H..H+2 = b3 terms
  static constexpr uint32_t kShared = kB3 + N3 * K2;
  static constexpr uint32_t kB1G = kShared;                // [H][K1G] codes of W1_s^T / s1; b1' terms per request
  static constexpr uint32_t kW1T = kB1G + H * K1G;         // [CT][H] f32 stored temporal weights s1 e4m3(W1_t / s1)
  static constexpr uint32_t kB1 = kW1T + CT * H * 4;       // [H] f32 b1
  static constexpr uint32_t kScale = kB1 + H * 4;          // Fp8Scales
  static constexpr uint32_t kWsBytes = kScale + sizeof(Fp8Scales);
  static constexpr uint32_t kSliceOff = (kWsBytes + 255) / 256 * 256;   // then the texel-sliced BC4 copy
  static_assert(CS + 3 <= K1G && H % 32 == 0 && H <= 128, "FP8 pages: cs <= 29, hidden a multiple of 32");
  static_assert(kShared % 16 == 0 && kW1T % 16 == 0 && kScale % 16 == 0 && kWsBytes % 16 == 0, "granularity");
};

// ---- E4M3 helpers ----------------------------------------------------------
// Two floats -> two E4M3 codes (nearest even, saturating at +-448), `lo` in bits 0..7.
__device__ __forceinline__ uint32_t e4m3x2(float lo, float hi) {
  uint16_t d;
  asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(d) : "f"(hi), "f"(lo));
  return d;
}
__device__ __forceinline__ uint32_t e4m3x2_relu(float lo, float hi) {
  uint16_t d;
  asm("cvt.rn.satfinite.relu.e4m3x2.f32 %0, %1, %2;" : "=h"(d) : "f"(hi), "f"(lo));
  return d;
}
// Packed half2 -> two E4M3 codes, the low half in bits 0..7.
__device__ __forceinline__ uint32_t e4m3x2_h(uint32_t h2) {
  uint16_t d;
  asm("cvt.rn.satfinite.e4m3x2.f16x2 %0, %1;" : "=h"(d) : "r"(h2));
  return d;
}
// Value of an E4M3 code, from the format (exact in FP32): exponent field e,
// mantissa m: (1 + m/8) 2^(e-7), or m/8 2^-6 when e = 0.
__device__ __forceinline__ float e4m3_value(uint32_t c) {
  const uint32_t e = (c >> 3) & 15u, m = c & 7u;
  const float v = e == 0 ? (float)m * 0x1p-9f : __uint_as_float(((e + 120u) << 23) | (m << 20));
  return (c & 0x80u) ? -v : v;
}
// Smallest power of two P with y <= 448 P (1 for y <= 0 or not finite); the
// comparisons are exact.
__device__ float fp8_p2(float y) {
  if (!(y > 0.0f) || !(y <= 3.4e38f)) return 1.0f;
  int e;
  frexpf(y / 448.0f, &e);
  float P = ldexpf(1.0f, e);
  while (y > 448.0f * P) P *= 2.0f;
  while (y <= 448.0f * (P * 0.5f)) P *= 0.5f;
  return P;
}
// beta / v as three E4M3 terms t1 + t2 + t3 (each the rounding of what the
// previous terms left; the residuals are exact in FP32): codes in bytes 0..2.
__device__ uint32_t fp8_terms(float beta, float v) {
  const float r0 = beta * (1.0f / v);
  const uint32_t c1 = e4m3x2(r0, 0.0f) & 0xFFu;
  const float r1 = __fsub_rn(r0, e4m3_value(c1));
  const uint32_t c2 = e4m3x2(r1, 0.0f) & 0xFFu;
  const float r2 = __fsub_rn(r1, e4m3_value(c2));
  const uint32_t c3 = e4m3x2(r2, 0.0f) & 0xFFu;
  return c1 | (c2 << 8) | (c3 << 16);
}
// E4M3 code of a power of two 2^k, k in -6..8.
__device__ __forceinline__ uint32_t e4m3_pow2_code(float v) {
  int e;
  frexpf(v, &e);
  return (uint32_t)(e - 1 + 7) << 3;
}

template <bool BF16>
__device__ __forceinline__ uint16_t to_bits(float x) {
  if (BF16) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    return *reinterpret_cast<const uint16_t*>(&h);
  }
  const __half h = __float2half_rn(x);
  return *reinterpret_cast<const uint16_t*>(&h);
}

template <bool BF16>
__device__ __forceinline__ float round_stored(float x) {
  if (BF16) return __bfloat162float(__float2bfloat16_rn(x));
  return __half2float(__float2half_rn(x));
}

// Two floats -> packed pair, `lo` in the low half.
template <bool BF16>
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  uint32_t d;
  if (BF16) asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  else asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}
// Same with ReLU fused into the conversion.
template <bool BF16>
__device__ __forceinline__ uint32_t pack2_relu(float lo, float hi) {
  uint32_t d;
  if (BF16) asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  else asm("cvt.rn.relu.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

// Stored b3 of an FP16/BF16 image (column H of the B3 tile) as FP32.
template <bool BF16>
__device__ __forceinline__ float stored_b3(const unsigned char* b3_img, int n, int H, int K2) {
  const uint16_t b = *reinterpret_cast<const uint16_t*>(b3_img + kmajor_offset(n, H, K2));
  if (BF16) return __uint_as_float((uint32_t)b << 16);
  return __half2float(__ushort_as_half(b));
}

template <int CS, int CT, int H, bool BF16>
__global__ void k_tc_prepare(DevModel m, unsigned char* __restrict__ ws) {
  using L = TcLayout<CS, CT, H>;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
  for (int i = tid; i < H * L::K2; i += nt) {      // B2[n][k] = W2[k][n], column H = b2
    const int n = i / L::K2, k = i % L::K2;
    const float v = k < H ? m.w2[k * H + n] : (k == H ? m.b2[n] : 0.0f);
    *reinterpret_cast<uint16_t*>(ws + L::kB2 + kmajor_offset(n, k, L::K2)) = to_bits<BF16>(v);
  }
  for (int i = tid; i < L::N3 * L::K2; i += nt) {  // B3[n][k] = W3[k][n], column H = b3
    const int n = i / L::K2, k = i % L::K2;
    const float v = n >= 3 ? 0.0f : (k < H ? m.w3[k * 3 + n] : (k == H ? m.b3[n] : 0.0f));
    *reinterpret_cast<uint16_t*>(ws + L::kB3 + kmajor_offset(n, k, L::K2)) = to_bits<BF16>(v);
  }
  for (int i = tid; i < H * L::K1P; i += nt) {     // points: B1[n][k] = W1[k][n], column CIN = b1
    const int n = i / L::K1P, k = i % L::K1P;
    const float v = k < L::CIN ? m.w1[k * H + n] : (k == L::CIN ? m.b1[n] : 0.0f);
    *reinterpret_cast<uint16_t*>(ws + L::kB1P + kmajor_offset(n, k, L::K1P)) = to_bits<BF16>(v);
  }
  for (int i = tid; i < H * L::K1G; i += nt) {     // pages: spatial rows of W1; bias columns filled per request
    const int n = i / L::K1G, k = i % L::K1G;
    *reinterpret_cast<uint16_t*>(ws + L::kB1G + kmajor_offset(n, k, L::K1G)) =
        to_bits<BF16>(k < CS ? m.w1[k * H + n] : 0.0f);
  }
  for (int i = tid; i < CT * H; i += nt)
    reinterpret_cast<float*>(ws + L::kW1T)[i] = round_stored<BF16>(m.w1[(CS + i / H) * H + i % H]);
  for (int i = tid; i < H; i += nt) reinterpret_cast<float*>(ws + L::kB1)[i] = round_stored<BF16>(m.b1[i]);
}

// FP8 image from the FP32 master weights and the calibration maxima
// m1 = max|layer-1 input|, m2 = max relu(z1), m3 = max relu(z2).  With p2(y) the
// smallest power of two P with y <= 448 P:
//   a1 = p2(m1), s1 = p2(max(max|W1|, m2/a1)), a2 = a1 s1,
//   s2 = p2(max(max|W2|, m3/a2)), a3 = a2 s2, s3 = p2(max|W3|), out = a3 s3.
// Weights are stored as codes of W_l / s_l; a layer's accumulator is then the
// layer output in units a_(l+1).  Bias b of a layer with output unit u:
// v = max(1, p2(max|b/u|)) and the codes of the three terms of b/u/v.
// One CTA of 256 threads.
template <int CS, int CT, int H>
__global__ void __launch_bounds__(256) k_tc_prepare8(DevModel m, float m1, float m2, float m3,
                                                     unsigned char* __restrict__ ws) {
  using L = TcLayout8<CS, CT, H>;
  constexpr int CIN = CS + CT;
  __shared__ unsigned int s_max[5];   // float bits (non-negative): |W1|, |W2|, |W3|, |b2/a3|, |b3/out|
  __shared__ float s_sc[8];           // a1, s1, a2, s2, a3, s3, out, -
  __shared__ float s_v[2];            // v2, v3
  const int tid = threadIdx.x;
  if (tid < 5) s_max[tid] = 0u;
  __syncthreads();
  float w1 = 0.0f, w2 = 0.0f, w3 = 0.0f;
  for (int i = tid; i < CIN * H; i += 256) w1 = fmaxf(w1, fabsf(m.w1[i]));
  for (int i = tid; i < H * H; i += 256) w2 = fmaxf(w2, fabsf(m.w2[i]));
  for (int i = tid; i < H * 3; i += 256) w3 = fmaxf(w3, fabsf(m.w3[i]));
  atomicMax(&s_max[0], __float_as_uint(w1));
  atomicMax(&s_max[1], __float_as_uint(w2));
  atomicMax(&s_max[2], __float_as_uint(w3));
  __syncthreads();
  if (tid == 0) {
    const float a1 = fp8_p2(m1);
    const float s1 = fp8_p2(fmaxf(__uint_as_float(s_max[0]), m2 / a1)), a2 = a1 * s1;
    const float s2 = fp8_p2(fmaxf(__uint_as_float(s_max[1]), m3 / a2)), a3 = a2 * s2;
    const float s3 = fp8_p2(__uint_as_float(s_max[2]));
    s_sc[0] = a1; s_sc[1] = s1; s_sc[2] = a2; s_sc[3] = s2; s_sc[4] = a3; s_sc[5] = s3; s_sc[6] = a3 * s3;
  }
  __syncthreads();
  const float s1 = s_sc[1], s2 = s_sc[3], s3 = s_sc[5], a3 = s_sc[4], out = s_sc[6];
  if (tid < H) atomicMax(&s_max[3], __float_as_uint(fabsf(m.b2[tid] / a3)));
  if (tid < 3) atomicMax(&s_max[4], __float_as_uint(fabsf(m.b3[tid] / out)));
  __syncthreads();
  if (tid == 0) {
    const float v2 = fmaxf(1.0f, fp8_p2(__uint_as_float(s_max[3]))), v3 = fmaxf(1.0f, fp8_p2(__uint_as_float(s_max[4])));
    s_v[0] = v2;
    s_v[1] = v3;
    Fp8Scales sc;
    sc.a1 = s_sc[0];
    sc.inv_a1 = 1.0f / s_sc[0];
    sc.inv_a2 = 1.0f / s_sc[2];
    sc.out = out;
    const uint32_t c2 = e4m3_pow2_code(fminf(v2, 256.0f)), c3 = e4m3_pow2_code(fminf(v3, 256.0f));
    sc.ones2 = c2 | (c2 << 8) | (c2 << 16);
    sc.ones3 = c3 | (c3 << 8) | (c3 << 16);
    sc.a2 = s_sc[2];
    sc.status = (v2 > 256.0f || v3 > 256.0f ? 1u : 0u) | (sc.inv_a1 > 16384.0f ? 2u : 0u);
    sc.s1 = s_sc[1];
    sc.s2 = s_sc[3];
    sc.s3 = s_sc[5];
    sc.a3 = s_sc[4];
    sc.v2 = v2;
    sc.v3 = v3;
    sc.pad0 = sc.pad1 = 0.0f;
    *reinterpret_cast<Fp8Scales*>(ws + L::kScale) = sc;
  }
  __syncthreads();
  const float v2 = s_v[0], v3 = s_v[1];
  for (int i = tid; i < H * L::K2; i += 256) {      // B2[n][k]: W2[k][n] / s2, then the b2 terms
    const int n = i / L::K2, k = i % L::K2;
    uint32_t c = 0u;
    if (k < H) c = e4m3x2(m.w2[k * H + n] * (1.0f / s2), 0.0f) & 0xFFu;
    else if (k < H + 3) c = (fp8_terms(m.b2[n] / a3, v2) >> (8 * (k - H))) & 0xFFu;
    ws[L::kB2 + kmajor_offset8(n, k, L::K2)] = (unsigned char)c;
  }
  for (int i = tid; i < L::N3 * L::K2; i += 256) {  // B3[n][k]: W3[k][n] / s3, then the b3 terms
    const int n = i / L::K2, k = i % L::K2;
    uint32_t c = 0u;
    if (n < 3 && k < H) c = e4m3x2(m.w3[k * 3 + n] * (1.0f / s3), 0.0f) & 0xFFu;
    else if (n < 3 && k < H + 3) c = (fp8_terms(m.b3[n] / out, v3) >> (8 * (k - H))) & 0xFFu;
    ws[L::kB3 + kmajor_offset8(n, k, L::K2)] = (unsigned char)c;
  }
  for (int i = tid; i < H * L::K1G; i += 256) {     // B1[n][k]: spatial W1[k][n] / s1; bias columns per request
    const int n = i / L::K1G, k = i % L::K1G;
    const uint32_t c = k < CS ? e4m3x2(m.w1[k * H + n] * (1.0f / s1), 0.0f) & 0xFFu : 0u;
    ws[L::kB1G + kmajor_offset8(n, k, L::K1G)] = (unsigned char)c;
  }
  for (int i = tid; i < CT * H; i += 256)
    reinterpret_cast<float*>(ws + L::kW1T)[i] =
        s1 * e4m3_value(e4m3x2(m.w1[(CS + i / H) * H + i % H] * (1.0f / s1), 0.0f) & 0xFFu);
  for (int i = tid; i < H; i += 256) reinterpret_cast<float*>(ws + L::kB1)[i] = m.b1[i];
}

// ---------------------------------------------------------------------------
// tcgen05 helpers specific to this file
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&r)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
}
// Barrier over the 128 threads of lane `wg` (ids 1.. ; 0 is __syncthreads).
__device__ __forceinline__ void lane_sync(int wg) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + wg), "r"(kLaneThreads) : "memory");
}
// Lane barrier that also returns whether any of the lane's threads passed v = true.
__device__ __forceinline__ bool lane_any(int wg, bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(1 + wg), "r"(kLaneThreads)
      : "memory");
  return r != 0;
}
constexpr uint32_t tmem_alloc_cols(int cols) {
  return cols <= 32 ? 32u : (cols <= 64 ? 64u : (cols <= 128 ? 128u : (cols <= 256 ? 256u : 512u)));
}

// ---------------------------------------------------------------------------
// One lane's MLP engine with SL tile slots.
//
// A slot is one 128-row tile in flight: a region of tensor memory and an
// mbarrier.  Its columns (FP16 example, H = 64):
//   [0, H)             accumulator D of layers 1 and 2 (FP32)
//   [H, H + K2/2)      A operand of layer 2 (ReLU(H1), then the ones column
//                      that carries b2 in the K padding) and of layer 3
//                      (ReLU(H2) only: b3 is added when D3 is read)
//   [kD3Col, +16)      layer-3 accumulator (N = 16, 3 used)
//   [kA1Col, ...)      A operand of layer 1 (features, bias ones columns)
// Layer 3 of a tile and layer 1 of the slot's next tile touch disjoint
// columns, so they are issued back to back under one commit: a tile costs
// two MMA round trips (layer 1 with the previous tile's layer 3, then
// layer 2), not three.  D3 shares columns with the tail of the layer-2 A
// region only across time: each thread reads its D3 row before it writes
// its next layer-2 row.
// All operands but the small weight tiles B live in tensor memory, written
// from registers with tcgen05.st.  Every thread of the lane waits on the
// slot's mbarrier itself (no barrier round trip after completion); a wait
// that times out is carried to the lane's next barrier, where the lane
// decides uniformly to stop.  The thread that issues (one per lane, in a
// different warp of each lane so the four issuers sit on different SM
// sub-partitions) waits like the others.
// P: kF16 / kBF16 (kind::f16, K step 16) or kE4M3 (kind::f8f6f4, K step 32);
// either way a K step is 32 bytes of a row: 8 TMEM columns, 256 B of B.
// E4M3 keeps b3 in the K padding (three E4M3 terms), as for layer 2.
// ---------------------------------------------------------------------------
constexpr uint64_t kDescK = 256 >> 4;   // B descriptor start-address step per K step (256 B)

template <int H, int P, int K1, int SL>
struct Engine {
  static constexpr bool BF16 = P == kBF16, F8 = P == kE4M3;
  static constexpr int KS = F8 ? 32 : 16;                    // K elements per MMA
  static constexpr int EB = F8 ? 1 : 2;                      // bytes per element
  static constexpr int K2 = H + KS;                          // layer 2: hidden + the bias K step
  static constexpr int K3 = F8 ? K2 : H;                     // layer 3 (FP16/BF16: b3 added on read)
  static constexpr uint32_t kACol = H;                       // hidden A region starts after D
  static constexpr int kA1Words = K1 * EB / 4;               // 32-bit words of a layer-1 row
  static constexpr uint32_t kA2End = kACol + K2 * EB / 4;   // end of the hidden A region
  // Merged layout: D3 after the layer-3 A columns, the layer-1 rows after D3.
  static constexpr uint32_t kD3Merged = (kACol + K3 * EB / 4 + 15) / 16 * 16;
  static constexpr uint32_t kA1Merged = kD3Merged + 16 > kA2End ? kD3Merged + 16 : kA2End;
  // Layer 3 is merged with the next tile's layer 1 only when that layout
  // fits a quarter of the SM's tensor memory (the kernels run four slots per
  // CTA); otherwise D3 goes to D's columns and the layer-1 rows follow the
  // hidden A region.  Not merged: 32 inputs at H = 64.
  static constexpr bool kMerge = kA1Merged + kA1Words <= 128;
  static constexpr uint32_t kD3Col = kMerge ? kD3Merged : 0u;
  static constexpr uint32_t kA1Col = kMerge ? kA1Merged : kA2End;
  static constexpr uint32_t kSlotCols = tmem_alloc_cols(kA1Col + kA1Words);
  static_assert(!F8 || H % 32 == 0, "FP8 epilogue works on 32-column chunks");
  int wg, t, it;         // lane, thread in lane, the lane's issuing thread
  bool late;             // a wait of this thread timed out
  uint32_t tmem[SL];     // slot base, lane 0
  uint32_t lane_off;     // this warp's lane quadrant, in the TMEM address
  uint64_t* bar[SL];
  uint32_t phase[SL];
  uint64_t db1, db2, db3;
  const float* b3;       // shared: stored b3 (FP16/BF16)

  template <int KSTEPS, int N>
  __device__ __forceinline__ void mma(int s, uint32_t d_col, uint32_t a_col, uint64_t b_desc) {
#pragma unroll
    for (int ks = 0; ks < KSTEPS; ++ks) {
      if constexpr (F8)
        umma_f8_ts(tmem[s] + d_col, tmem[s] + a_col + 8u * ks, b_desc + kDescK * ks, idesc_f16(128, N, false),
                   ks > 0 ? 1u : 0u);
      else
        umma_f16_ts(tmem[s] + d_col, tmem[s] + a_col + 8u * ks, b_desc + kDescK * ks, idesc_f16(128, N, BF16),
                    ks > 0 ? 1u : 0u);
    }
  }
  // Make this lane's tcgen05.st writes visible and meet at the lane barrier;
  // false (uniform over the lane) if any of its threads saw a wait time out.
  __device__ __forceinline__ bool publish() {
    tmem_st_wait();
    tc_fence_before();
    return !lane_any(wg, late);
  }
  __device__ __forceinline__ bool layer1(int s) {
    if (!publish()) return false;
    if (t == it) {
      tc_fence_after();
      mma<K1 / KS, H>(s, 0u, kA1Col, db1);
      umma_commit(bar[s]);
    }
    return true;
  }
  __device__ __forceinline__ bool layer2(int s) {
    if (!publish()) return false;
    if (t == it) {
      tc_fence_after();
      mma<K2 / KS, H>(s, 0u, kACol, db2);
      umma_commit(bar[s]);
    }
    return true;
  }
  // Layer 3 of the slot's tile and, if `next` (lane-uniform; only with
  // kMerge), layer 1 of the slot's next tile, whose rows are already in the
  // layer-1 columns.
  __device__ __forceinline__ bool layer3(int s, bool next) {
    if (!publish()) return false;
    if (t == it) {
      tc_fence_after();
      mma<K3 / KS, 16>(s, kD3Col, kACol, db3);
      if (kMerge && next) mma<K1 / KS, H>(s, 0u, kA1Col, db1);
      umma_commit(bar[s]);
    }
    return true;
  }
  // Waits (bounded) for slot s's MMAs; returns this thread's own result,
  // which callers use for bookkeeping only (never to branch the lane).
  __device__ __forceinline__ bool wait(int s) {
    const bool ok = mbar_wait(bar[s], phase[s]);
    if (ok) phase[s] ^= 1u;
    late = late || !ok;
    tc_fence_after();
    return ok;
  }
  // Layer-1 row of this thread: kA1Words packed words (once the slot's
  // previous layer-1 MMA has completed).
  __device__ __forceinline__ void write_a1(int s, const uint32_t* w) {
    const uint32_t a = tmem[s] + lane_off + kA1Col;
#pragma unroll
    for (int c = 0; c < kA1Words; c += 8) {
      if (c + 16 <= kA1Words && (c % 16) == 0) {
        uint32_t r[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) r[j] = w[c + j];
        tmem_st16(a + c, r);
        c += 8;
      } else {
        uint32_t r[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) r[j] = w[c + j];
        tmem_st8(a + c, r);
      }
    }
  }
  // Slot s: this thread's row of D -> ReLU -> FP16/BF16/E4M3 -> the hidden A
  // tile; with ONES also the bias ones columns (for FP8 `ones` holds the
  // three codes of the next layer's ones value; FP16/BF16 use 1.0).
  template <bool ONES>
  __device__ __forceinline__ void epilogue(int s, uint32_t ones = 0u) {
    const uint32_t d = tmem[s] + lane_off, a = d + kACol;
    if constexpr (F8) {
#pragma unroll
      for (int c = 0; c < H; c += 32) {
        uint32_t r[32], w[8];
        tmem_ld32(d + c, r);
        tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 8; ++j)
          w[j] = e4m3x2_relu(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1])) |
                 (e4m3x2_relu(__uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3])) << 16);
        tmem_st8(a + c / 4, w);
      }
      if constexpr (ONES) {
        const uint32_t ow[8] = {ones, 0, 0, 0, 0, 0, 0, 0};
        tmem_st8(a + H / 4, ow);
      }
    } else {
#pragma unroll
      for (int c = 0; c < H; c += 32) {
        if (H - c >= 32) {
          uint32_t r[32], w[16];
          tmem_ld32(d + c, r);
          tmem_ld_wait();
#pragma unroll
          for (int j = 0; j < 16; ++j)
            w[j] = pack2_relu<BF16>(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1]));
          tmem_st16(a + c / 2, w);
        } else {
          uint32_t r[16], w[8];
          tmem_ld16(d + c, r);
          tmem_ld_wait();
#pragma unroll
          for (int j = 0; j < 8; ++j)
            w[j] = pack2_relu<BF16>(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1]));
          tmem_st8(a + c / 2, w);
        }
      }
      if constexpr (ONES) {
        const uint32_t one = BF16 ? 0x3F80u : 0x3C00u;
        const uint32_t ow[8] = {one, 0, 0, 0, 0, 0, 0, 0};
        tmem_st8(a + H / 2, ow);
      }
    }
  }
  // The same in 16-column chunks (fewer live registers; FP16/BF16 only).
  template <bool ONES>
  __device__ __forceinline__ void epilogue16(int s) {
    static_assert(!F8 && H % 16 == 0, "16-column FP16/BF16 epilogue");
    const uint32_t d = tmem[s] + lane_off, a = d + kACol;
#pragma unroll
    for (int c = 0; c < H; c += 16) {
      uint32_t r[16], w[8];
      tmem_ld16(d + c, r);
      tmem_ld_wait();
#pragma unroll
      for (int j = 0; j < 8; ++j) w[j] = pack2_relu<BF16>(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1]));
      tmem_st8(a + c / 2, w);
    }
    if constexpr (ONES) {
      const uint32_t one = BF16 ? 0x3F80u : 0x3C00u;
      const uint32_t ow[8] = {one, 0, 0, 0, 0, 0, 0, 0};
      tmem_st8(a + H / 2, ow);
    }
  }
  // Slot s after layer 3: this thread's RGB (FP16/BF16: + stored b3; E4M3:
  // still in the output unit, the caller scales it).
  __device__ __forceinline__ void output(int s, float& y0, float& y1, float& y2) {
    uint32_t r[4];
    tmem_ld4(tmem[s] + lane_off + kD3Col, r);
    tmem_ld_wait();
    y0 = __uint_as_float(r[0]);
    y1 = __uint_as_float(r[1]);
    y2 = __uint_as_float(r[2]);
    if constexpr (!F8) {
      y0 += b3[0];
      y1 += b3[1];
      y2 += b3[2];
    }
  }
};

// CTA set-up: TMEM for all slots, one mbarrier per slot.
template <int NSLOTS, int COLS>
__device__ __forceinline__ uint32_t cta_setup(uint64_t* bars, uint32_t* slot, int tid) {
  if ((tid >> 5) == 0) {
    tmem_alloc(slot, tmem_alloc_cols(NSLOTS * COLS));
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int i = 0; i < NSLOTS; ++i) mbar_init(&bars[i], 1);
    mbar_fence_init();
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  return *slot;
}

// CTA end.  A thread whose wait timed out latches the error word; the issuer
// of each lane first waits (bounded) for the MMAs it has not seen complete,
// so the tensor memory is freed with nothing in flight.
template <int NSLOTS, int COLS, typename E, int SL>
__device__ __forceinline__ void cta_teardown(uint32_t tbase, E& e, const bool (&inflight)[SL], bool timed_out,
                                             int tid) {
  if (timed_out || e.late) atomicOr(&g_tc_error, 1);
  if (e.t == e.it) {
    for (int s = 0; s < SL; ++s)
      if (inflight[s] && !mbar_wait(e.bar[s], e.phase[s])) atomicOr(&g_tc_error, 1);
  }
  tc_fence_before();
  __syncthreads();
  if ((tid >> 5) == 0) {
    tc_fence_after();
    tmem_dealloc(tbase, tmem_alloc_cols(NSLOTS * COLS));
  }
}

__device__ __forceinline__ void copy16(unsigned char* dst, const unsigned char* src, uint32_t bytes, int tid,
                                       int nthreads) {
  for (uint32_t i = tid * 16; i < bytes; i += nthreads * 16)
    *reinterpret_cast<uint4*>(dst + i) = *reinterpret_cast<const uint4*>(src + i);
}

template <int H, int P, int K1, int SL>
__device__ __forceinline__ void engine_init(Engine<H, P, K1, SL>& e, uint32_t tbase, uint64_t* bars, int tid,
                                            uint32_t b1_smem, uint32_t b2_smem, uint32_t b3_smem) {
  using E = Engine<H, P, K1, SL>;
  e.wg = tid >> 7;
  e.t = tid & (kLaneThreads - 1);
  e.it = 32 * (e.wg & 3);
  e.late = false;
  e.b3 = nullptr;
  e.lane_off = (uint32_t)(((e.t >> 5) * 32) << 16);
#pragma unroll
  for (int s = 0; s < SL; ++s) {
    e.tmem[s] = tbase + (uint32_t)((SL * e.wg + s) * E::kSlotCols);
    e.bar[s] = &bars[SL * e.wg + s];
    e.phase[s] = 0;
  }
  e.db1 = sdesc(b1_smem, 128u, K1 * E::EB * 8u);       // 8-row group stride: (row bytes / 16) x 128 B
  e.db2 = sdesc(b2_smem, 128u, E::K2 * E::EB * 8u);
  e.db3 = sdesc(b3_smem, 128u, E::K2 * E::EB * 8u);
}

// ---------------------------------------------------------------------------
// Random-access points
// ---------------------------------------------------------------------------
template <int CS, int CT, int H>
struct PointsSmem {
  using L = TcLayout<CS, CT, H>;
  static constexpr uint32_t kW = 0;                                  // shared part of the image
  static constexpr uint32_t kB1 = kW + L::kShared;                   // points B1
  static constexpr uint32_t kLut = kB1 + H * L::K1P * 2;             // 16 x uint2 palette table
  static constexpr uint32_t kBytes = kLut + 128;
};

// Layer-1 words of one query: features, the ones column for b1, zeros.
template <int CIN, int K1, bool BF16>
__device__ __forceinline__ void pack_a1(const float (&x)[CIN], uint32_t (&w)[K1 / 2]) {
#pragma unroll
  for (int j = 0; j < K1 / 2; ++j) {
    float v[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int k = 2 * j + e;
      v[e] = k < CIN ? x[k < CIN ? k : 0] : (k == CIN ? 1.0f : 0.0f);
    }
    w[j] = pack2<BF16>(v[0], v[1]);
  }
}

template <int CS, int CT, int H, bool BF16, int NWG, int SL>
__global__ void __launch_bounds__(kLaneThreads* NWG, 1) k_points_tc(DevModel m, const unsigned char* __restrict__ ws,
                                                                    const float* __restrict__ uvt, int64_t n,
                                                                    float* __restrict__ rgb) {
  using L = TcLayout<CS, CT, H>;
  using S = PointsSmem<CS, CT, H>;
  constexpr int P = BF16 ? kBF16 : kF16;
  using E = Engine<H, P, L::K1P, SL>;
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ uint64_t bars[SL * NWG];
  __shared__ uint32_t slot;
  const int tid = threadIdx.x;
  copy16(sm + S::kW, ws, L::kShared, tid, kLaneThreads * NWG);
  copy16(sm + S::kB1, ws + L::kB1P, H * L::K1P * 2, tid, kLaneThreads * NWG);
  const uint2* lut = reinterpret_cast<const uint2*>(sm + S::kLut);
  init_p35_lut_sliced(reinterpret_cast<uint2*>(sm + S::kLut), tid);
  const uint8_t* sliced = ws + L::kSliceOff;
  __shared__ float s_b3[3];
  if (tid < 3) s_b3[tid] = stored_b3<BF16>(ws + L::kB3, tid, H, L::K2);
  const uint32_t tbase = cta_setup<SL * NWG, E::kSlotCols>(bars, &slot, tid);
  const uint32_t base = smem_addr(sm);
  E e;
  engine_init<H, P, L::K1P, SL>(e, tbase, bars, tid, base + S::kB1, base + S::kW + L::kB2, base + S::kW + L::kB3);
  const int t = e.t;
  // inflight[s]: slot s has MMAs issued and not yet waited for.
  bool inflight[SL], timed_out = false;
#pragma unroll
  for (int s = 0; s < SL; ++s) inflight[s] = false;
  const int64_t tiles = (n + 127) / 128;
  const int64_t lanes = (int64_t)gridDim.x * NWG, lane_id = (int64_t)blockIdx.x * NWG + e.wg;
  const int64_t qstep = (int64_t)SL * lanes * 128;   // from a slot's tile to its next tile, per query
  // Each slot's next query coordinates are loaded one tile ahead, so their
  // DRAM latency overlaps the current tile.  (Prefetching the next tile's
  // block lines into L1 as well measured 6% slower.)
  float nu[SL], nv[SL], nt[SL];
#pragma unroll
  for (int s = 0; s < SL; ++s) {
    const int64_t q0 = (lane_id + (int64_t)s * lanes) * 128 + t;
    nu[s] = nv[s] = nt[s] = 0.0f;
    if (q0 < n) {
      nu[s] = __ldcs(uvt + 3 * q0);
      nv[s] = __ldcs(uvt + 3 * q0 + 1);
      nt[s] = __ldcs(uvt + 3 * q0 + 2);
    }
  }
  // One tile in flight per lane, software-pipelined: the next tile's gather
  // runs while this tile's layer 2 is on the tensor core, and its layer 1 is
  // issued with this tile's layer 3 (two MMA round trips per tile):
  //   [wait: layer 1 (+ previous layer 3)] [previous RGB out] [ReLU -> layer 2]
  //   [gather the next tile] [wait: layer 2] [ReLU -> layer 3 + next layer 1]
  static_assert(SL == 1, "the point decode pipelines one tile per lane");
  static_assert(SL * NWG * E::kSlotCols <= 512, "slots exceed the SM's tensor memory");
  e.b3 = s_b3;
  // Gathers tile `tl` into the slot's layer-1 columns (their previous MMA has completed).
  auto produce = [&](int64_t tl) {
    const int64_t q = tl * 128 + t, qn = q + qstep;
    const float qu = nu[0], qv = nv[0], qt = nt[0];
    if (qn < n) {
      nu[0] = __ldcs(uvt + 3 * qn);
      nv[0] = __ldcs(uvt + 3 * qn + 1);
      nt[0] = __ldcs(uvt + 3 * qn + 2);
    }
    float x[L::CIN];
    if (q < n) {
      gather_sliced<CS, CT>(m, sliced, qu, qv, qt, x, lut);
    } else {
#pragma unroll
      for (int k = 0; k < L::CIN; ++k) x[k] = 0.0f;
    }
    uint32_t w[L::K1P / 2];
    pack_a1<L::CIN, L::K1P, BF16>(x, w);
    e.write_a1(0, w);
  };
  int64_t tile = lane_id;
  if (tile < tiles) {
    produce(tile);
    e.layer1(0);   // no wait has run yet: cannot report a timeout
    inflight[0] = true;
    int64_t q_cur = tile * 128 + t, q_prev = -1;
    tile += lanes;
    for (;;) {
      inflight[0] = !e.wait(0);   // layer 1 of q_cur (and layer 3 of q_prev)
      if (q_prev >= 0) {   // false only on the first tile, for every thread (tcgen05.ld is warp-wide)
        float y0, y1, y2;
        e.output(0, y0, y1, y2);
        if (q_prev < n) {
          rgb[3 * q_prev] = y0;
          rgb[3 * q_prev + 1] = y1;
          rgb[3 * q_prev + 2] = y2;
        }
      }
      e.template epilogue<true>(0);
      if (!e.layer2(0)) {
        timed_out = true;
        break;
      }
      inflight[0] = true;
      const bool more = tile < tiles;
      if (more) produce(tile);
      inflight[0] = !e.wait(0);   // layer 2
      e.template epilogue<false>(0);
      if (!e.layer3(0, more)) {
        timed_out = true;
        break;
      }
      inflight[0] = true;
      if constexpr (!E::kMerge) {   // layer 3 alone, then the next tile's layer 1
        inflight[0] = !e.wait(0);
        float y0, y1, y2;
        e.output(0, y0, y1, y2);
        if (q_cur < n) {
          rgb[3 * q_cur] = y0;
          rgb[3 * q_cur + 1] = y1;
          rgb[3 * q_cur + 2] = y2;
        }
        if (!more) break;
        if (!e.layer1(0)) {
          timed_out = true;
          break;
        }
        inflight[0] = true;
      } else {
        q_prev = q_cur;
        if (!more) break;
      }
      q_cur = tile * 128 + t;
      tile += lanes;
    }
    if (E::kMerge && !timed_out) {   // the last tile's layer 3
      inflight[0] = !e.wait(0);
      float y0, y1, y2;
      e.output(0, y0, y1, y2);
      if (q_prev < n) {
        rgb[3 * q_prev] = y0;
        rgb[3 * q_prev + 1] = y1;
        rgb[3 * q_prev + 2] = y2;
      }
    }
  }
  cta_teardown<SL * NWG, E::kSlotCols>(tbase, e, inflight, timed_out, tid);
}

// ---------------------------------------------------------------------------
// Batched pages
// ---------------------------------------------------------------------------
constexpr int kRingRows = 16;     // decoded feature rows kept per lane
constexpr int kRingCols = 40;     // feature columns per ring row (>= 64 * 1/2 + 2)
constexpr int kQuad = 64;         // page quadrant side (texels)
constexpr int kDecodeAhead = 4;   // extra feature rows decoded per batch
constexpr uint32_t kRingPlane = kRingRows * kRingCols * 16;   // one 8-channel plane

template <int CS, int CT, int H, int P>
using PagesLayout = std::conditional_t<P == kE4M3, TcLayout8<CS, CT, H>, TcLayout<CS, CT, H>>;

template <int CS, int CT, int H, int NWG, int P>
struct PagesSmem {
  using L = PagesLayout<CS, CT, H, P>;
  static constexpr uint32_t kW = 0;
  static constexpr uint32_t kB1 = kW + L::kShared;                      // pages B1 [H][K1G]
  static constexpr uint32_t kTail = L::kWsBytes - L::kB1G;              // B1, W1T, b1 (and FP8 scales) of the image
  static constexpr uint32_t kW1T = kB1 + (L::kW1T - L::kB1G);           // [CT][H] f32
  static constexpr uint32_t kBias1 = kB1 + (L::kB1 - L::kB1G);          // [H] f32 stored b1
  static constexpr uint32_t kLut = (kB1 + kTail + 127) / 128 * 128;
  static constexpr uint32_t kLutS = kLut + 128;                         // palette table of the sliced decode
  static constexpr uint32_t kLanes = kLutS + 128;
  // per lane: the feature ring and the row table
  static constexpr uint32_t kRing = 0;
  static constexpr uint32_t kRowTab = kRing + (CS / 8) * kRingPlane;   // [64] int4
  static constexpr uint32_t kLaneBytes = (kRowTab + kQuad * 16 + 127) / 128 * 128;
  static constexpr uint32_t kBytes = kLanes + NWG * kLaneBytes;
};

// Per-CTA state shared by the lanes for the current request.
struct PageItem {
  ndgi_page_req r;
  int valid;          // 1 decode, 0 skip
};

// Decodes feature rows r_from..r_to, columns fc0..fc0+ncols-1, into the ring:
// one work unit = (row, column, 8-plane group), read as four 16-byte block
// loads, written as one 16-byte ring entry of 8 FP16 values.
template <int CS>
__device__ __forceinline__ void decode_rows(const DevModel& m, unsigned char* ring, int r_from, int r_to, int fc0,
                                            int ncols, int t, const uint2* lut) {
  constexpr int G = CS / 8;
  const int per_row = ncols * G;
  const int total = (r_to - r_from + 1) * per_row;
  for (int u = t; u < total; u += kLaneThreads) {
    const int rr = u / per_row, rem = u - rr * per_row;
    const int col = rem / G, g = rem - col * G;
    const int fr = r_from + rr, fc = fc0 + col;
    const uint32_t shift = 16u + 3u * (uint32_t)(((fr & 3) << 2) | (fc & 3));
    const uint4* line =
        reinterpret_cast<const uint4*>(m.bc4 + (((size_t)(fr >> 2) * m.bw + (fc >> 2)) * CS + 8 * g) * 8);
    uint4 b[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) b[q] = __ldg(line + q);
    uint32_t h[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float f0 = p35_value(bc4_p35_lut(b[q].x, b[q].y, shift, lut));
      const float f1 = p35_value(bc4_p35_lut(b[q].z, b[q].w, shift, lut));
      h[q] = pack2<false>(f0, f1);
    }
    *reinterpret_cast<uint4*>(ring + g * kRingPlane + ((fr & (kRingRows - 1)) * kRingCols + col) * 16) =
        make_uint4(h[0], h[1], h[2], h[3]);
  }
}

// The same from the texel-sliced copy of the planes: one work unit = one
// feature texel of all 16 planes (two 16-byte endpoint loads and one 8-byte
// index word), written as the two 16-byte ring entries.  The values are the
// same FP16 roundings of fl32(P35) * fl32(1/8925).
template <int CS>
__device__ __forceinline__ void decode_rows_sliced(const DevModel& m, const uint8_t* sl, unsigned char* ring,
                                                   int r_from, int r_to, int fc0, int ncols, int t,
                                                   const uint2* luts) {
  static_assert(CS == 16, "two ring planes of 8 channels");
  using SLc = Sliced<CS>;
  const int total = (r_to - r_from + 1) * ncols;
  for (int u = t; u < total; u += kLaneThreads) {
    const int rr = u / ncols, col = u - rr * ncols;
    const int fr = r_from + rr, fc = fc0 + col;
    const uint8_t* base = sl + ((size_t)(fr >> 2) * m.bw + (fc >> 2)) * SLc::BLOCK;
    const int p = ((fr & 3) << 2) | (fc & 3);
    const uint4 e0 = __ldg(reinterpret_cast<const uint4*>(base));
    const uint4 e1 = __ldg(reinterpret_cast<const uint4*>(base) + 1);
    const uint2 ix = __ldg(reinterpret_cast<const uint2*>(base + SLc::EP) + p);
    const uint32_t ew[8] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y, e1.z, e1.w};
    uint32_t h[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint32_t w = ew[j];
      const uint2 el = luts[nibble_at(ix, 2 * j)];
      const uint2 eh = luts[nibble_at(ix, 2 * j + 1)];
      const float f0 = __fmul_rn(__uint_as_float(__dp2a_lo(el.x, w, el.y)) - 8388608.0f, kInv8925);
      const float f1 = __fmul_rn(__uint_as_float(__dp2a_hi(eh.x, w, eh.y)) - 8388608.0f, kInv8925);
      h[j] = pack2<false>(f0, f1);
    }
    unsigned char* dst = ring + ((fr & (kRingRows - 1)) * kRingCols + col) * 16;
    *reinterpret_cast<uint4*>(dst) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(dst + kRingPlane) = make_uint4(h[4], h[5], h[6], h[7]);
  }
}

// Layer-1 words of one page texel from the ring: bilinear blend of the four
// taps in half2 (16 channels).  FP16/BF16: one channel pair per word; E4M3
// (the x weights then carry the 1/a1 scale): four channels per word.
template <int CS, int P, int NW>
__device__ __forceinline__ void ring_texel(uint32_t (&w)[NW], const unsigned char* ring, int4 rt, int c0, int c1,
                                           __half2 wx0, __half2 wx1) {
  constexpr bool BF16 = P == kBF16;
  const float fy = __int_as_float(rt.z);
  const __half2 wy1 = __float2half2_rn(fy), wy0 = __float2half2_rn(1.0f - fy);
  const __half2 w00 = __hmul2(wx0, wy0), w10 = __hmul2(wx1, wy0), w01 = __hmul2(wx0, wy1), w11 = __hmul2(wx1, wy1);
  const unsigned char* r0p = ring + (rt.x & (kRingRows - 1)) * (kRingCols * 16);
  const unsigned char* r1p = ring + (rt.y & (kRingRows - 1)) * (kRingCols * 16);
#pragma unroll
  for (int g = 0; g < CS / 8; ++g) {
    const int po = g * (int)kRingPlane;
    const uint4 a = *reinterpret_cast<const uint4*>(r0p + po + c0);
    const uint4 b = *reinterpret_cast<const uint4*>(r0p + po + c1);
    const uint4 cq = *reinterpret_cast<const uint4*>(r1p + po + c0);
    const uint4 dd = *reinterpret_cast<const uint4*>(r1p + po + c1);
    const uint32_t av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w}, cv[4] = {cq.x, cq.y, cq.z, cq.w},
                   dv[4] = {dd.x, dd.y, dd.z, dd.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      __half2 v = __hmul2(w00, *reinterpret_cast<const __half2*>(&av[k]));
      v = __hfma2(w10, *reinterpret_cast<const __half2*>(&bv[k]), v);
      v = __hfma2(w01, *reinterpret_cast<const __half2*>(&cv[k]), v);
      v = __hfma2(w11, *reinterpret_cast<const __half2*>(&dv[k]), v);
      if constexpr (P == kE4M3) {
        const uint32_t q = e4m3x2_h(*reinterpret_cast<const uint32_t*>(&v));
        if (k & 1) w[2 * g + k / 2] |= q << 16;
        else w[2 * g + k / 2] = q;
      } else if constexpr (BF16) {
        const float2 f = __half22float2(v);
        w[4 * g + k] = pack2<true>(f.x, f.y);
      } else {
        w[4 * g + k] = *reinterpret_cast<const uint32_t*>(&v);
      }
    }
  }
}

// The layer-1 bias columns after the CS feature channels: FP16/BF16 two ones
// (b1' hi, lo); E4M3 the per-request ones word (three codes of v1); zeros.
template <int CS, int P, int NW>
__device__ __forceinline__ void a1_bias_words(uint32_t (&w)[NW], uint32_t ones8) {
  constexpr int first = P == kE4M3 ? CS / 4 : CS / 2;
  if constexpr (P == kE4M3) {
    w[first] = ones8;
  } else {
    const uint32_t one = P == kBF16 ? 0x3F80u : 0x3C00u;
    w[first] = one | (one << 16);
  }
#pragma unroll
  for (int j = first + 1; j < NW; ++j) w[j] = 0u;
}

// Shared-memory state of the request a page-decode CTA is working on.
template <int CT, int H, bool F8>
struct PageReqState {
  int item;
  PageItem req;
  float vt[CT];
  float beta[F8 ? H : 1];
  uint32_t bmax, ones1;   // FP8: max |b1'/a2| of the request, its ones word
  float b3[3];            // FP16/BF16: stored b3 of the loaded model
};

// The CTA takes its next request (all NT threads call this; it holds CTA
// barriers): thread 0 pulls and validates it.  Returns -1 once the frame is
// done, 0 for a rejected request (skip it), 1 to decode it; then the
// request's model is in shared memory (swapped in if it changed) and its
// folded layer-1 bias b1' sits in B1's bias columns.
template <int CS, int CT, int H, int P, int NT, typename S>
__device__ __forceinline__ int page_take_request(const PagesCtx& c, const ndgi_page_req* __restrict__ reqs, int n,
                                                 int tid, unsigned char* sm, PageReqState<CT, H, P == kE4M3>& st,
                                                 int& loaded, const Fp8Scales* sc) {
  using L = PagesLayout<CS, CT, H, P>;
  constexpr bool BF16 = P == kBF16, F8 = P == kE4M3;
  (void)sc;
  // ---- CTA: next request (the barrier keeps thread 0 from overwriting the
  // shared request slot while a skipped request is still being read) ----
  __syncthreads();
  if (tid == 0) {
    const int item = (int)atomicAdd(c.work_counter, 1u);
    st.item = item;
    if (item < n) {
      const ndgi_page_req r = reqs[item];
      st.req.r = r;
      int ok = r.model >= 0 && r.model < c.n_models && r.w >= 1 && r.w <= 128 && r.h >= 1 && r.h <= 128;
      if (!ok) atomicOr(c.error_word, 2);
      if (ok) {
        const DevModel& mm = c.models[r.model];
        ok = r.x0 >= 0 && r.y0 >= 0 && (int64_t)r.x0 + r.w <= mm.lm_w && (int64_t)r.y0 + r.h <= mm.lm_h &&
             r.dst_x >= 0 && r.dst_y >= 0 && (int64_t)r.dst_x + r.w <= c.phys_w &&
             (int64_t)r.dst_y + r.h <= c.phys_h;
        if (!ok) atomicOr(c.error_word, 4);
      }
      st.req.valid = ok;
    }
  }
  __syncthreads();
  if (st.item >= n) return -1;
  if (!st.req.valid) return 0;
  const ndgi_page_req r = st.req.r;
  const DevModel& m = c.models[r.model];
  if (r.model != loaded) {   // swap in this model's weights (no MMA is in flight here)
    const unsigned char* w = static_cast<const unsigned char*>(c.ws[r.model]);
    copy16(sm + S::kW, w, L::kShared, tid, NT);
    copy16(sm + S::kB1, w + L::kB1G, S::kTail, tid, NT);
    if constexpr (!F8) {
      if (tid < 3) st.b3[tid] = stored_b3<BF16>(w + L::kB3, tid, H, L::K2);
    }
    loaded = r.model;
  }
  if constexpr (F8) {
    if (tid == 0) st.bmax = 0u;
    __syncthreads();   // the scales are read below
  }
  // temporal line at this request's t (FP8: quantised like any layer-1 input)
  if (tid < CT) {
    int j0, j1;
    float a;
    temporal_setup(r.t, m.t_count, j0, j1, a);
    float vt = (1.0f - a) * load_temporal(m.temporal, m.temporal_f16, j0 * CT + tid) +
               a * load_temporal(m.temporal, m.temporal_f16, j1 * CT + tid);
    if constexpr (F8) vt = sc->a1 * e4m3_value(e4m3x2(vt * sc->inv_a1, 0.0f) & 0xFFu);
    st.vt[tid] = vt;
  }
  __syncthreads();
  if constexpr (F8) {
    // folded layer-1 bias b1' = b1 + W1_t vq (FP32) in units a2, stored in
    // B1's columns CS..CS+2 as three E4M3 terms against ones value v1 =
    // max(1, p2(max |b1'/a2|)) (one per request)
    if (tid < H) {
      const float* w1t = reinterpret_cast<const float*>(sm + S::kW1T);
      float b = reinterpret_cast<const float*>(sm + S::kBias1)[tid];
#pragma unroll
      for (int cc = 0; cc < CT; ++cc) b = fmaf(w1t[cc * H + tid], st.vt[cc], b);
      const float beta = b * sc->inv_a2;
      st.beta[tid] = beta;
      atomicMax(&st.bmax, __float_as_uint(fabsf(beta)));
    }
    __syncthreads();
    if (tid < H) {
      const float v1 = fmaxf(1.0f, fp8_p2(__uint_as_float(st.bmax)));
      *reinterpret_cast<uint32_t*>(sm + S::kB1 + kmajor_offset8(tid, CS, L::K1G)) = fp8_terms(st.beta[tid], v1);
      if (tid == 0) {
        const uint32_t oc = e4m3_pow2_code(fminf(v1, 256.0f));
        st.ones1 = oc | (oc << 8) | (oc << 16);
        if (v1 > 256.0f) atomicOr(c.error_word, 8);
      }
    }
  } else if (tid < H) {
    // folded layer-1 bias b1' = b1 + W1_t v_t (FP32), stored in B1's columns
    // CS and CS+1 as a hi + lo pair so the MMA adds it at FP32 accuracy
    const float* w1t = reinterpret_cast<const float*>(sm + S::kW1T);
    float b = reinterpret_cast<const float*>(sm + S::kBias1)[tid];
#pragma unroll
    for (int cc = 0; cc < CT; ++cc) b = fmaf(w1t[cc * H + tid], st.vt[cc], b);
    const uint16_t hi = to_bits<BF16>(b);
    const float hif =
        BF16 ? __uint_as_float((uint32_t)hi << 16) : __half2float(*reinterpret_cast<const __half*>(&hi));
    const uint16_t lo = to_bits<BF16>(b - hif);
    *reinterpret_cast<uint32_t*>(sm + S::kB1 + kmajor_offset(tid, CS, L::K1G)) =
        (uint32_t)hi | ((uint32_t)lo << 16);
  }
  fence_async_smem();   // weights and b1' are read by the tensor core
  __syncthreads();
  return 1;
}

// staged (host-side plan flag): features are at most half the lightmap
// resolution in every model of the plan, so each quadrant's feature rows are
// decoded once into the ring; otherwise each texel gathers its taps directly
// with the lighter gather (its register needs shape the whole kernel's
// allocation, and the hot staged loop must not spill).
template <int CS, int CT, int H, int P, int NWG, int SL>
__global__ void __launch_bounds__(kLaneThreads* NWG, 1) k_pages_tc(PagesCtx c, const ndgi_page_req* __restrict__ reqs,
                                                                   const int32_t* __restrict__ n_dev, int plan_staged) {
  using L = PagesLayout<CS, CT, H, P>;
  using S = PagesSmem<CS, CT, H, NWG, P>;
  using E = Engine<H, P, L::K1G, SL>;
  constexpr bool BF16 = P == kBF16, F8 = P == kE4M3;
  constexpr int NW = E::kA1Words;
  static_assert(CS == 16, "the staged page path is built for 16 spatial channels");
  static_assert(SL * NWG * E::kSlotCols <= 512, "slots exceed the SM's tensor memory");
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ uint64_t bars[SL * NWG];
  __shared__ uint32_t slot;
  __shared__ PageReqState<CT, H, F8> st;
  const Fp8Scales* sc = nullptr;
  if constexpr (F8) sc = reinterpret_cast<const Fp8Scales*>(sm + S::kB1 + (L::kScale - L::kB1G));
  constexpr int NT = kLaneThreads * NWG;
  const int tid = threadIdx.x;
  int n = *n_dev;
  if (n > c.max_reqs || n < 0) {   // reject the whole frame: the request buffer may be shorter
    if (blockIdx.x == 0 && tid == 0) atomicOr(c.error_word, 1);
    n = 0;
  }
  const uint2* lut = reinterpret_cast<const uint2*>(sm + S::kLut);
  const uint2* luts = reinterpret_cast<const uint2*>(sm + S::kLutS);
  init_p35_lut(reinterpret_cast<uint2*>(sm + S::kLut), tid);
  if (tid >= 32 && tid < 48) init_p35_lut_sliced(reinterpret_cast<uint2*>(sm + S::kLutS), tid - 32);
  const uint32_t tbase = cta_setup<SL * NWG, E::kSlotCols>(bars, &slot, tid);
  const uint32_t base = smem_addr(sm);
  E e;
  engine_init<H, P, L::K1G, SL>(e, tbase, bars, tid, base + S::kB1, base + S::kW + L::kB2, base + S::kW + L::kB3);
  e.b3 = st.b3;
  const int wg = e.wg, t = e.t;
  unsigned char* lb = sm + S::kLanes + wg * S::kLaneBytes;
  unsigned char* ring = lb + S::kRing;
  int4* rowtab = reinterpret_cast<int4*>(lb + S::kRowTab);
  int loaded = -1;
  bool inflight[SL], need_out[SL], timed_out = false;   // per slot: MMAs not yet waited for / result to read out
#pragma unroll
  for (int s = 0; s < SL; ++s) inflight[s] = need_out[s] = false;
  for (;;) {
    const int take = page_take_request<CS, CT, H, P, NT, S>(c, reqs, n, tid, sm, st, loaded, sc);
    if (take < 0) break;
    if (take == 0) continue;
    const ndgi_page_req r = st.req.r;
    const DevModel& m = c.models[r.model];
    // ---- lane: 64 x 64 quadrants of the request; a tile = 64 columns x 2 rows ----
    for (int quad = wg; quad < 4 && !timed_out; quad += NWG) {
      const int ox = (quad & 1) * kQuad, oy = (quad >> 1) * kQuad;
      const int qw = min(kQuad, r.w - ox), qh = min(kQuad, r.h - oy);
      if (qw <= 0 || qh <= 0) continue;
      const int col = t & (kQuad - 1);
      int cx0, cx1;
      float fx;
      axis_setup(((float)(r.x0 + ox + col) + 0.5f) / (float)m.lm_w, m.feat_w, m.address_mode, cx0, cx1, fx);
      int fa0, fa1, fb0, fb1;
      float fdum;
      axis_setup(((float)(r.x0 + ox) + 0.5f) / (float)m.lm_w, m.feat_w, m.address_mode, fa0, fa1, fdum);
      axis_setup(((float)(r.x0 + ox + qw - 1) + 0.5f) / (float)m.lm_w, m.feat_w, m.address_mode, fb0, fb1, fdum);
      const int fc0 = min(min(fa0, fa1), min(fb0, fb1));
      const int ncols = max(max(fa0, fa1), max(fb0, fb1)) - fc0 + 1;
      if (t < qh) {
        int ry0, ry1;
        float fy;
        axis_setup(((float)(r.y0 + oy + t) + 0.5f) / (float)m.lm_h, m.feat_h, m.address_mode, ry0, ry1, fy);
        rowtab[t] = make_int4(ry0, ry1, __float_as_int(fy), 0);
      }
      lane_sync(wg);
      // at most half resolution: a 64-texel quadrant side spans <= 34 feature
      // columns and two output rows plus the look-ahead fit the 16-row ring
      const bool staged = plan_staged && ncols <= kRingCols;
      const int fr_last = rowtab[qh - 1].y;
      const float xs = F8 ? sc->inv_a1 : 1.0f;   // FP8: the blend lands in units a1
      const __half2 wx1 = __float2half2_rn(fx * xs), wx0 = __float2half2_rn((1.0f - fx) * xs);
      const int c0 = (cx0 - fc0) * 16, c1 = (cx1 - fc0) * 16;
      int decoded_hi = -1000000;
      int prev_row[SL];
#pragma unroll
      for (int s = 0; s < SL; ++s) prev_row[s] = -1;
      const int ntiles = (qh + 1) / 2;
      // Writes tile tl's layer-1 rows (two output rows of 64 texels) into
      // slot s, decoding the feature rows they need into the ring first;
      // returns this thread's output row.
      // Decodes into the ring the feature rows tile tl's output rows need,
      // plus kDecodeAhead (lane-uniform; ends with a lane barrier).
      auto decode_ahead = [&](int tl) {
        const int need_hi = rowtab[min(2 * tl + 1, qh - 1)].y;
        if (need_hi > decoded_hi) {
          const int from = max(decoded_hi + 1, rowtab[2 * tl].x);
          const int to = min(need_hi + kDecodeAhead, fr_last);
          decode_rows_sliced<CS>(m, static_cast<const uint8_t*>(c.ws[r.model]) + L::kSliceOff, ring, from, to, fc0,
                                 ncols, t, luts);
          decoded_hi = to;
          lane_sync(wg);
        }
      };
      auto produce = [&](int s, int tl) -> int {
        const int row_base = 2 * tl;
        if (staged) decode_ahead(tl);   // feature rows needed by output rows row_base, row_base + 1
        const int orow = row_base + (t >> 6);
        uint32_t w[NW];
        if (col < qw && orow < qh) {
          if (staged) {
            ring_texel<CS, P, NW>(w, ring, rowtab[orow], c0, c1, wx0, wx1);
          } else {
            float x[CS + CT];
            gather_f32<CS, CT, false>(m, ((float)(r.x0 + ox + col) + 0.5f) / (float)m.lm_w,
                                      ((float)(r.y0 + oy + orow) + 0.5f) / (float)m.lm_h, r.t, x, nullptr, lut);
            if constexpr (F8) {
#pragma unroll
              for (int j = 0; j < CS / 4; ++j)
                w[j] = e4m3x2(x[4 * j] * xs, x[4 * j + 1] * xs) | (e4m3x2(x[4 * j + 2] * xs, x[4 * j + 3] * xs) << 16);
            } else {
#pragma unroll
              for (int j = 0; j < CS / 2; ++j) w[j] = pack2<BF16>(x[2 * j], x[2 * j + 1]);
            }
          }
        } else {
#pragma unroll
          for (int j = 0; j < CS * E::EB / 4; ++j) w[j] = 0u;
        }
        a1_bias_words<CS, P, NW>(w, F8 ? st.ones1 : 0u);
        e.write_a1(s, w);
        return orow;
      };
      // Reads slot s's RGB (every thread: tcgen05.ld is warp-wide) and stores
      // the texel of output row orow.
      auto store = [&](int s, int orow) {
        float y0, y1, y2;
        e.output(s, y0, y1, y2);
        if constexpr (F8) {
          const float so = sc->out;
          y0 *= so;
          y1 *= so;
          y2 *= so;
        }
        if (col < qw && orow < qh) {
          const int64_t o = (int64_t)(r.dst_y + oy + orow) * c.phys_w + (r.dst_x + ox + col);
          if (c.out_format == NDGI_RGBA32F) {
            reinterpret_cast<float4*>(c.phys)[o] = make_float4(y0, y1, y2, 1.0f);
          } else {
            reinterpret_cast<uint2*>(c.phys)[o] = make_uint2(pack2<false>(y0, y1), pack2<false>(y2, 1.0f));
          }
        }
      };
      if constexpr (SL == 1) {
        static_assert(E::kMerge, "16 spatial channels: layer 3 always merges with the next layer 1");
        // One tile in flight per lane, software-pipelined: the next tile's
        // layer-1 rows are written (ring decode and blend) while this tile's
        // layer 2 runs, and its layer 1 is issued with this tile's layer 3.
        int cur_row = produce(0, 0), prev = -1;
        bool pending = false;   // the previous tile's layer 3 was issued with this tile's layer 1
        if (!e.layer1(0)) {
          timed_out = true;
        } else {
          inflight[0] = true;
          for (int tile = 1;; ++tile) {
            inflight[0] = !e.wait(0);   // layer 1 (+ the previous tile's layer 3)
            if (pending) store(0, prev);
            e.template epilogue<true>(0, F8 ? sc->ones2 : 0u);
            if (!e.layer2(0)) {
              timed_out = true;
              break;
            }
            inflight[0] = true;
            const bool more = tile < ntiles;
            const int next_row = more ? produce(0, tile) : -1;
            inflight[0] = !e.wait(0);   // layer 2
            e.template epilogue<F8>(0, F8 ? sc->ones3 : 0u);
            if (!e.layer3(0, more)) {
              timed_out = true;
              break;
            }
            inflight[0] = true;
            prev = cur_row;
            pending = true;
            if (!more) break;
            cur_row = next_row;
          }
          if (!timed_out) {   // the last tile's layer 3
            inflight[0] = !e.wait(0);
            store(0, prev);
          }
        }
      } else {
        // SL slots per lane in rounds: each round starts one tile per slot and
        // runs the slots' layers interleaved.
        for (int round = 0; !timed_out; ++round) {
          bool active[SL], any = false;
#pragma unroll
          for (int s = 0; s < SL; ++s) {
            const int tile = SL * round + s;
            active[s] = tile < ntiles;
            any = any || active[s];
            if (timed_out) continue;
            if (need_out[s]) {   // finish this slot's previous tile
              inflight[s] = !e.wait(s);
              need_out[s] = false;
              store(s, prev_row[s]);
            }
            if (!active[s]) continue;
            prev_row[s] = produce(s, tile);
            if (!e.layer1(s)) {
              timed_out = true;
              continue;
            }
            inflight[s] = true;
          }
          if (timed_out || !any) break;
#pragma unroll
          for (int layer = 2; layer <= 3; ++layer) {
#pragma unroll
            for (int s = 0; s < SL; ++s) {
              if (!active[s] || timed_out) continue;
              inflight[s] = !e.wait(s);
              bool ok;
              if (layer == 2) {
                e.template epilogue<true>(s, F8 ? sc->ones2 : 0u);
                ok = e.layer2(s);
              } else {
                e.template epilogue<F8>(s, F8 ? sc->ones3 : 0u);
                ok = e.layer3(s, false);
              }
              if (!ok) {
                timed_out = true;
                continue;
              }
              inflight[s] = true;
              if (layer == 3) need_out[s] = true;
            }
          }
        }
      }
    }
    // every lane must be done with the weights and b1' before the next request
    if (__syncthreads_or(timed_out || e.late)) break;
  }
  cta_teardown<SL * NWG, E::kSlotCols>(tbase, e, inflight, timed_out, tid);
}

// ---------------------------------------------------------------------------
// Warp-specialised page decode.  Each of the CTA's four lanes (one 64 x 64
// quadrant of the request, one tensor-memory slot) has two warpgroups:
//   consumer  runs the MMA chain and the epilogues: [layer 3 of the previous
//             tile + layer 1] -> RGB out, ReLU -> [layer 2] -> ReLU -> A3;
//   producer  writes the layer-1 rows of the lane's next tile (half2 blend
//             from the ring, tcgen05.st) as soon as the slot's previous layer 1
//             has completed, arrives, and then decodes the ring rows of the
//             tile after it while the consumer runs the MMA chain, so the
//             feature work leaves the consumer's critical path and the SM has
//             eight warps per sub-partition.
// Warp w of either warpgroup reaches the same TMEM lane quarter (w mod 4),
// so both address the slot's rows alike.  The two meet at a named barrier
// per tile (the producer arrives, the consumer waits); the producer learns
// that the layer-1 columns are free from the slot's layer-1 mbarrier.
// Waits are bounded and never leave the loop: a wait that gives up sets a
// CTA abort flag, after which every wait returns at once and no more MMAs
// are issued, so every named barrier still sees all its threads and the CTA
// drains quickly with the error latched.
// ---------------------------------------------------------------------------
constexpr int kWsLanes = 4;
// Look-ahead of the warp-specialised producer's ring decode: batches of up to
// five rows, each decoded while the consumer runs the previous tile's MMA
// chain; a quadrant's first batch holds only the first tile's rows, so the
// first MMA starts early.
constexpr int kWsDecodeAhead = 4;

__device__ __forceinline__ void named_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int nthreads) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
// Bounded wait that gives up at once when the CTA has aborted; false if it
// did not see the phase complete.
__device__ __forceinline__ bool ws_wait(uint64_t* bar, uint32_t& phase, volatile int* abort) {
  for (uint32_t i = 0; i < kSpinLimit; ++i) {
    if (mbar_try_wait(bar, phase)) {
      phase ^= 1u;
      tc_fence_after();
      return true;
    }
    if (*abort) return false;
  }
  *abort = 1;
  return false;
}

template <int CS, int CT, int H, int P>
__global__ void __launch_bounds__(2 * kLaneThreads * kWsLanes, 1)
    k_pages_ws(PagesCtx c, const ndgi_page_req* __restrict__ reqs, const int32_t* __restrict__ n_dev) {
  constexpr int NL = kWsLanes;
  using L = PagesLayout<CS, CT, H, P>;
  using S = PagesSmem<CS, CT, H, NL, P>;
  using E = Engine<H, P, L::K1G, 1>;
  constexpr bool BF16 = P == kBF16, F8 = P == kE4M3;
  constexpr int NW = E::kA1Words;
  constexpr int NT = 2 * kLaneThreads * NL;
  static_assert(CS == 16, "the staged page path is built for 16 spatial channels");
  static_assert(E::kMerge && NL * E::kSlotCols <= 512, "one merged slot per lane");
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ uint64_t bar1[NL], bar2[NL];   // per lane: layer-1 (+ layer-3) and layer-2 completion
  __shared__ uint32_t slot;
  __shared__ int s_abort;
  __shared__ PageReqState<CT, H, F8> st;
  const Fp8Scales* sc = nullptr;
  if constexpr (F8) sc = reinterpret_cast<const Fp8Scales*>(sm + S::kB1 + (L::kScale - L::kB1G));
  const int tid = threadIdx.x, wg = tid >> 7, lane = wg & (NL - 1), t = tid & (kLaneThreads - 1);
  const bool producer = wg >= NL;
  // named barriers: 1 + lane ready (256), 5 + lane consumer (128), 9 + lane producer (128)
  const int bar_ready = 1 + lane, bar_cons = 1 + NL + lane, bar_prod = 1 + 2 * NL + lane;
  int n = *n_dev;
  if (n > c.max_reqs || n < 0) {   // reject the whole frame: the request buffer may be shorter
    if (blockIdx.x == 0 && tid == 0) atomicOr(c.error_word, 1);
    n = 0;
  }
  const uint2* luts = reinterpret_cast<const uint2*>(sm + S::kLutS);
  if (tid < 16) init_p35_lut_sliced(reinterpret_cast<uint2*>(sm + S::kLutS), tid);
  if ((tid >> 5) == 0) {
    tmem_alloc(&slot, tmem_alloc_cols(NL * E::kSlotCols));
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int i = 0; i < NL; ++i) {
      mbar_init(&bar1[i], 1);
      mbar_init(&bar2[i], 1);
    }
    mbar_fence_init();
    s_abort = 0;
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = slot, base = smem_addr(sm);
  volatile int* abort = &s_abort;
  E e;   // this lane's slot, seen from either warpgroup
  e.wg = lane;
  e.t = t;
  e.it = 32 * lane;
  e.late = false;
  e.b3 = st.b3;
  e.lane_off = (uint32_t)(((t >> 5) * 32) << 16);
  e.tmem[0] = tbase + (uint32_t)(lane * E::kSlotCols);
  e.bar[0] = &bar1[lane];
  e.phase[0] = 0;
  e.db1 = sdesc(base + S::kB1, 128u, L::K1G * E::EB * 8u);
  e.db2 = sdesc(base + S::kW + L::kB2, 128u, E::K2 * E::EB * 8u);
  e.db3 = sdesc(base + S::kW + L::kB3, 128u, E::K2 * E::EB * 8u);
  const bool issuer = !producer && t == e.it;
  uint32_t ph1 = 0, ph2 = 0;   // parity of the next bar1 / bar2 phase this thread waits for
  bool out1 = false, out2 = false;   // issuer: a commit whose completion it has not seen
  unsigned char* lb = sm + S::kLanes + lane * S::kLaneBytes;
  unsigned char* ring = lb + S::kRing;
  int4* rowtab = reinterpret_cast<int4*>(lb + S::kRowTab);
  int loaded = -1;
  for (;;) {
    const int take = page_take_request<CS, CT, H, P, NT, S>(c, reqs, n, tid, sm, st, loaded, sc);
    if (take < 0) break;
    if (take == 0) continue;
    const ndgi_page_req r = st.req.r;
    const DevModel& m = c.models[r.model];
    const int ox = (lane & 1) * kQuad, oy = (lane >> 1) * kQuad;
    const int qw = min(kQuad, r.w - ox), qh = min(kQuad, r.h - oy);
    const int col = t & (kQuad - 1);
    if (qw > 0 && qh > 0) {   // uniform over the lane's two warpgroups
      const int ntiles = (qh + 1) / 2;
      if (producer) {
        // ---- producer: the layer-1 rows of every tile of the quadrant ----
        int cx0, cx1;
        float fx;
        axis_setup(((float)(r.x0 + ox + col) + 0.5f) / (float)m.lm_w, m.feat_w, m.address_mode, cx0, cx1, fx);
        int fa0, fa1, fb0, fb1;
        float fdum;
        axis_setup(((float)(r.x0 + ox) + 0.5f) / (float)m.lm_w, m.feat_w, m.address_mode, fa0, fa1, fdum);
        axis_setup(((float)(r.x0 + ox + qw - 1) + 0.5f) / (float)m.lm_w, m.feat_w, m.address_mode, fb0, fb1, fdum);
        const int fc0 = min(min(fa0, fa1), min(fb0, fb1));
        const int ncols = max(max(fa0, fa1), max(fb0, fb1)) - fc0 + 1;
        if (t < qh) {
          int ry0, ry1;
          float fy;
          axis_setup(((float)(r.y0 + oy + t) + 0.5f) / (float)m.lm_h, m.feat_h, m.address_mode, ry0, ry1, fy);
          rowtab[t] = make_int4(ry0, ry1, __float_as_int(fy), 0);
        }
        named_sync(bar_prod, kLaneThreads);
        const int fr_last = rowtab[qh - 1].y;
        const float xs = F8 ? sc->inv_a1 : 1.0f;   // FP8: the blend lands in units a1
        const __half2 wx1 = __float2half2_rn(fx * xs), wx0 = __float2half2_rn((1.0f - fx) * xs);
        const int c0 = (cx0 - fc0) * 16, c1 = (cx1 - fc0) * 16;
        int decoded_hi = -1000000;
        // Decodes into the ring the feature rows that tile tl's output rows
        // need, plus a short look-ahead (lane-uniform; the caller syncs).
        // The rows written never share a ring slot with the rows of the tile
        // before it (a span of at most kWsDecodeAhead + 3 < 16 rows), so one
        // thread may decode while another still blends that tile.
        auto decode_for = [&](int tl) {
          const int need_hi = rowtab[min(2 * tl + 1, qh - 1)].y;
          if (need_hi > decoded_hi) {
            const int from = max(decoded_hi + 1, rowtab[2 * tl].x);
            const int to = min(need_hi + (tl == 0 ? 0 : kWsDecodeAhead), fr_last);
            decode_rows_sliced<CS>(m, static_cast<const uint8_t*>(c.ws[r.model]) + L::kSliceOff, ring, from, to,
                                   fc0, ncols, t, luts);
            decoded_hi = to;
          }
        };
        decode_for(0);
        named_sync(bar_prod, kLaneThreads);
        for (int tile = 0; tile < ntiles; ++tile) {
          // the slot's layer-1 columns are free once the previous tile's layer 1 has completed
          if (tile > 0) ws_wait(&bar1[lane], ph1, abort);
          const int row_base = 2 * tile;
          const int orow = row_base + (t >> 6);
          uint32_t w[NW];
          if (col < qw && orow < qh) {
            ring_texel<CS, P, NW>(w, ring, rowtab[orow], c0, c1, wx0, wx1);
          } else {
#pragma unroll
            for (int j = 0; j < CS * E::EB / 4; ++j) w[j] = 0u;
          }
          a1_bias_words<CS, P, NW>(w, F8 ? st.ones1 : 0u);
          e.write_a1(0, w);
          tmem_st_wait();
          tc_fence_before();
          named_arrive(bar_ready, 2 * kLaneThreads);
          // the next tile's rows are decoded while the consumer runs this tile's MMA chain
          if (tile + 1 < ntiles) {
            decode_for(tile + 1);
            named_sync(bar_prod, kLaneThreads);
          }
        }
        // bar1 completes ntiles + 1 phases per quadrant (the last one carries
        // the last tile's layer 3 alone); the producer waited ntiles - 1 of
        // them, and the consumer has seen the other two complete before the
        // CTA barrier that ends the request, so the parity skips both.
      } else {
        // ---- consumer: the MMA chain and the epilogues ----
        auto put = [&](int orow, float y0, float y1, float y2) {
          if constexpr (F8) {
            const float so = sc->out;
            y0 *= so;
            y1 *= so;
            y2 *= so;
          }
          if (col < qw && orow < qh) {
            const int64_t o = (int64_t)(r.dst_y + oy + orow) * c.phys_w + (r.dst_x + ox + col);
            if (c.out_format == NDGI_RGBA32F) {
              reinterpret_cast<float4*>(c.phys)[o] = make_float4(y0, y1, y2, 1.0f);
            } else {
              reinterpret_cast<uint2*>(c.phys)[o] = make_uint2(pack2<false>(y0, y1), pack2<false>(y2, 1.0f));
            }
          }
        };
        int prev_row = 0;
        for (int tile = 0; tile < ntiles; ++tile) {
          // this lane's layer-3 rows (previous tile) and the producer's layer-1 rows are written
          tmem_st_wait();
          tc_fence_before();
          named_sync(bar_ready, 2 * kLaneThreads);
          if (issuer && !*abort) {
            tc_fence_after();
            if (tile > 0) e.template mma<E::K3 / E::KS, 16>(0, E::kD3Col, E::kACol, e.db3);
            e.template mma<L::K1G / E::KS, H>(0, 0u, E::kA1Col, e.db1);
            umma_commit(&bar1[lane]);
            out1 = true;
          }
          if (ws_wait(&bar1[lane], ph1, abort) && issuer) out1 = false;
          if (tile > 0) {   // the previous tile's RGB leaves tensor memory before the layer-2 rows overwrite it
            float y0, y1, y2;
            e.output(0, y0, y1, y2);
            put(prev_row, y0, y1, y2);
          }
          if constexpr (F8) e.template epilogue<true>(0, sc->ones2);
          else e.template epilogue16<true>(0);
          tmem_st_wait();
          tc_fence_before();
          named_sync(bar_cons, kLaneThreads);
          if (issuer && !*abort) {
            tc_fence_after();
            e.template mma<E::K2 / E::KS, H>(0, 0u, E::kACol, e.db2);
            umma_commit(&bar2[lane]);
            out2 = true;
          }
          if (ws_wait(&bar2[lane], ph2, abort) && issuer) out2 = false;
          if constexpr (F8) e.template epilogue<true>(0, sc->ones3);
          else e.template epilogue16<false>(0);
          prev_row = 2 * tile + (t >> 6);
        }
        // the last tile's layer 3 alone
        tmem_st_wait();
        tc_fence_before();
        named_sync(bar_cons, kLaneThreads);
        if (issuer && !*abort) {
          tc_fence_after();
          e.template mma<E::K3 / E::KS, 16>(0, E::kD3Col, E::kACol, e.db3);
          umma_commit(&bar1[lane]);
          out1 = true;
        }
        if (ws_wait(&bar1[lane], ph1, abort) && issuer) out1 = false;
        float y0, y1, y2;
        e.output(0, y0, y1, y2);
        put(prev_row, y0, y1, y2);
      }
    }
    // every lane is done with the weights and b1' before the next request
    __syncthreads();
    if (*abort) break;
  }
  // teardown: an issuer that gave up waiting waits (bounded) for its MMAs
  // before the tensor memory is freed
  if (issuer) {
    if (out1 && !mbar_wait(&bar1[lane], ph1)) atomicOr(&g_tc_error, 1);
    if (out2 && !mbar_wait(&bar2[lane], ph2)) atomicOr(&g_tc_error, 1);
  }
  if (tid == 0 && *abort) atomicOr(&g_tc_error, 1);
  tc_fence_before();
  __syncthreads();
  if ((tid >> 5) == 0) {
    tc_fence_after();
    tmem_dealloc(tbase, tmem_alloc_cols(NL * E::kSlotCols));
  }
}

// The tensor-core point decode's feature gather alone (on the texel-sliced
// copy in a prepared workspace), for validation.
template <int CS, int CT, int H>
__global__ void __launch_bounds__(128) k_debug_features_tc(DevModel m, const unsigned char* __restrict__ ws,
                                                           const float* __restrict__ uvt, int64_t n,
                                                           float* __restrict__ xo) {
  __shared__ uint2 lut[16];
  init_p35_lut_sliced(lut, threadIdx.x);
  __syncthreads();
  const uint8_t* sliced = ws + TcLayout<CS, CT, H>::kSliceOff;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float x[CS + CT];
    gather_sliced<CS, CT>(m, sliced, uvt[3 * i], uvt[3 * i + 1], uvt[3 * i + 2], x, lut);
#pragma unroll
    for (int c = 0; c < CS + CT; ++c) xo[i * (CS + CT) + c] = x[c];
  }
}

// ---------------------------------------------------------------------------
// Dispatch
// ---------------------------------------------------------------------------
#define NDGI_TC_SHAPES(X) \
  X(4, 4, 16)             \
  X(8, 8, 16)             \
  X(8, 8, 32)             \
  X(16, 8, 16)            \
  X(16, 8, 32)            \
  X(16, 8, 64)            \
  X(16, 16, 64)

bool tc_supported(int cs, int ct, int hidden) {
#define X(A, B, C) if (cs == A && ct == B && hidden == C) return true;
  NDGI_TC_SHAPES(X)
#undef X
  return false;
}

bool tc_pages_supported(int cs, int ct, int hidden) { return tc_supported(cs, ct, hidden) && cs == 16; }

size_t tc_workspace_bytes(int cs, int ct, int hidden, int feat_w, int feat_h) {
  const size_t nblocks = (size_t)(feat_w / 4) * (size_t)(feat_h / 4);
#define X(A, B, C) \
  if (cs == A && ct == B && hidden == C) return TcLayout<A, B, C>::kSliceOff + nblocks * Sliced<A>::BLOCK;
  NDGI_TC_SHAPES(X)
#undef X
  return 0;
}

cudaError_t launch_tc_prepare(const DevModel& m, bool bf16, void* ws, cudaStream_t s) {
  const int64_t nblocks = (int64_t)(m.feat_w / 4) * (m.feat_h / 4);
  const int grid = (int)std::min<int64_t>((nblocks + 255) / 256, (int64_t)num_sms() * 8);
#define X(A, B, C)                                                                                       \
  if (m.cs == A && m.ct == B && m.hidden == C) {                                                         \
    if (bf16) k_tc_prepare<A, B, C, true><<<16, 256, 0, s>>>(m, static_cast<unsigned char*>(ws));       \
    else k_tc_prepare<A, B, C, false><<<16, 256, 0, s>>>(m, static_cast<unsigned char*>(ws));           \
    cudaError_t e = cudaGetLastError();                                                                  \
    if (e != cudaSuccess) return e;                                                                      \
    k_slice_features<A><<<grid > 0 ? grid : 1, 256, 0, s>>>(                                             \
        m.bc4, nblocks, static_cast<unsigned char*>(ws) + TcLayout<A, B, C>::kSliceOff);                 \
    return cudaGetLastError();                                                                           \
  }
  NDGI_TC_SHAPES(X)
#undef X
  return cudaErrorInvalidValue;
}

// A tensor-core CTA allocates most of its SM's tensor memory for the whole
// (persistent) kernel, so a second CTA placed on the same SM would block in
// tcgen05.alloc until the first exits.  Asking for more than half of the
// SM's shared memory keeps the placement at one CTA per SM.
constexpr uint32_t kOneCtaPerSmSmem = 116 * 1024;
constexpr uint32_t tc_smem(uint32_t need) { return need > kOneCtaPerSmSmem ? need : kOneCtaPerSmSmem; }

template <typename K>
static cudaError_t set_smem(K kern, uint32_t bytes) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Points: 4 lanes x 1 slot per CTA, one CTA per SM (4 tiles in flight: the
// tensor memory holds 4 slots of 128 columns).
constexpr int kPointsLanes = 4, kPointsSlots = 1;

cudaError_t launch_tc_points(const DevModel& m, bool bf16, const void* ws, const float* uvt, int64_t n, float* rgb,
                             cudaStream_t s) {
  const int64_t tiles = (n + 127) / 128;
  const int64_t need = (tiles + kPointsLanes * kPointsSlots - 1) / (kPointsLanes * kPointsSlots);
  const int64_t cap = num_sms();
  const int grid = (int)(need < cap ? need : cap);
#define X(A, B, C)                                                                                              \
  if (m.cs == A && m.ct == B && m.hidden == C) {                                                                \
    using S = PointsSmem<A, B, C>;                                                                              \
    auto kern = bf16 ? k_points_tc<A, B, C, true, kPointsLanes, kPointsSlots>                                   \
                     : k_points_tc<A, B, C, false, kPointsLanes, kPointsSlots>;                                 \
    const uint32_t smem = tc_smem(S::kBytes);                                                                   \
    cudaError_t e = set_smem(kern, smem);                                                                       \
    if (e != cudaSuccess) return e;                                                                             \
    kern<<<grid, kLaneThreads * kPointsLanes, smem, s>>>(m, static_cast<const unsigned char*>(ws), uvt, n, rgb); \
    return cudaGetLastError();                                                                                  \
  }
  NDGI_TC_SHAPES(X)
#undef X
  return cudaErrorInvalidValue;
}

template <int CS, int CT, int H, int P, int NW, int SL>
static cudaError_t launch_pages_kind(const PagesCtx& c, bool staged, const ndgi_page_req* reqs, const int32_t* n_dev,
                                     cudaStream_t s, int grid) {
  using S = PagesSmem<CS, CT, H, NW, P>;
  auto kern = k_pages_tc<CS, CT, H, P, NW, SL>;
  cudaError_t e = set_smem(kern, tc_smem(S::kBytes));
  if (e != cudaSuccess) return e;
  kern<<<grid, kLaneThreads * NW, tc_smem(S::kBytes), s>>>(c, reqs, n_dev, staged ? 1 : 0);
  return cudaGetLastError();
}

template <int CS, int CT, int H, int NW, int SL>
static cudaError_t launch_pages_shape(const PagesCtx& c, int prec, bool staged, const ndgi_page_req* reqs,
                                      const int32_t* n_dev, cudaStream_t s, int grid) {
  if (prec == kF16) return launch_pages_kind<CS, CT, H, kF16, NW, SL>(c, staged, reqs, n_dev, s, grid);
  if (prec == kBF16) return launch_pages_kind<CS, CT, H, kBF16, NW, SL>(c, staged, reqs, n_dev, s, grid);
  if constexpr (H % 32 == 0) {
    if (prec == kE4M3) return launch_pages_kind<CS, CT, H, kE4M3, NW, SL>(c, staged, reqs, n_dev, s, grid);
  }
  return cudaErrorInvalidValue;
}

template <int CS, int CT, int H, int P>
static cudaError_t launch_pages_ws_kind(const PagesCtx& c, const ndgi_page_req* reqs,
                                        const int32_t* n_dev, cudaStream_t s, int grid) {
  using S = PagesSmem<CS, CT, H, kWsLanes, P>;
  auto kern = k_pages_ws<CS, CT, H, P>;
  cudaError_t e = set_smem(kern, tc_smem(S::kBytes));
  if (e != cudaSuccess) return e;
  kern<<<grid, 2 * kLaneThreads * kWsLanes, tc_smem(S::kBytes), s>>>(c, reqs, n_dev);
  return cudaGetLastError();
}

template <int CS, int CT, int H>
static cudaError_t launch_pages_ws(const PagesCtx& c, int prec, const ndgi_page_req* reqs,
                                   const int32_t* n_dev, cudaStream_t s, int grid) {
  if (prec == kF16) return launch_pages_ws_kind<CS, CT, H, kF16>(c, reqs, n_dev, s, grid);
  if (prec == kBF16) return launch_pages_ws_kind<CS, CT, H, kBF16>(c, reqs, n_dev, s, grid);
  if constexpr (H % 32 == 0) {
    if (prec == kE4M3) return launch_pages_ws_kind<CS, CT, H, kE4M3>(c, reqs, n_dev, s, grid);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_tc_pages(const PagesCtx& c, int prec, int cs, int ct, int hidden, const TcPagesShape& shape,
                            bool staged, const ndgi_page_req* reqs, const int32_t* n_dev, cudaStream_t s) {
  const int grid = num_sms() * shape.ctas_per_sm;
  // warp-specialised: 4 lanes, each with a producer; its ring needs features
  // at most half the lightmap resolution (otherwise the 4 x 1 shape runs)
  if (shape.lanes == 2 * kWsLanes && shape.slots == 1 && staged) {
#define X(A, B, C) \
  if (cs == A && ct == B && hidden == C) return launch_pages_ws<A, B, C>(c, prec, reqs, n_dev, s, grid);
    X(16, 8, 16) X(16, 8, 32) X(16, 8, 64) X(16, 16, 64)
#undef X
    return cudaErrorInvalidValue;
  }
  const TcPagesShape sh = shape.lanes == 2 * kWsLanes ? TcPagesShape{shape.ctas_per_sm, 4, 1} : shape;
#define X(A, B, C, NW, SL)                                                                           \
  if (cs == A && ct == B && hidden == C && sh.lanes == NW && sh.slots == SL)                         \
    return launch_pages_shape<A, B, C, NW, SL>(c, prec, staged, reqs, n_dev, s, grid);
  X(16, 8, 16, 4, 1) X(16, 8, 32, 4, 1) X(16, 8, 64, 4, 1) X(16, 16, 64, 4, 1)
  X(16, 8, 16, 2, 2) X(16, 8, 32, 2, 2) X(16, 8, 64, 2, 2) X(16, 16, 64, 2, 2)
#undef X
  return cudaErrorInvalidValue;
}

bool tc_fp8_pages_supported(int cs, int ct, int hidden) { return tc_pages_supported(cs, ct, hidden) && hidden % 32 == 0; }

// Per-shape FP8 helpers (only shapes with cs = 16 and hidden % 32 == 0 have an FP8 image).
template <int CS, int CT, int H>
static size_t fp8_ws_bytes(size_t nblocks) {
  if constexpr (CS == 16 && H % 32 == 0) return TcLayout8<CS, CT, H>::kSliceOff + nblocks * Sliced<CS>::BLOCK;
  else return 0;
}
template <int CS, int CT, int H>
static uint32_t fp8_status_offset() {
  if constexpr (CS == 16 && H % 32 == 0) return TcLayout8<CS, CT, H>::kScale + offsetof(Fp8Scales, status);
  else return 0;
}
template <int CS, int CT, int H>
static cudaError_t fp8_prepare(const DevModel& m, const float act_max[3], void* ws, cudaStream_t s) {
  if constexpr (CS == 16 && H % 32 == 0) {
    k_tc_prepare8<CS, CT, H><<<1, 256, 0, s>>>(m, act_max[0], act_max[1], act_max[2], static_cast<unsigned char*>(ws));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t nblocks = (int64_t)(m.feat_w / 4) * (m.feat_h / 4);
    const int grid = (int)std::min<int64_t>((nblocks + 255) / 256, (int64_t)num_sms() * 8);
    k_slice_features<CS><<<grid > 0 ? grid : 1, 256, 0, s>>>(m.bc4, nblocks,
                                                            static_cast<unsigned char*>(ws) + TcLayout8<CS, CT, H>::kSliceOff);
    return cudaGetLastError();
  } else {
    return cudaErrorInvalidValue;
  }
}

// E4M3 code -> value on the host (the format definition, exact in FP32).
static float e4m3_host(uint32_t c) {
  const uint32_t e = (c >> 3) & 15u, m = c & 7u;
  const float v = e == 0 ? (float)m * 0x1p-9f : ldexpf(1.0f + (float)m * 0.125f, (int)e - 7);
  return (c & 0x80u) ? -v : v;
}

template <int CS, int CT, int H>
static size_t fp8_unpack(const unsigned char* img, float* out, size_t len) {
  if constexpr (CS == 16 && H % 32 == 0) {
    using L = TcLayout8<CS, CT, H>;
    constexpr int CIN = CS + CT;
    const size_t need = 16 + (size_t)CIN * H + (size_t)H * H + H * 3 + H + 3;
    if (!out || len < need) return need;
    Fp8Scales sc;
    memcpy(&sc, img + L::kScale, sizeof sc);
    const float head[16] = {sc.a1, sc.a2, sc.a3, sc.out, sc.s1, sc.s2, sc.s3, sc.v2, sc.v3, (float)sc.status,
                            0, 0, 0, 0, 0, 0};
    size_t o = 0;
    for (int i = 0; i < 16; ++i) out[o++] = head[i];
    for (int k = 0; k < CIN; ++k)
      for (int n = 0; n < H; ++n)
        out[o++] = k < CS ? sc.s1 * e4m3_host(img[L::kB1G + kmajor_offset8(n, k, L::K1G)])
                          : reinterpret_cast<const float*>(img + L::kW1T)[(k - CS) * H + n];
    for (int k = 0; k < H; ++k)
      for (int n = 0; n < H; ++n) out[o++] = sc.s2 * e4m3_host(img[L::kB2 + kmajor_offset8(n, k, L::K2)]);
    for (int k = 0; k < H; ++k)
      for (int n = 0; n < 3; ++n) out[o++] = sc.s3 * e4m3_host(img[L::kB3 + kmajor_offset8(n, k, L::K2)]);
    for (int n = 0; n < H; ++n) {
      float t = 0.0f;
      for (int j = 0; j < 3; ++j) t += e4m3_host(img[L::kB2 + kmajor_offset8(n, H + j, L::K2)]);
      out[o++] = sc.a3 * sc.v2 * t;
    }
    for (int n = 0; n < 3; ++n) {
      float t = 0.0f;
      for (int j = 0; j < 3; ++j) t += e4m3_host(img[L::kB3 + kmajor_offset8(n, H + j, L::K2)]);
      out[o++] = sc.out * sc.v3 * t;
    }
    return o;
  } else {
    return 0;
  }
}

size_t tc_fp8_unpack(int cs, int ct, int hidden, const unsigned char* image, float* out, size_t len) {
#define X(A, B, C) if (cs == A && ct == B && hidden == C) return fp8_unpack<A, B, C>(image, out, len);
  NDGI_TC_SHAPES(X)
#undef X
  return 0;
}

size_t tc_fp8_workspace_bytes(int cs, int ct, int hidden, int feat_w, int feat_h) {
  const size_t nblocks = (size_t)(feat_w / 4) * (size_t)(feat_h / 4);
#define X(A, B, C) if (cs == A && ct == B && hidden == C) return fp8_ws_bytes<A, B, C>(nblocks);
  NDGI_TC_SHAPES(X)
#undef X
  return 0;
}

cudaError_t launch_tc_prepare8(const DevModel& m, const float act_max[3], void* ws, cudaStream_t s) {
#define X(A, B, C) if (m.cs == A && m.ct == B && m.hidden == C) return fp8_prepare<A, B, C>(m, act_max, ws, s);
  NDGI_TC_SHAPES(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t launch_debug_features_tc(const DevModel& m, const void* ws, const float* uvt, int64_t n, float* x,
                                     cudaStream_t s) {
  const int64_t blocks = (n + 127) / 128;
  const int grid = (int)std::min<int64_t>(blocks > 0 ? blocks : 1, (int64_t)num_sms() * 16);
#define X(A, B, C)                                                                                              \
  if (m.cs == A && m.ct == B && m.hidden == C) {                                                                \
    k_debug_features_tc<A, B, C><<<grid, 128, 0, s>>>(m, static_cast<const unsigned char*>(ws), uvt, n, x);     \
    return cudaGetLastError();                                                                                  \
  }
  NDGI_TC_SHAPES(X)
#undef X
  return cudaErrorInvalidValue;
}

uint32_t tc_fp8_status_offset(int cs, int ct, int hidden) {
#define X(A, B, C) if (cs == A && ct == B && hidden == C) return fp8_status_offset<A, B, C>();
  NDGI_TC_SHAPES(X)
#undef X
  return 0;
}

TcPagesShape tc_default_pages_shape() { return TcPagesShape{1, 4, 1}; }

std::vector<TcPagesShape> tc_pages_candidates(int) {
  return {TcPagesShape{1, 4, 1}, TcPagesShape{1, 2, 2}, TcPagesShape{1, 2 * kWsLanes, 1}};
}

int tc_take_error() {
  int h = 0;
  if (cudaMemcpyFromSymbol(&h, g_tc_error, sizeof(int)) != cudaSuccess) return -1;
  if (h) {
    const int z = 0;
    cudaMemcpyToSymbol(g_tc_error, &z, sizeof(int));
  }
  return h;
}

}  // namespace ndgi
