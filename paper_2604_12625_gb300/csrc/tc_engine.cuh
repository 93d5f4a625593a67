// The tensor-core (tcgen05) MLP engine shared by the point decode
// (tc_points.cu) and the page decode (tc_decode.cu): the operand images
// ndgi_prepare writes (FP16/BF16 and E4M3), the conversion helpers, the
// per-lane Engine that runs a tile's three layers from tensor memory, the CTA
// set-up and tear-down of tensor memory and barriers, and the launch-shape
// helpers.  Everything here is a template or inline: both translation units
// include it.
#pragma once

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
  static constexpr uint32_t kErrOff = kWsBytes;            // int: error word of the point decodes using this image
  static constexpr uint32_t kDbgOff = kWsBytes + 4;        // int: debug word (kDbgInjectTimeout)
  static constexpr uint32_t kSliceOff = (kWsBytes + 16 + 255) / 256 * 256;   // then the texel-sliced BC4 copy
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
static __device__ float fp8_p2(float y) {
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
static __device__ uint32_t fp8_terms(float beta, float v) {
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

// CTA end.  A thread whose wait timed out latches kErrTimeout in the caller's
// error word; the issuer of each lane first waits (bounded) for the MMAs it
// has not seen complete, so the tensor memory is freed with nothing in flight.
template <int NSLOTS, int COLS, typename E, int SL>
__device__ __forceinline__ void cta_teardown(uint32_t tbase, E& e, const bool (&inflight)[SL], bool timed_out,
                                             int tid, int* err) {
  if (timed_out || e.late) atomicOr(err, kErrTimeout);
  if (e.t == e.it) {
    for (int s = 0; s < SL; ++s)
      if (inflight[s] && !mbar_wait(e.bar[s], e.phase[s])) atomicOr(err, kErrTimeout);
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

// Debug injection (kDbgInjectTimeout): every thread waits, with a short limit,
// for a phase of its lane's first slot barrier that nothing completes (no MMA
// has been committed yet), so the lane carries a timeout into its first
// barrier and the kernel unwinds along its real timeout path.
// Each poll suspends at most kInjectHintNs, so the injected wait ends within
// about kInjectSpin * kInjectHintNs = 0.25 ms.
constexpr uint32_t kInjectSpin = 256, kInjectHintNs = 1000;
template <typename E>
__device__ __forceinline__ void inject_timeout(E& e) {
  bool done = false;
  for (uint32_t i = 0; i < kInjectSpin && !done; ++i) done = mbar_try_wait_for(e.bar[0], e.phase[0], kInjectHintNs) != 0;
  e.late = e.late || !done;
}

// Warp-specialised kernels (pages and points): kWsLanes MMA lanes per CTA,
// each with a producer warpgroup that writes the layer-1 rows of the lane's
// next tile while the lane's consumer warpgroup runs the MMA chain.  The two
// meet at named barriers; every wait is bounded and gives up at once after a
// CTA abort (a flag in shared memory), so all barriers still complete.
constexpr int kWsLanes = 4;
__device__ __forceinline__ void named_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int nthreads) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
// Bounded wait that gives up at once when the CTA has aborted; false if it
// did not see the phase complete.
static __device__ __noinline__ bool ws_wait_slow(uint64_t* bar, uint32_t phase, volatile int* abort) {
  const uint64_t t0 = global_ns();
  for (uint32_t i = 0; i < kSpinLimit; ++i) {
    if (mbar_try_wait_for(bar, phase, kPollHintNs)) return true;
    if (*abort) return false;
    if (global_ns() - t0 > kWaitLimitNs) break;
  }
  *abort = 1;
  return false;
}
__device__ __forceinline__ bool ws_wait(uint64_t* bar, uint32_t& phase, volatile int* abort) {
  if (*abort) return false;
  if (!mbar_try_wait(bar, phase)) {
    if (*abort || !ws_wait_slow(bar, phase, abort)) return false;
  }
  phase ^= 1u;
  tc_fence_after();
  return true;
}


// ---------------------------------------------------------------------------
// Built shapes (cs, ct, hidden) and launch helpers
// ---------------------------------------------------------------------------
#define NDGI_TC_SHAPES(X) \
  X(4, 4, 16)             \
  X(8, 8, 16)             \
  X(8, 8, 32)             \
  X(16, 8, 16)            \
  X(16, 8, 32)            \
  X(16, 8, 64)            \
  X(16, 16, 64)

// Decoded-texel cache of the point decode (tc_points.cu): FP16
// [feat_h][feat_w][cs] after the texel-sliced planes in an FP16/BF16
// workspace, kept only for maps whose cache fits kPointsCacheMax (so that it
// stays resident in the 129 MB L2 while queries stream through).
constexpr size_t kPointsCacheMax = (size_t)64 << 20;
inline size_t points_cache_bytes(int cs, int feat_w, int feat_h) {
  const size_t b = (size_t)feat_w * (size_t)feat_h * (size_t)cs * 2;
  return b <= kPointsCacheMax ? b : 0;
}
template <int CS, int CT, int H>
inline size_t points_cache_offset(int feat_w, int feat_h) {
  const size_t nblocks = (size_t)(feat_w / 4) * (size_t)(feat_h / 4);
  return (TcLayout<CS, CT, H>::kSliceOff + nblocks * Sliced<CS>::BLOCK + 255) / 256 * 256;
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

}  // namespace ndgi
