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
// the caller owns (the prepared workspace for points, the plan's block for
// pages), and the CTA unwinds and frees its tensor memory.
#include "tc_engine.cuh"

namespace ndgi {
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
  if (tid == 0) {
    *reinterpret_cast<int*>(ws + L::kErrOff) = 0;
    *reinterpret_cast<int*>(ws + L::kDbgOff) = 0;
  }
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
    temporal_setup_k(r.t, m.t_count, m.key_t, j0, j1, a);
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
  if (c.debug_word && (*c.debug_word & kDbgInjectTimeout)) inject_timeout(e);
  e.b3 = st.b3;
  const int wg = e.wg, t = e.t;
  // FP8 operand dump (test hook, off unless the plan's debug word asks for it)
  uint32_t* dump = nullptr;
  int dump_item = -1;
  if constexpr (F8) {
    if (c.debug_word && (c.debug_word[0] & kDbgDumpFp8)) {
      dump_item = c.debug_word[1];
      dump = *reinterpret_cast<uint32_t* const*>(c.debug_word + 2);
    }
  }
  constexpr int kDumpRow = fp8_dump_row_words(H), kDumpQ = (H + 32) / 4;
  // Copies nw words of this thread's tensor-memory row from column col to
  // word off of its dump row (warp-uniform: tcgen05.ld is warp-wide).
  auto dump_tmem = [&](uint32_t col, int nw, int off) {
    tmem_st_wait();
    for (int k = 0; k < nw; k += 4) {
      uint32_t v[4];
      tmem_ld4(e.tmem[0] + e.lane_off + col + (uint32_t)k, v);
      tmem_ld_wait();
#pragma unroll
      for (int j = 0; j < 4; ++j) dump[t * kDumpRow + off + k + j] = v[j];
    }
  };
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
      const bool dumping = F8 && dump != nullptr && st.item == dump_item && quad == 0;   // lane-uniform
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
        if constexpr (F8) {
          if (dumping && tl == 0) {
#pragma unroll
            for (int j = 0; j < NW; ++j) dump[t * kDumpRow + j] = w[j];
            uint32_t* tail = dump + kLaneThreads * kDumpRow;
            if (t < CT) tail[t] = __float_as_uint(st.vt[t]);
            if (t < H) tail[CT + t] = *reinterpret_cast<const uint32_t*>(sm + S::kB1 + kmajor_offset8(t, CS, L::K1G));
          }
        }
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
            if constexpr (F8) {
              if (dumping && tile == 1) dump_tmem(0u, H, 8);                              // D1
              if (dumping && tile == 2) dump_tmem(E::kD3Col, 4, 8 + 2 * H + 2 * kDumpQ);   // D3
            }
            if (pending) store(0, prev);
            e.template epilogue<true>(0, F8 ? sc->ones2 : 0u);
            if constexpr (F8) {
              if (dumping && tile == 1) dump_tmem(E::kACol, kDumpQ, 8 + H);               // A2
            }
            if (!e.layer2(0)) {
              timed_out = true;
              break;
            }
            inflight[0] = true;
            const bool more = tile < ntiles;
            const int next_row = more ? produce(0, tile) : -1;
            inflight[0] = !e.wait(0);   // layer 2
            if constexpr (F8) {
              if (dumping && tile == 1) dump_tmem(0u, H, 8 + H + kDumpQ);                 // D2
            }
            e.template epilogue<F8>(0, F8 ? sc->ones3 : 0u);
            if constexpr (F8) {
              if (dumping && tile == 1) dump_tmem(E::kACol, kDumpQ, 8 + 2 * H + kDumpQ);   // A3
            }
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
  cta_teardown<SL * NWG, E::kSlotCols>(tbase, e, inflight, timed_out, tid, c.error_word);
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
// Look-ahead of the warp-specialised producer's ring decode: batches of up to
// five rows, each decoded while the consumer runs the previous tile's MMA
// chain; a quadrant's first batch holds only the first tile's rows, so the
// first MMA starts early.
constexpr int kWsDecodeAhead = 4;

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
  e.it = 32 * ((lane + 1) & (NL - 1));   // issuers in warps 1, 2, 3, 0 of their lanes: none in the CTA's warp 0
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
  if (tid == 0 && c.debug_word && (*c.debug_word & kDbgInjectTimeout)) {
    // injected timeout: a short wait on a phase nothing completes, then the real abort path
    bool done = false;
    for (uint32_t i = 0; i < kInjectSpin && !done; ++i) done = mbar_try_wait_for(&bar1[0], 0u, kInjectHintNs) != 0;
    if (!done) *abort = 1;
  }
  __syncthreads();
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
          // Normally the producer cannot get ahead (it waited for this slot's previous
          // layer 1), so arriving is enough; once the CTA has aborted its waits return
          // at once, and it must sync instead so that it never arrives twice before
          // the consumer's sync of the same barrier generation.
          if (*abort) named_sync(bar_ready, 2 * kLaneThreads);
          else named_arrive(bar_ready, 2 * kLaneThreads);
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
    if (out1 && !mbar_wait(&bar1[lane], ph1)) atomicOr(c.error_word, kErrTimeout);
    if (out2 && !mbar_wait(&bar2[lane], ph2)) atomicOr(c.error_word, kErrTimeout);
  }
  if (tid == 0 && *abort) atomicOr(c.error_word, kErrTimeout);
  tc_fence_before();
  __syncthreads();
  if ((tid >> 5) == 0) {
    tc_fence_after();
    tmem_dealloc(tbase, tmem_alloc_cols(NL * E::kSlotCols));
  }
}

// ---------------------------------------------------------------------------
// Dispatch
// ---------------------------------------------------------------------------
bool tc_supported(int cs, int ct, int hidden) {
#define X(A, B, C) if (cs == A && ct == B && hidden == C) return true;
  NDGI_TC_SHAPES(X)
#undef X
  return false;
}

bool tc_pages_supported(int cs, int ct, int hidden) { return tc_supported(cs, ct, hidden) && cs == 16; }

size_t tc_workspace_bytes(int cs, int ct, int hidden, int feat_w, int feat_h) {
  const size_t cache = points_cache_bytes(cs, feat_w, feat_h);
#define X(A, B, C)                                                                                          \
  if (cs == A && ct == B && hidden == C) {                                                                  \
    const size_t off = points_cache_offset<A, B, C>(feat_w, feat_h);                                        \
    return cache ? off + cache                                                                              \
                 : TcLayout<A, B, C>::kSliceOff + (size_t)(feat_w / 4) * (size_t)(feat_h / 4) * Sliced<A>::BLOCK; \
  }
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

uint32_t tc_error_offset(int cs, int ct, int hidden) {
#define X(A, B, C) if (cs == A && ct == B && hidden == C) return TcLayout<A, B, C>::kErrOff;
  NDGI_TC_SHAPES(X)
#undef X
  return 0;
}

}  // namespace ndgi

