// Differentiable fit of the decoder (Sec. 3.4 BC simulation, Sec. 4 training).
//
// Forward per sample (a query (u, v, t), as for the point decode): the four
// bilinear taps of the feature map are rebuilt from the block endpoints and
// weights (Eq. 7) with straight-through quantisation, so the features equal
// the packed BC4 decode bit for bit; the temporal feature is the linear
// interpolation (Eq. 2) of the keyframe rows j0, j1 around t; then the MLP.
//
// Backward (recompute, nothing stored between passes): a persistent CTA
// processes tiles of 128 samples.  Per tile each thread runs its sample's
// forward, then the backward of the output and hidden layers; the weight
// gradients of the tile are the contractions H2^T dY, H1^T dZ2 and X^T dZ1
// over the tile's samples, done from shared memory into per-thread register
// accumulators that persist across tiles and are flushed once per CTA.
// Temporal-line gradients (a sample splits its gradient between rows j0 and
// j1 in the ratio (1 - alpha) : alpha) are reduced in shared memory first.  Feature-map gradients go straight to global memory
// with FP32 atomics, after merging the endpoint gradients of taps that fall
// in the same block.
#include <cmath>

#include "ndgi_internal.h"
#include "sampler.cuh"
#include "bc4.cuh"

namespace ndgi {

constexpr int kFitThreads = 128;
constexpr int kFitTile = 128;

struct FitArgs {
  int lm_w, lm_h, feat_w, feat_h, cs, bw, t_count, ct, hidden, address_mode;
  const float* key_t;           // keyframe times [t_count] or null (j / t_count)
  const float *ea, *eb, *w, *temporal, *w1, *b1, *w2, *b2, *w3, *b3;
  float *g_ea, *g_eb, *g_w, *g_temporal, *g_w1, *g_b1, *g_w2, *g_b2, *g_w3, *g_b3;
  int relaxed;
  int vec_red;                  // g_ea, g_eb 16-byte aligned: endpoint gradients use vector reductions
  int vec_ld;                   // ea, eb 16-byte aligned: endpoints are read with vector loads
  int64_t n;
  const float* uvt;             // mode 0: queries [n][3]
  const float* grad_rgb;        // mode 0
  const __half* targets;        // mode 1: keyframe targets [T][lm_h][lm_w][3], interpolated in t
  uint64_t seed;                // mode 1
  const int64_t* step;          // mode 1: device step counter
  double* loss_acc;             // mode 1: sum of squared errors
  int n_models;                 // mode 1: models trained side by side (CTA row blockIdx.y = model)
  int64_t ms[10];               // per-model element count of each tensor (and of its gradient)
  int64_t tgt_stride;           // per-model element count of the targets
};

// Batched fit (mode 1): the ten tensors, their gradients and the targets hold
// n_models models one after another; CTA row m trains model m, drawing its
// samples with seed + m.
__device__ __forceinline__ void fit_select_model(FitArgs& a) {
  const int64_t m = blockIdx.y;
  if (m == 0) return;
  a.ea += m * a.ms[0];
  a.eb += m * a.ms[1];
  a.w += m * a.ms[2];
  a.temporal += m * a.ms[3];
  a.w1 += m * a.ms[4];
  a.b1 += m * a.ms[5];
  a.w2 += m * a.ms[6];
  a.b2 += m * a.ms[7];
  a.w3 += m * a.ms[8];
  a.b3 += m * a.ms[9];
  a.g_ea += m * a.ms[0];
  a.g_eb += m * a.ms[1];
  a.g_w += m * a.ms[2];
  a.g_temporal += m * a.ms[3];
  a.g_w1 += m * a.ms[4];
  a.g_b1 += m * a.ms[5];
  a.g_w2 += m * a.ms[6];
  a.g_b2 += m * a.ms[7];
  a.g_w3 += m * a.ms[8];
  a.g_b3 += m * a.ms[9];
  a.targets += m * a.tgt_stride;
  a.seed += (uint64_t)m;
}


// ---------------------------------------------------------------------------
// BC-simulated feature texel and its straight-through chain-rule factors.
// ---------------------------------------------------------------------------
struct TapInfo {
  int64_t blk;    // (by*bw + bx)*cs  (channel 0)
  int p;          // texel in block
  float wt;       // bilinear weight
};

__device__ __forceinline__ void fit_taps(const FitArgs& a, float u, float v, TapInfo (&t)[4], float& fx, float& fy) {
  int x0, x1, y0, y1;
  axis_setup(u, a.feat_w, a.address_mode, x0, x1, fx);
  axis_setup(v, a.feat_h, a.address_mode, y0, y1, fy);
  const int tx[4] = {x0, x1, x0, x1}, ty[4] = {y0, y0, y1, y1};
  const float wt[4] = {(1.0f - fx) * (1.0f - fy), fx * (1.0f - fy), (1.0f - fx) * fy, fx * fy};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    t[q].blk = ((int64_t)(ty[q] >> 2) * a.bw + (tx[q] >> 2)) * a.cs;
    t[q].p = ((ty[q] & 3) << 2) | (tx[q] & 3);
    t[q].wt = wt[q];
  }
}

// Feature value f and factors df/dea, df/deb, df/dw of (block*cs + c, texel p).
__device__ __forceinline__ float sim_value(const FitArgs& a, int64_t bc, int p, float& dea, float& deb, float& dw) {
  const float ea = a.ea[bc], eb = a.eb[bc], w = a.w[bc * 16 + p];
  if (a.relaxed) {
    dea = 1.0f - w;
    deb = w;
    dw = eb - ea;
    return (1.0f - w) * ea + w * eb;
  }
  const int A = quant(ea, 255.0f), B = quant(eb, 255.0f), k = quant(w, 7.0f);
  const float qw = (float)k * (1.0f / 7.0f);
  dea = 1.0f - qw;
  deb = qw;
  dw = (float)(B - A) * (1.0f / 255.0f);
  return p35_value(5 * ((7 - k) * A + k * B));
}

// The same for N consecutive channels k0 .. k0+N-1 of one tap (N = 1, 2, 4;
// the endpoints of the N channels are read with one vector load each).
template <int N>
__device__ __forceinline__ void sim_values(const FitArgs& a, int64_t blk, int k0, int p, float (&f)[N],
                                           float (&dea)[N], float (&deb)[N], float (&dw)[N]) {
  float ea[N], eb[N];
  if (!a.vec_ld) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      ea[i] = __ldg(a.ea + blk + k0 + i);
      eb[i] = __ldg(a.eb + blk + k0 + i);
    }
  } else if constexpr (N == 4) {
    const float4 x = __ldg(reinterpret_cast<const float4*>(a.ea + blk + k0));
    const float4 y = __ldg(reinterpret_cast<const float4*>(a.eb + blk + k0));
    ea[0] = x.x; ea[1] = x.y; ea[2] = x.z; ea[3] = x.w;
    eb[0] = y.x; eb[1] = y.y; eb[2] = y.z; eb[3] = y.w;
  } else if constexpr (N == 2) {
    const float2 x = __ldg(reinterpret_cast<const float2*>(a.ea + blk + k0));
    const float2 y = __ldg(reinterpret_cast<const float2*>(a.eb + blk + k0));
    ea[0] = x.x; ea[1] = x.y;
    eb[0] = y.x; eb[1] = y.y;
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      ea[i] = __ldg(a.ea + blk + k0 + i);
      eb[i] = __ldg(a.eb + blk + k0 + i);
    }
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const float w = __ldg(a.w + (blk + k0 + i) * 16 + p);
    if (a.relaxed) {
      dea[i] = 1.0f - w;
      deb[i] = w;
      dw[i] = eb[i] - ea[i];
      f[i] = (1.0f - w) * ea[i] + w * eb[i];
    } else {
      const int A = quant(ea[i], 255.0f), B = quant(eb[i], 255.0f), k = quant(w, 7.0f);
      const float qw = (float)k * (1.0f / 7.0f);
      dea[i] = 1.0f - qw;
      deb[i] = qw;
      dw[i] = (float)(B - A) * (1.0f / 255.0f);
      f[i] = p35_value(5 * ((7 - k) * A + k * B));
    }
  }
}

template <int CS, int CT>
__device__ __forceinline__ void fit_gather(const FitArgs& a, float u, float v, float tq, float (&x)[CS + CT]) {
  TapInfo t[4];
  float fx, fy;
  fit_taps(a, u, v, t, fx, fy);
  const float gx = 1.0f - fx, gy = 1.0f - fy;
#pragma unroll
  for (int c = 0; c < CS; ++c) {
    float f[4], d0, d1, d2;
#pragma unroll
    for (int q = 0; q < 4; ++q) f[q] = sim_value(a, t[q].blk + c, t[q].p, d0, d1, d2);
    x[c] = gy * (gx * f[0] + fx * f[1]) + fy * (gx * f[2] + fx * f[3]);   // same blend order as the decode
  }
  int j0, j1;
  float al;
  temporal_setup_k(tq, a.t_count, a.key_t, j0, j1, al);
  const float ga = 1.0f - al;
#pragma unroll
  for (int c = 0; c < CT; ++c) x[CS + c] = ga * a.temporal[j0 * CT + c] + al * a.temporal[j1 * CT + c];
}

// ---------------------------------------------------------------------------
// Forward only (one thread per sample).
// ---------------------------------------------------------------------------
template <int CS, int CT, int H>
__global__ void __launch_bounds__(kFitThreads) k_fit_forward(FitArgs a, float* __restrict__ rgb) {
  constexpr int CIN = CS + CT;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < a.n; s += (int64_t)gridDim.x * blockDim.x) {
    float x[CIN];
    fit_gather<CS, CT>(a, a.uvt[3 * s], a.uvt[3 * s + 1], a.uvt[3 * s + 2], x);
    float h1[H];
#pragma unroll
    for (int o = 0; o < H; ++o) {
      float z = a.b1[o];
#pragma unroll
      for (int i = 0; i < CIN; ++i) z = fmaf(x[i], a.w1[i * H + o], z);
      h1[o] = fmaxf(z, 0.0f);
    }
    float y0 = a.b3[0], y1 = a.b3[1], y2 = a.b3[2];
    for (int o = 0; o < H; ++o) {
      float z = a.b2[o];
#pragma unroll
      for (int i = 0; i < H; ++i) z = fmaf(h1[i], a.w2[i * H + o], z);
      const float h = fmaxf(z, 0.0f);
      y0 = fmaf(h, a.w3[o * 3 + 0], y0);
      y1 = fmaf(h, a.w3[o * 3 + 1], y1);
      y2 = fmaf(h, a.w3[o * 3 + 2], y2);
    }
    rgb[3 * s] = y0;
    rgb[3 * s + 1] = y1;
    rgb[3 * s + 2] = y2;
  }
}

// ---------------------------------------------------------------------------
// Backward (persistent, tiles of kFitTile samples, kFitQ threads per sample).
// MODE 0: samples + dL/drgb given.  MODE 1: samples drawn on device, dL/drgb
// from the MSE against the FP16 targets, FP64 loss accumulated.  MODE 2: MODE 1
// for a batch of stacked models (CTA row blockIdx.y = model; fit_select_model).
//
// Each sample's forward and backward is split over kFitQ = 4 threads (q),
// each computing HQ = H/4 of the hidden units, which gives 16 warps per SM
// (the per-tile buffers the weight-gradient contraction reads, about 1 KB per
// sample, bound the tile).  Shared-memory layouts are chosen so that the four
// threads of a sample never hit the same bank with different addresses:
// weight rows are stored "skewed" (4 padding floats after each quarter's HQ
// columns) so the quarters' float4 reads fall in distinct banks, the backward
// reads transposed skewed copies (W2^T, W1^T) so every thread of a sample
// walks the same row, and activation rows are padded to whole float4s.
// ---------------------------------------------------------------------------
constexpr int kBwdThreads = 512;
constexpr int kFitQ = kBwdThreads / kFitTile;

template <int CS, int CT, int H>
struct FitSmem {
  static constexpr int CIN = CS + CT;
  static constexpr int HQ = H / kFitQ;
  static constexpr int HS = H + 4 * kFitQ;          // skewed row: HQ columns + 4 padding floats per quarter
  static constexpr int LX = CIN + 4, LH = H + 4;    // activation rows (float4-aligned)
  static constexpr int kW1s = 0;                     // [CIN][HS]  W1, skewed columns
  static constexpr int kW2s = kW1s + CIN * HS;       // [H][HS]    W2, skewed columns
  static constexpr int kW2t = kW2s + H * HS;         // [H][HS]    W2^T (row o, skewed columns i)
  static constexpr int kW1t = kW2t + H * HS;         // [H][CIN]   W1^T (row o, columns k)
  static constexpr int kB1 = kW1t + H * CIN, kB2 = kB1 + H;
  static constexpr int kW3 = kB2 + H, kB3 = kW3 + H * 4;
  static constexpr int kX = kB3 + 4, kH1 = kX + kFitTile * LX, kH2 = kH1 + kFitTile * LH;
  static constexpr int kG1 = kH2 + kFitTile * LH, kY = kG1 + kFitTile * LH, kDY = kY + kFitTile * kFitQ * 4;
  static constexpr int kGK = kDY + kFitTile * 4;
  static constexpr int kFloatsNoGK = kGK;
  static_assert(kW2s % 4 == 0 && kW2t % 4 == 0 && kW1t % 4 == 0 && kW3 % 4 == 0 && kX % 4 == 0 && kH1 % 4 == 0 &&
                    kY % 4 == 0 && kDY % 4 == 0 && HS % 4 == 0 && CIN % 4 == 0,
                "float4 rows");
  __host__ __device__ static constexpr int skew(int o) { return o + 4 * (o / HQ); }
};

// N consecutive floats of shared memory (N = 1, 2, 4; 4N-byte aligned).
template <int N>
__device__ __forceinline__ void lds(const float* p, float (&v)[N]) {
  if constexpr (N == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else if constexpr (N == 2) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    v[0] = t.x; v[1] = t.y;
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = p[i];
  }
}

template <int CS, int CT, int H, int MODE>
__global__ void __launch_bounds__(kBwdThreads, 1) k_fit_backward(FitArgs a_in) {
  using L = FitSmem<CS, CT, H>;
  FitArgs a = a_in;
  if constexpr (MODE == 2) fit_select_model(a);
  constexpr int CIN = CS + CT;
  constexpr int LX = L::LX, LH = L::LH, HS = L::HS, HQ = L::HQ;
  constexpr int SC = CS / kFitQ, TC = CT / kFitQ;   // spatial / temporal channels per thread of a sample
  static_assert(CS % kFitQ == 0 && CT % kFitQ == 0 && SC <= 4 && TC <= 4 && (SC & (SC - 1)) == 0 &&
                    (TC & (TC - 1)) == 0 && H % kFitQ == 0 && HQ % 4 == 0 && kBwdThreads % H == 0,
                "shape");
  constexpr bool kBlocked = H == 64;                 // dW2 as 2 x 4 register blocks per thread
  constexpr int K2 = (H * H + kBwdThreads - 1) / kBwdThreads;     // generic dW2 ownership (other H)
  constexpr int K1 = (CIN * H + kBwdThreads - 1) / kBwdThreads;   // dW1 entries per thread (rows k < CIN)
  extern __shared__ __align__(16) float sm[];
  float* sW1s = sm + L::kW1s;
  float* sW2s = sm + L::kW2s;
  float* sW2t = sm + L::kW2t;
  float* sW1t = sm + L::kW1t;
  float* sB1 = sm + L::kB1;
  float* sB2 = sm + L::kB2;
  float* sW3 = sm + L::kW3;
  float* sB3 = sm + L::kB3;
  float* sX = sm + L::kX;
  float* sH1 = sm + L::kH1;
  float* sH2 = sm + L::kH2;     // H2, then dZ2
  float* sG1 = sm + L::kG1;     // dZ1
  float* sY = sm + L::kY;       // [tile][Q][4] partial outputs
  float* sDY = sm + L::kDY;
  float* sGK = sm + L::kGK;     // [T][CT] temporal gradient
  const int tid = threadIdx.x;
  for (int i = tid; i < CIN * HS; i += kBwdThreads) sW1s[i] = 0.0f;
  for (int i = tid; i < 2 * H * HS; i += kBwdThreads) sW2s[i] = 0.0f;   // W2s and W2t
  __syncthreads();
  for (int i = tid; i < CIN * H; i += kBwdThreads) {
    const int k = i / H, o = i % H;
    const float w = a.w1[i];
    sW1s[k * HS + L::skew(o)] = w;
    sW1t[o * CIN + k] = w;
  }
  for (int i = tid; i < H * H; i += kBwdThreads) {
    const int r = i / H, c = i % H;
    const float w = a.w2[i];   // W2[r][c]: input r, output c
    sW2s[r * HS + L::skew(c)] = w;
    sW2t[c * HS + L::skew(r)] = w;
  }
  for (int i = tid; i < H; i += kBwdThreads) {
    sB1[i] = a.b1[i];
    sB2[i] = a.b2[i];
  }
  for (int i = tid; i < H * 4; i += kBwdThreads) sW3[i] = (i % 4) < 3 ? a.w3[(i / 4) * 3 + (i % 4)] : 0.0f;
  if (tid < 4) sB3[tid] = tid < 3 ? a.b3[tid] : 0.0f;
  for (int i = tid; i < a.t_count * CT; i += kBwdThreads) sGK[i] = 0.0f;
  __syncthreads();

  const int r = tid / kFitQ, q = tid % kFitQ;   // this thread's sample in the tile and its quarter
  const int o0 = q * HQ;                         // its hidden units o0 .. o0+HQ-1
  const int c0 = L::skew(o0);                    // their first column in a skewed row
  float acc2[kBlocked ? 8 : K2], acc1[K1], acc3 = 0.0f, accb2[4] = {0, 0, 0, 0}, accb1 = 0.0f;
#pragma unroll
  for (int k = 0; k < (kBlocked ? 8 : K2); ++k) acc2[k] = 0.0f;
#pragma unroll
  for (int k = 0; k < K1; ++k) acc1[k] = 0.0f;
  double loss = 0.0;
  int64_t step = 0;
  if (MODE != 0) step = *a.step;

  const int64_t n_tiles = (a.n + kFitTile - 1) / kFitTile;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t s = tile * kFitTile + r;
    const bool valid = s < a.n;
    int ix = 0, iy = 0;
    float u = 0.5f, v = 0.5f, tq = 0.0f;
    if (valid) {
      if (MODE == 0) {
        u = a.uvt[3 * s];
        v = a.uvt[3 * s + 1];
        tq = a.uvt[3 * s + 2];
      } else {
        draw_sample(a.seed, step, s, a.lm_w, a.lm_h, ix, iy, tq);
        u = ((float)ix + 0.5f) / (float)a.lm_w;
        v = ((float)iy + 0.5f) / (float)a.lm_h;
      }
    }
    int j0, j1;
    float al;
    temporal_setup_k(tq, a.t_count, a.key_t, j0, j1, al);
    // ---- A1: features (spatial channels q*SC.., temporal q*TC.. of this thread) ----
    {
      TapInfo t[4];
      float fx, fy;
      fit_taps(a, u, v, t, fx, fy);
      const float gx = 1.0f - fx, gy = 1.0f - fy;
      float f[4][SC];
#pragma unroll
      for (int tq = 0; tq < 4; ++tq) {
        float d0[SC], d1[SC], d2[SC];
        if (valid) sim_values<SC>(a, t[tq].blk, q * SC, t[tq].p, f[tq], d0, d1, d2);
      }
#pragma unroll
      for (int kk = 0; kk < SC; ++kk)   // the decode's blend order
        sX[r * LX + q * SC + kk] =
            valid ? gy * (gx * f[0][kk] + fx * f[1][kk]) + fy * (gx * f[2][kk] + fx * f[3][kk]) : 0.0f;
      const float ga = 1.0f - al;
#pragma unroll
      for (int kk = 0; kk < TC; ++kk) {
        const int c = q * TC + kk;
        sX[r * LX + CS + c] = valid ? ga * a.temporal[j0 * CT + c] + al * a.temporal[j1 * CT + c] : 0.0f;
      }
    }
    __syncthreads();
    // ---- A2: layer 1, this thread's HQ units ----
    {
      float h[HQ];
#pragma unroll
      for (int u = 0; u < HQ; ++u) h[u] = sB1[o0 + u];
#pragma unroll 4
      for (int k = 0; k < CIN; ++k) {
        const float xv = sX[r * LX + k];
#pragma unroll
        for (int u4 = 0; u4 < HQ / 4; ++u4) {
          const float4 wv = *reinterpret_cast<const float4*>(sW1s + k * HS + c0 + 4 * u4);
          h[4 * u4] = fmaf(xv, wv.x, h[4 * u4]);
          h[4 * u4 + 1] = fmaf(xv, wv.y, h[4 * u4 + 1]);
          h[4 * u4 + 2] = fmaf(xv, wv.z, h[4 * u4 + 2]);
          h[4 * u4 + 3] = fmaf(xv, wv.w, h[4 * u4 + 3]);
        }
      }
#pragma unroll
      for (int u4 = 0; u4 < HQ / 4; ++u4)
        *reinterpret_cast<float4*>(sH1 + r * LH + o0 + 4 * u4) =
            valid ? make_float4(fmaxf(h[4 * u4], 0.0f), fmaxf(h[4 * u4 + 1], 0.0f), fmaxf(h[4 * u4 + 2], 0.0f),
                                fmaxf(h[4 * u4 + 3], 0.0f))
                  : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    __syncthreads();
    // ---- A3: layer 2 (this thread's HQ units) and its share of the output layer ----
    {
      float h[HQ];
#pragma unroll
      for (int u = 0; u < HQ; ++u) h[u] = sB2[o0 + u];
#pragma unroll 4
      for (int i = 0; i < H; ++i) {
        const float hv = sH1[r * LH + i];
#pragma unroll
        for (int u4 = 0; u4 < HQ / 4; ++u4) {
          const float4 wv = *reinterpret_cast<const float4*>(sW2s + i * HS + c0 + 4 * u4);
          h[4 * u4] = fmaf(hv, wv.x, h[4 * u4]);
          h[4 * u4 + 1] = fmaf(hv, wv.y, h[4 * u4 + 1]);
          h[4 * u4 + 2] = fmaf(hv, wv.z, h[4 * u4 + 2]);
          h[4 * u4 + 3] = fmaf(hv, wv.w, h[4 * u4 + 3]);
        }
      }
      float y0 = 0.0f, y1 = 0.0f, y2 = 0.0f;
#pragma unroll
      for (int u = 0; u < HQ; ++u) {
        h[u] = valid ? fmaxf(h[u], 0.0f) : 0.0f;
        const float4 w3 = *reinterpret_cast<const float4*>(sW3 + (o0 + u) * 4);
        y0 = fmaf(h[u], w3.x, y0);
        y1 = fmaf(h[u], w3.y, y1);
        y2 = fmaf(h[u], w3.z, y2);
      }
#pragma unroll
      for (int u4 = 0; u4 < HQ / 4; ++u4)
        *reinterpret_cast<float4*>(sH2 + r * LH + o0 + 4 * u4) =
            make_float4(h[4 * u4], h[4 * u4 + 1], h[4 * u4 + 2], h[4 * u4 + 3]);
      *reinterpret_cast<float4*>(sY + (r * kFitQ + q) * 4) = make_float4(y0, y1, y2, 0.0f);
    }
    __syncthreads();
    // ---- A4: output and dL/dy (one thread per sample) ----
    if (q == 0) {
      float dy0 = 0.f, dy1 = 0.f, dy2 = 0.f;
      if (valid) {
        float y0 = sB3[0], y1 = sB3[1], y2 = sB3[2];
#pragma unroll
        for (int qq = 0; qq < kFitQ; ++qq) {
          const float4 p = *reinterpret_cast<const float4*>(sY + (r * kFitQ + qq) * 4);
          y0 += p.x;
          y1 += p.y;
          y2 += p.z;
        }
        if (MODE == 0) {
          dy0 = a.grad_rgb[3 * s];
          dy1 = a.grad_rgb[3 * s + 1];
          dy2 = a.grad_rgb[3 * s + 2];
        } else {
          // the target at t: the keyframe targets around t interpolated like the features (Eq. 2)
          const int64_t plane = (int64_t)a.lm_h * a.lm_w * 3, px = ((int64_t)iy * a.lm_w + ix) * 3;
          const __half* t0 = a.targets + j0 * plane + px;
          const __half* t1 = a.targets + j1 * plane + px;
          const float ga = 1.0f - al;
          const float d0 = y0 - (ga * __half2float(t0[0]) + al * __half2float(t1[0]));
          const float d1 = y1 - (ga * __half2float(t0[1]) + al * __half2float(t1[1]));
          const float d2 = y2 - (ga * __half2float(t0[2]) + al * __half2float(t1[2]));
          loss += (double)d0 * d0 + (double)d1 * d1 + (double)d2 * d2;
          const float sc = 2.0f / (3.0f * (float)a.n);
          dy0 = sc * d0;
          dy1 = sc * d1;
          dy2 = sc * d2;
        }
      }
      *reinterpret_cast<float4*>(sDY + r * 4) = make_float4(dy0, dy1, dy2, 0.0f);
    }
    __syncthreads();
    // ---- B: dW3 += H2^T dY (3H owners), db3 (3 owners) ----
    if (tid < 3 * H) {
      const int o = tid / 3, c = tid % 3;
      for (int rr = 0; rr < kFitTile; ++rr) acc3 = fmaf(sH2[rr * LH + o], sDY[rr * 4 + c], acc3);
    } else if (tid < 3 * H + 3) {
      const int c = tid - 3 * H;
      for (int rr = 0; rr < kFitTile; ++rr) acc3 += sDY[rr * 4 + c];
    }
    __syncthreads();
    // ---- C1: dZ2 for this thread's units ----
    {
      const float4 dy = *reinterpret_cast<const float4*>(sDY + r * 4);
#pragma unroll
      for (int u4 = 0; u4 < HQ / 4; ++u4) {
        const float4 h = *reinterpret_cast<const float4*>(sH2 + r * LH + o0 + 4 * u4);
        const float hv[4] = {h.x, h.y, h.z, h.w};
        float g[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float4 w3 = *reinterpret_cast<const float4*>(sW3 + (o0 + 4 * u4 + e) * 4);
          const float gg = w3.x * dy.x + w3.y * dy.y + w3.z * dy.z;
          g[e] = (valid && hv[e] > 0.0f) ? gg : 0.0f;
        }
        *reinterpret_cast<float4*>(sH2 + r * LH + o0 + 4 * u4) = make_float4(g[0], g[1], g[2], g[3]);
      }
    }
    __syncthreads();
    // ---- C2: dZ1 for this thread's units: dZ1[i] = [h1_i > 0] sum_o W2[i][o] dZ2[o] ----
    {
      float g[HQ];
#pragma unroll
      for (int u = 0; u < HQ; ++u) g[u] = 0.0f;
#pragma unroll 4
      for (int o = 0; o < H; ++o) {
        const float gz = sH2[r * LH + o];
#pragma unroll
        for (int u4 = 0; u4 < HQ / 4; ++u4) {
          const float4 wv = *reinterpret_cast<const float4*>(sW2t + o * HS + c0 + 4 * u4);
          g[4 * u4] = fmaf(gz, wv.x, g[4 * u4]);
          g[4 * u4 + 1] = fmaf(gz, wv.y, g[4 * u4 + 1]);
          g[4 * u4 + 2] = fmaf(gz, wv.z, g[4 * u4 + 2]);
          g[4 * u4 + 3] = fmaf(gz, wv.w, g[4 * u4 + 3]);
        }
      }
#pragma unroll
      for (int u4 = 0; u4 < HQ / 4; ++u4) {
        const float4 h = *reinterpret_cast<const float4*>(sH1 + r * LH + o0 + 4 * u4);
        *reinterpret_cast<float4*>(sG1 + r * LH + o0 + 4 * u4) =
            make_float4(h.x > 0.0f ? g[4 * u4] : 0.0f, h.y > 0.0f ? g[4 * u4 + 1] : 0.0f,
                        h.z > 0.0f ? g[4 * u4 + 2] : 0.0f, h.w > 0.0f ? g[4 * u4 + 3] : 0.0f);
      }
    }
    __syncthreads();
    // ---- C3: dx for this thread's channels (W1^T rows), then the feature / temporal scatter ----
    if (valid) {
      float gs[SC], gt[TC];
#pragma unroll
      for (int kk = 0; kk < SC; ++kk) gs[kk] = 0.0f;
#pragma unroll
      for (int kk = 0; kk < TC; ++kk) gt[kk] = 0.0f;
#pragma unroll 4
      for (int o = 0; o < H; ++o) {
        const float gz = sG1[r * LH + o];
        float ws[SC], wt[TC];
        lds<SC>(sW1t + o * CIN + q * SC, ws);
        lds<TC>(sW1t + o * CIN + CS + q * TC, wt);
#pragma unroll
        for (int kk = 0; kk < SC; ++kk) gs[kk] = fmaf(gz, ws[kk], gs[kk]);
#pragma unroll
        for (int kk = 0; kk < TC; ++kk) gt[kk] = fmaf(gz, wt[kk], gt[kk]);
      }
      // v_t = (1 - alpha) K[j0] + alpha K[j1]: the gradient splits between the two rows
#pragma unroll
      for (int kk = 0; kk < TC; ++kk) {
        atomicAdd(&sGK[j0 * CT + q * TC + kk], (1.0f - al) * gt[kk]);
        if (al != 0.0f) atomicAdd(&sGK[j1 * CT + q * TC + kk], al * gt[kk]);
      }
      TapInfo t[4];
      float fx, fy;
      fit_taps(a, u, v, t, fx, fy);
      // per tap: the weight-index gradients (one texel each), and the endpoint
      // gradients of this thread's SC channels
      float gea[4][SC], geb[4][SC];
#pragma unroll
      for (int tq = 0; tq < 4; ++tq) {
        float fv[SC], dea[SC], deb[SC], dw[SC];
        sim_values<SC>(a, t[tq].blk, q * SC, t[tq].p, fv, dea, deb, dw);
#pragma unroll
        for (int kk = 0; kk < SC; ++kk) {
          const float gf = t[tq].wt * gs[kk];
          gea[tq][kk] = dea[kk] * gf;
          geb[tq][kk] = deb[kk] * gf;
          atomicAdd(&a.g_w[(t[tq].blk + q * SC + kk) * 16 + t[tq].p], dw[kk] * gf);
        }
      }
      // merge the endpoint gradients of taps in the same block, one reduction per block
#pragma unroll
      for (int tq = 0; tq < 4; ++tq) {
        bool first = true;
#pragma unroll
        for (int rq = 0; rq < tq; ++rq) first = first && (t[rq].blk != t[tq].blk);
        if (!first) continue;
        float sa[SC], sb[SC];
#pragma unroll
        for (int kk = 0; kk < SC; ++kk) {
          sa[kk] = gea[tq][kk];
          sb[kk] = geb[tq][kk];
        }
#pragma unroll
        for (int rq = tq + 1; rq < 4; ++rq) {
          if (t[rq].blk == t[tq].blk) {
#pragma unroll
            for (int kk = 0; kk < SC; ++kk) {
              sa[kk] += gea[rq][kk];
              sb[kk] += geb[rq][kk];
            }
          }
        }
        float* pa = a.g_ea + t[tq].blk + q * SC;
        float* pb = a.g_eb + t[tq].blk + q * SC;
        if constexpr (SC == 4) {
          if (a.vec_red) {
            asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(pa), "f"(sa[0]), "f"(sa[1]),
                         "f"(sa[2]), "f"(sa[3]) : "memory");
            asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(pb), "f"(sb[0]), "f"(sb[1]),
                         "f"(sb[2]), "f"(sb[3]) : "memory");
            continue;
          }
        } else if constexpr (SC == 2) {
          if (a.vec_red) {
            asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(pa), "f"(sa[0]), "f"(sa[1]) : "memory");
            asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(pb), "f"(sb[0]), "f"(sb[1]) : "memory");
            continue;
          }
        }
#pragma unroll
        for (int kk = 0; kk < SC; ++kk) {
          atomicAdd(pa + kk, sa[kk]);
          atomicAdd(pb + kk, sb[kk]);
        }
      }
    }
    // ---- D: dW2 += H1^T dZ2, dW1 += X^T dZ1, db2, db1 (sH1, sX, sH2 = dZ2, sG1 = dZ1 are final) ----
    if constexpr (kBlocked) {
      const int ob = tid % 16, ib = tid / 16;   // dW2 rows 2ib, 2ib+1 x columns 4ob .. 4ob+3
      for (int rr = 0; rr < kFitTile; ++rr) {
        const float2 h = *reinterpret_cast<const float2*>(sH1 + rr * LH + 2 * ib);
        const float4 g = *reinterpret_cast<const float4*>(sH2 + rr * LH + 4 * ob);
        acc2[0] = fmaf(h.x, g.x, acc2[0]);
        acc2[1] = fmaf(h.x, g.y, acc2[1]);
        acc2[2] = fmaf(h.x, g.z, acc2[2]);
        acc2[3] = fmaf(h.x, g.w, acc2[3]);
        acc2[4] = fmaf(h.y, g.x, acc2[4]);
        acc2[5] = fmaf(h.y, g.y, acc2[5]);
        acc2[6] = fmaf(h.y, g.z, acc2[6]);
        acc2[7] = fmaf(h.y, g.w, acc2[7]);
        if (ib == 0) {   // db2 = colsum dZ2
          accb2[0] += g.x;
          accb2[1] += g.y;
          accb2[2] += g.z;
          accb2[3] += g.w;
        }
      }
    } else {
      const int o = tid % H, i0 = tid / H;
      constexpr int RPT = kBwdThreads / H;
      for (int rr = 0; rr < kFitTile; ++rr) {
        const float g2 = sH2[rr * LH + o];
#pragma unroll
        for (int k = 0; k < K2; ++k)
          if (i0 + RPT * k < H) acc2[k] = fmaf(sH1[rr * LH + i0 + RPT * k], g2, acc2[k]);
        if (i0 == 0) accb2[0] += g2;
      }
    }
    {
      const int o = tid % H, k0 = tid / H;   // dW1 rows k0 + (512/H) m, column o; db1 by the first H threads
      constexpr int RPT = kBwdThreads / H;
      for (int rr = 0; rr < kFitTile; ++rr) {
        const float g1 = sG1[rr * LH + o];
#pragma unroll
        for (int m = 0; m < K1; ++m)
          if (k0 + RPT * m < CIN) acc1[m] = fmaf(sX[rr * LX + k0 + RPT * m], g1, acc1[m]);
        if (k0 == 0) accb1 += g1;
      }
    }
    __syncthreads();
  }
  // ---- flush per-CTA accumulators ----
  if constexpr (kBlocked) {
    const int ob = tid % 16, ib = tid / 16;
#pragma unroll
    for (int e = 0; e < 8; ++e) atomicAdd(&a.g_w2[(2 * ib + e / 4) * H + 4 * ob + e % 4], acc2[e]);
    if (ib == 0) {
#pragma unroll
      for (int e = 0; e < 4; ++e) atomicAdd(&a.g_b2[4 * ob + e], accb2[e]);
    }
  } else {
    const int o = tid % H, i0 = tid / H;
    constexpr int RPT = kBwdThreads / H;
#pragma unroll
    for (int k = 0; k < K2; ++k)
      if (i0 + RPT * k < H) atomicAdd(&a.g_w2[(i0 + RPT * k) * H + o], acc2[k]);
    if (i0 == 0) atomicAdd(&a.g_b2[o], accb2[0]);
  }
  {
    const int o = tid % H, k0 = tid / H;
    constexpr int RPT = kBwdThreads / H;
#pragma unroll
    for (int m = 0; m < K1; ++m)
      if (k0 + RPT * m < CIN) atomicAdd(&a.g_w1[(k0 + RPT * m) * H + o], acc1[m]);
    if (k0 == 0) atomicAdd(&a.g_b1[o], accb1);
  }
  if (tid < 3 * H) atomicAdd(&a.g_w3[(tid / 3) * 3 + tid % 3], acc3);
  else if (tid < 3 * H + 3) atomicAdd(&a.g_b3[tid - 3 * H], acc3);
  __syncthreads();
  for (int i = tid; i < a.t_count * CT; i += kBwdThreads) atomicAdd(&a.g_temporal[i], sGK[i]);
  if (MODE != 0) {
    for (int off = 16; off > 0; off >>= 1) loss += __shfl_down_sync(0xffffffffu, loss, off);
    if ((tid & 31) == 0) atomicAdd(a.loss_acc, loss);
  }
}

// ---------------------------------------------------------------------------
// Adam over all ten parameter tensors in one launch (Kingma & Ba).  The step
// number t = *step + 1 is read on the device so one captured step replays.
// Endpoints and weights are projected onto [0,1] (Eq. 6); during the freeze
// stage only the MLP tensors (k >= 4) are updated.
// ---------------------------------------------------------------------------
struct AdamTable {
  float* p[10];
  int64_t off[11];
  const float* g;
  float *m, *v;
  const int64_t* step;        // global step counter (steps already taken)
  const int64_t* local;       // steps taken in this call
  int64_t freeze_from;        // local step index from which features are frozen
  float lr, beta1, beta2, eps;
};

__global__ void k_adam(AdamTable t) {
  __shared__ float s_c1, s_c2;
  __shared__ int s_freeze;
  if (threadIdx.x == 0) {
    const double step = (double)(*t.step + 1);
    s_c1 = (float)(1.0 - pow((double)t.beta1, step));
    s_c2 = (float)(1.0 - pow((double)t.beta2, step));
    s_freeze = *t.local >= t.freeze_from;
  }
  __syncthreads();
  const float c1 = s_c1, c2 = s_c2;
  const int freeze = s_freeze;
  const int64_t n = t.off[10];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int k = 0;
#pragma unroll
    for (int q = 1; q < 10; ++q) k += (i >= t.off[q]);
    if (freeze && k < 4) continue;
    const float g = t.g[i];
    const float m = t.beta1 * t.m[i] + (1.0f - t.beta1) * g;
    const float v = t.beta2 * t.v[i] + (1.0f - t.beta2) * g * g;
    t.m[i] = m;
    t.v[i] = v;
    float* pp = t.p[k] + (i - t.off[k]);
    float q = *pp - t.lr * (m / c1) / (sqrtf(v / c2) + t.eps);
    if (k < 3) q = fminf(fmaxf(q, 0.0f), 1.0f);
    *pp = q;
  }
}

// Logs the batch loss (every `every` local steps) and advances the counters.
__global__ void k_fit_step_end(int64_t* step, int64_t* local, const double* loss_acc, double* loss_log, int every,
                               int64_t batch) {
  const int64_t l = *local;
  if (loss_log && every > 0 && l % every == 0) loss_log[l / every] = *loss_acc / (3.0 * (double)batch);
  *local = l + 1;
  *step = *step + 1;
}

// ---------------------------------------------------------------------------
// Launch helpers and shape dispatch
// ---------------------------------------------------------------------------
#define NDGI_FIT_SHAPES(X) \
  X(4, 4, 16)              \
  X(8, 8, 16)              \
  X(8, 8, 32)              \
  X(16, 8, 16)             \
  X(16, 8, 32)             \
  X(16, 8, 64)             \
  X(16, 16, 64)

static bool fit_supported(int cs, int ct, int h) {
#define X(A, B, C) if (cs == A && ct == B && h == C) return true;
  NDGI_FIT_SHAPES(X)
#undef X
  return false;
}

template <int CS, int CT, int H>
static size_t fit_smem_bytes(int t_count) {
  return (size_t)(FitSmem<CS, CT, H>::kFloatsNoGK + t_count * CT) * sizeof(float);
}

static cudaError_t launch_fit_backward(const FitArgs& args, int mode, cudaStream_t s) {
  FitArgs a = args;
  a.vec_red = ((reinterpret_cast<uintptr_t>(a.g_ea) | reinterpret_cast<uintptr_t>(a.g_eb)) & 15u) == 0u;
  a.vec_ld = ((reinterpret_cast<uintptr_t>(a.ea) | reinterpret_cast<uintptr_t>(a.eb)) & 15u) == 0u;
  const int64_t tiles = (a.n + kFitTile - 1) / kFitTile;
  const int models = a.n_models > 0 ? a.n_models : 1;
  // about two CTAs per SM in all (one model: one per SM), at most one per tile
  const int64_t cap = models == 1 ? (int64_t)num_sms() : ((int64_t)num_sms() * 2 + models - 1) / models;
  const int grid = (int)(tiles < cap ? (tiles > 0 ? tiles : 1) : cap);
#define X(A, B, C)                                                                                   \
  if (a.cs == A && a.ct == B && a.hidden == C) {                                                     \
    const size_t smem = fit_smem_bytes<A, B, C>(a.t_count);                                          \
    auto kern = mode == 0 ? k_fit_backward<A, B, C, 0>                                               \
                          : (models > 1 ? k_fit_backward<A, B, C, 2> : k_fit_backward<A, B, C, 1>);    \
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    if (e != cudaSuccess) return e;                                                                  \
    kern<<<dim3(grid, mode == 0 ? 1 : models), kBwdThreads, smem, s>>>(a);                           \
    return cudaGetLastError();                                                                       \
  }
  NDGI_FIT_SHAPES(X)
#undef X
  return cudaErrorInvalidValue;
}

static cudaError_t launch_fit_forward(const FitArgs& a, float* rgb, cudaStream_t s) {
  const int64_t blocks = (a.n + kFitThreads - 1) / kFitThreads;
  const int64_t cap = (int64_t)num_sms() * 16;
  const int grid = (int)(blocks < cap ? (blocks > 0 ? blocks : 1) : cap);
#define X(A, B, C)                                                   \
  if (a.cs == A && a.ct == B && a.hidden == C) {                     \
    k_fit_forward<A, B, C><<<grid, kFitThreads, 0, s>>>(a, rgb);     \
    return cudaGetLastError();                                       \
  }
  NDGI_FIT_SHAPES(X)
#undef X
  return cudaErrorInvalidValue;
}

static ndgi_status check_fit(const ndgi_fit_params* p, const char* who) {
  if (!p) return set_error(NDGI_ERR_INVALID_ARG, "%s: params is NULL", who);
  if (p->lm_w <= 0 || p->lm_h <= 0 || p->feat_w <= 0 || p->feat_h <= 0 || p->feat_w % 4 || p->feat_h % 4)
    return set_error(NDGI_ERR_INVALID_ARG, "%s: bad lightmap or feature size", who);
  if (p->t_count <= 0 || p->cs <= 0 || p->ct < 0 || p->hidden <= 0)
    return set_error(NDGI_ERR_INVALID_ARG, "%s: bad channel counts", who);
  if (!p->ea || !p->eb || !p->w || !p->w1 || !p->b1 || !p->w2 || !p->b2 || !p->w3 || !p->b3 ||
      (p->ct > 0 && !p->temporal))
    return set_error(NDGI_ERR_INVALID_ARG, "%s: a parameter pointer is NULL", who);
  if (p->address_mode != 0 && p->address_mode != 1)
    return set_error(NDGI_ERR_INVALID_ARG, "%s: address_mode must be 0 or 1", who);
  if (!fit_supported(p->cs, p->ct, p->hidden))
    return set_error(NDGI_ERR_UNSUPPORTED, "%s: shape cs=%d ct=%d hidden=%d is not built", who, p->cs, p->ct,
                     p->hidden);
  return NDGI_OK;
}

static FitArgs make_args(const ndgi_fit_params* p) {
  FitArgs a{};
  a.lm_w = p->lm_w; a.lm_h = p->lm_h; a.feat_w = p->feat_w; a.feat_h = p->feat_h; a.cs = p->cs;
  a.bw = p->feat_w / 4; a.t_count = p->t_count; a.ct = p->ct; a.hidden = p->hidden;
  a.address_mode = p->address_mode;
  a.key_t = p->key_t;
  a.n_models = 1;
  a.ea = p->ea; a.eb = p->eb; a.w = p->w; a.temporal = p->temporal;
  a.w1 = p->w1; a.b1 = p->b1; a.w2 = p->w2; a.b2 = p->b2; a.w3 = p->w3; a.b3 = p->b3;
  return a;
}

// Element counts of the ten tensors, in ndgi_fit_params order.
static void fit_sizes(const ndgi_fit_params* p, int64_t (&n)[10]) {
  const int64_t nb = (int64_t)(p->feat_w / 4) * (p->feat_h / 4) * p->cs;
  const int64_t cin = p->cs + p->ct, H = p->hidden;
  n[0] = nb; n[1] = nb; n[2] = nb * 16; n[3] = (int64_t)p->t_count * p->ct;
  n[4] = cin * H; n[5] = H; n[6] = H * H; n[7] = H; n[8] = H * 3; n[9] = 3;
}

static size_t round256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace ndgi

using namespace ndgi;

extern "C" {

ndgi_status ndgi_fit_forward(const ndgi_fit_params* params, const float* uvt, int64_t n, int32_t relaxed,
                             float* rgb, void* stream) {
  ndgi_status st = check_fit(params, "ndgi_fit_forward");
  if (st != NDGI_OK) return st;
  if (n < 0) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_fit_forward: n < 0");
  if (n == 0) return NDGI_OK;
  if (!uvt || !rgb) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_fit_forward: uvt or rgb is NULL");
  FitArgs a = make_args(params);
  a.relaxed = relaxed != 0;
  a.n = n;
  a.uvt = uvt;
  return cuda_status(launch_fit_forward(a, rgb, (cudaStream_t)stream), "ndgi_fit_forward");
}

ndgi_status ndgi_fit_backward(const ndgi_fit_params* params, const float* uvt, int64_t n, int32_t relaxed,
                              const float* grad_rgb, const ndgi_fit_grads* grads, void* stream) {
  ndgi_status st = check_fit(params, "ndgi_fit_backward");
  if (st != NDGI_OK) return st;
  if (n < 0) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_fit_backward: n < 0");
  if (n == 0) return NDGI_OK;
  if (!uvt || !grad_rgb || !grads)
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_fit_backward: uvt, grad_rgb or grads is NULL");
  if (!grads->ea || !grads->eb || !grads->w || !grads->w1 || !grads->b1 || !grads->w2 || !grads->b2 || !grads->w3 ||
      !grads->b3 || (params->ct > 0 && !grads->temporal))
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_fit_backward: a gradient pointer is NULL");
  FitArgs a = make_args(params);
  a.relaxed = relaxed != 0;
  a.n = n;
  a.uvt = uvt;
  a.grad_rgb = grad_rgb;
  a.g_ea = grads->ea; a.g_eb = grads->eb; a.g_w = grads->w; a.g_temporal = grads->temporal;
  a.g_w1 = grads->w1; a.g_b1 = grads->b1; a.g_w2 = grads->w2; a.g_b2 = grads->b2; a.g_w3 = grads->w3;
  a.g_b3 = grads->b3;
  return cuda_status(launch_fit_backward(a, 0, (cudaStream_t)stream), "ndgi_fit_backward");
}

size_t ndgi_encode_fit_batch_workspace_size(const ndgi_fit_params* params, int32_t n_models,
                                            const ndgi_fit_config* cfg) {
  (void)cfg;
  if (!params || n_models < 1) return 0;
  int64_t n[10];
  fit_sizes(params, n);
  int64_t tot = 0;
  for (int k = 0; k < 10; ++k) tot += n[k] * n_models;
  return 256 + 3 * round256((size_t)tot * sizeof(float));
}

size_t ndgi_encode_fit_workspace_size(const ndgi_fit_params* params, const ndgi_fit_config* cfg) {
  return ndgi_encode_fit_batch_workspace_size(params, 1, cfg);
}

}  // extern "C"

namespace ndgi {
static ndgi_status encode_fit(const ndgi_fit_params* params, int32_t n_models, const uint16_t* targets,
                              const ndgi_fit_config* cfg, int32_t step_offset, void* ws, size_t ws_bytes,
                              double* loss_log, void* stream) {
  ndgi_status st = check_fit(params, "ndgi_encode_fit");
  if (st != NDGI_OK) return st;
  if (n_models < 1 || n_models > 65535)   // one CTA row (grid y) per model
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_encode_fit_batch: n_models must be in 1..65535");
  if (!cfg || !targets || !ws) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_encode_fit: NULL argument");
  if ((uintptr_t)targets % 2 || (uintptr_t)loss_log % 8)
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_encode_fit: targets must be 2-byte and loss_log 8-byte aligned");
  if (cfg->steps < 0 || cfg->batch <= 0 || cfg->freeze_steps < 0 || cfg->loss_every < 0 || step_offset < 0)
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_encode_fit: bad config");
  if (!(cfg->lr > 0.0f) || !(cfg->beta1 >= 0.0f && cfg->beta1 < 1.0f) || !(cfg->beta2 >= 0.0f && cfg->beta2 < 1.0f))
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_encode_fit: bad optimiser settings");
  const size_t need = ndgi_encode_fit_batch_workspace_size(params, n_models, cfg);
  if (ws_bytes < need || ((uintptr_t)ws % 256))
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_encode_fit: ws must be 256-byte aligned with >= %zu bytes", need);
  if (cfg->steps == 0) return NDGI_OK;
  cudaStream_t s = (cudaStream_t)stream;
  int64_t n[10], per_model[10];
  fit_sizes(params, per_model);
  for (int k = 0; k < 10; ++k) n[k] = per_model[k] * n_models;
  int64_t tot = 0;
  AdamTable t{};
  float* pp[10] = {params->ea, params->eb, params->w, params->temporal, params->w1,
                   params->b1, params->w2, params->b2, params->w3, params->b3};
  for (int k = 0; k < 10; ++k) {
    t.p[k] = pp[k];
    t.off[k] = tot;
    tot += n[k];
  }
  t.off[10] = tot;
  unsigned char* base = static_cast<unsigned char*>(ws);
  int64_t* d_step = reinterpret_cast<int64_t*>(base);
  int64_t* d_local = d_step + 1;
  double* d_loss = reinterpret_cast<double*>(base + 16);
  const size_t tb = round256((size_t)tot * sizeof(float));
  float* g = reinterpret_cast<float*>(base + 256);
  float* m = reinterpret_cast<float*>(base + 256 + tb);
  float* v = reinterpret_cast<float*>(base + 256 + 2 * tb);
  // Counters: global step = step_offset, local = 0.  Fresh runs zero the moments.
  const int64_t init[2] = {step_offset, 0};
  cudaError_t e = cudaMemcpyAsync(d_step, init, sizeof(init), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // `init` lives on this stack frame
  if (e == cudaSuccess && step_offset == 0) e = cudaMemsetAsync(m, 0, 2 * tb, s);
  if (e != cudaSuccess) return cuda_status(e, "ndgi_encode_fit: init");
  t.g = g;
  t.m = m;
  t.v = v;
  t.step = d_step;
  t.local = d_local;
  t.freeze_from = (int64_t)cfg->steps - cfg->freeze_steps;
  t.lr = cfg->lr;
  t.beta1 = cfg->beta1;
  t.beta2 = cfg->beta2;
  t.eps = cfg->eps;

  FitArgs a = make_args(params);
  a.relaxed = cfg->relaxed != 0;
  a.n = cfg->batch;
  a.targets = reinterpret_cast<const __half*>(targets);
  a.seed = cfg->seed;
  a.step = d_step;
  a.loss_acc = d_loss;
  a.n_models = n_models;
  for (int k = 0; k < 10; ++k) a.ms[k] = per_model[k];
  a.tgt_stride = (int64_t)params->t_count * params->lm_h * params->lm_w * 3;
  float* gp[10];
  for (int k = 0; k < 10; ++k) gp[k] = g + t.off[k];
  a.g_ea = gp[0]; a.g_eb = gp[1]; a.g_w = gp[2]; a.g_temporal = gp[3]; a.g_w1 = gp[4];
  a.g_b1 = gp[5]; a.g_w2 = gp[6]; a.g_b2 = gp[7]; a.g_w3 = gp[8]; a.g_b3 = gp[9];

  // Capture one step (zero grads and loss, forward+backward, Adam, counters)
  // and replay it cfg->steps times.
  cudaStream_t cs_ = nullptr;
  e = cudaStreamCreateWithFlags(&cs_, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_status(e, "ndgi_encode_fit: stream");
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  e = cudaStreamBeginCapture(cs_, cudaStreamCaptureModeThreadLocal);
  cudaError_t le = cudaSuccess;
  if (e == cudaSuccess) {
    le = cudaMemsetAsync(g, 0, (size_t)tot * sizeof(float), cs_);
    if (le == cudaSuccess) le = cudaMemsetAsync(d_loss, 0, sizeof(double), cs_);
    if (le == cudaSuccess) le = launch_fit_backward(a, 1, cs_);
    if (le == cudaSuccess) {
      const int threads = 256;
      int64_t blocks = (tot + threads - 1) / threads;
      if (blocks > (int64_t)num_sms() * 8) blocks = (int64_t)num_sms() * 8;
      k_adam<<<(int)blocks, threads, 0, cs_>>>(t);
      le = cudaGetLastError();
    }
    if (le == cudaSuccess) {
      k_fit_step_end<<<1, 1, 0, cs_>>>(d_step, d_local, d_loss, loss_log, cfg->loss_every,
                                       (int64_t)cfg->batch * n_models);
      le = cudaGetLastError();
    }
    e = cudaStreamEndCapture(cs_, &graph);
  }
  if (le != cudaSuccess) e = le;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  for (int i = 0; e == cudaSuccess && i < cfg->steps; ++i) e = cudaGraphLaunch(exec, s);
  if (exec) cudaGraphExecDestroy(exec);
  cudaStreamDestroy(cs_);
  return cuda_status(e, "ndgi_encode_fit");
}
}  // namespace ndgi

extern "C" {

ndgi_status ndgi_encode_fit(const ndgi_fit_params* params, const uint16_t* targets, const ndgi_fit_config* cfg,
                            int32_t step_offset, void* ws, size_t ws_bytes, double* loss_log, void* stream) {
  return ndgi::encode_fit(params, 1, targets, cfg, step_offset, ws, ws_bytes, loss_log, stream);
}

ndgi_status ndgi_encode_fit_batch(const ndgi_fit_params* params, int32_t n_models, const uint16_t* targets,
                                  const ndgi_fit_config* cfg, int32_t step_offset, void* ws, size_t ws_bytes,
                                  double* loss_log, void* stream) {
  return ndgi::encode_fit(params, n_models, targets, cfg, step_offset, ws, ws_bytes, loss_log, stream);
}

}  // extern "C"
