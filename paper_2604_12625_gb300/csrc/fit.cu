// Differentiable fit of the decoder (Sec. 3.4 BC simulation, Sec. 4 training).
//
// Forward per sample (texel ix, iy of keyframe j): the four bilinear taps of
// the feature map are rebuilt from the block endpoints and weights (Eq. 7)
// with straight-through quantisation, so the features equal the packed BC4
// decode bit for bit; the temporal feature is keyframe row j; then the MLP.
//
// Backward (recompute, nothing stored between passes): a persistent CTA
// processes tiles of 128 samples.  Per tile each thread runs its sample's
// forward, then the backward of the output and hidden layers; the weight
// gradients of the tile are the contractions H2^T dY, H1^T dZ2 and X^T dZ1
// over the tile's samples, done from shared memory into per-thread register
// accumulators that persist across tiles and are flushed once per CTA.
// Temporal-line gradients (every sample hits one of T rows) are reduced in
// shared memory first.  Feature-map gradients go straight to global memory
// with FP32 atomics, after merging the endpoint gradients of taps that fall
// in the same block.
#include <cmath>

#include "ndgi_internal.h"
#include "bc4.cuh"
#include "fit.h"

namespace ndgi {

constexpr int kFitThreads = 128;
constexpr int kFitTile = 128;

struct FitArgs {
  int lm_w, lm_h, feat_w, feat_h, cs, bw, t_count, ct, hidden, address_mode;
  const float *ea, *eb, *w, *temporal, *w1, *b1, *w2, *b2, *w3, *b3;
  float *g_ea, *g_eb, *g_w, *g_temporal, *g_w1, *g_b1, *g_w2, *g_b2, *g_w3, *g_b3;
  int relaxed;
  int64_t n;
  const int32_t* samples;       // mode 0
  const float* grad_rgb;        // mode 0
  const __half* targets;        // mode 1: [T][lm_h][lm_w][3]
  uint64_t seed;                // mode 1
  const int64_t* step;          // mode 1: device step counter
  double* loss_acc;             // mode 1: sum of squared errors
};

// ---------------------------------------------------------------------------
// Counter-based sample stream: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ void draw_sample(uint64_t seed, int64_t step, int64_t i, int lm_w, int lm_h, int T,
                                            int& ix, int& iy, int& j) {
  const uint64_t g = 0x9E3779B97F4A7C15ull;
  const uint64_t ctr = ((uint64_t)step << 32) + (uint64_t)i;
  const uint64_t base = seed + 2ull * ctr * g;
  const uint64_t z1 = splitmix64(base);
  const uint64_t z2 = splitmix64(base + g);
  ix = (int)((uint32_t)z1 % (uint32_t)lm_w);
  iy = (int)((uint32_t)(z1 >> 32) % (uint32_t)lm_h);
  j = (int)((uint32_t)z2 % (uint32_t)T);
}

// ---------------------------------------------------------------------------
// BC-simulated feature texel and its straight-through chain-rule factors.
// ---------------------------------------------------------------------------
struct TapInfo {
  int64_t blk;    // (by*bw + bx)*cs  (channel 0)
  int p;          // texel in block
  float wt;       // bilinear weight
};

__device__ __forceinline__ void fit_taps(const FitArgs& a, int ix, int iy, TapInfo (&t)[4], float& fx, float& fy) {
  const float u = ((float)ix + 0.5f) / (float)a.lm_w;
  const float v = ((float)iy + 0.5f) / (float)a.lm_h;
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

template <int CS, int CT>
__device__ __forceinline__ void fit_gather(const FitArgs& a, int ix, int iy, int j, float (&x)[CS + CT]) {
  TapInfo t[4];
  float fx, fy;
  fit_taps(a, ix, iy, t, fx, fy);
  const float gx = 1.0f - fx, gy = 1.0f - fy;
#pragma unroll
  for (int c = 0; c < CS; ++c) {
    float f[4], d0, d1, d2;
#pragma unroll
    for (int q = 0; q < 4; ++q) f[q] = sim_value(a, t[q].blk + c, t[q].p, d0, d1, d2);
    x[c] = gy * (gx * f[0] + fx * f[1]) + fy * (gx * f[2] + fx * f[3]);   // same blend order as the decode
  }
#pragma unroll
  for (int c = 0; c < CT; ++c) x[CS + c] = a.temporal[j * CT + c];
}

// ---------------------------------------------------------------------------
// Forward only (one thread per sample).
// ---------------------------------------------------------------------------
template <int CS, int CT, int H>
__global__ void __launch_bounds__(kFitThreads) k_fit_forward(FitArgs a, float* __restrict__ rgb) {
  constexpr int CIN = CS + CT;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < a.n; s += (int64_t)gridDim.x * blockDim.x) {
    const int ix = a.samples[3 * s], iy = a.samples[3 * s + 1], j = a.samples[3 * s + 2];
    float x[CIN];
    fit_gather<CS, CT>(a, ix, iy, j, x);
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
// Backward (persistent, tiles of 128 samples).  MODE 0: samples + dL/drgb
// given.  MODE 1: samples drawn on device, dL/drgb from the MSE against the
// FP16 targets, FP64 loss accumulated.
// ---------------------------------------------------------------------------
template <int CS, int CT, int H>
struct FitSmem {
  static constexpr int CIN = CS + CT;
  static constexpr int LX = CIN + 1, LH = H + 1;
  static constexpr int kW1 = 0, kB1 = kW1 + CIN * H, kW2 = kB1 + H, kW2t = kW2 + H * H, kB2 = kW2t + H * H;
  static constexpr int kW3 = kB2 + H, kB3 = kW3 + H * 4;
  static constexpr int kX = kB3 + 4, kH1 = kX + kFitTile * LX, kH2 = kH1 + kFitTile * LH;
  static constexpr int kG1 = kH2 + kFitTile * LH, kDY = kG1 + kFitTile * LH, kGK = kDY + kFitTile * 4;
  static constexpr int kFloatsNoGK = kGK;
};

template <int CS, int CT, int H, int MODE>
__global__ void __launch_bounds__(kFitThreads, 1) k_fit_backward(FitArgs a) {
  using L = FitSmem<CS, CT, H>;
  constexpr int CIN = CS + CT;
  constexpr int LX = L::LX, LH = L::LH;
  constexpr int RPT = kFitThreads / H;          // row stride of owned weight-gradient entries
  constexpr int K2 = H * H / kFitThreads;       // owned entries of dW2
  constexpr int K1 = CIN * H / kFitThreads;     // owned entries of dW1
  static_assert(kFitThreads % H == 0 && (CIN * H) % kFitThreads == 0 && (H * H) % kFitThreads == 0, "shape");
  extern __shared__ __align__(16) float sm[];
  float* sW1 = sm + L::kW1;
  float* sB1 = sm + L::kB1;
  float* sW2 = sm + L::kW2;
  float* sW2t = sm + L::kW2t;
  float* sB2 = sm + L::kB2;
  float* sW3 = sm + L::kW3;
  float* sB3 = sm + L::kB3;
  float* sX = sm + L::kX;
  float* sH1 = sm + L::kH1;
  float* sH2 = sm + L::kH2;     // H2, then dZ2
  float* sG1 = sm + L::kG1;     // dZ1
  float* sDY = sm + L::kDY;
  float* sGK = sm + L::kGK;     // [T][CT] temporal gradient
  const int tid = threadIdx.x;
  for (int i = tid; i < CIN * H; i += kFitThreads) sW1[i] = a.w1[i];
  for (int i = tid; i < H * H; i += kFitThreads) {
    sW2[i] = a.w2[i];
    sW2t[(i % H) * H + i / H] = a.w2[i];
  }
  for (int i = tid; i < H; i += kFitThreads) {
    sB1[i] = a.b1[i];
    sB2[i] = a.b2[i];
  }
  for (int i = tid; i < H * 4; i += kFitThreads) sW3[i] = (i % 4) < 3 ? a.w3[(i / 4) * 3 + (i % 4)] : 0.0f;
  if (tid < 4) sB3[tid] = tid < 3 ? a.b3[tid] : 0.0f;
  for (int i = tid; i < a.t_count * CT; i += kFitThreads) sGK[i] = 0.0f;
  __syncthreads();

  float acc2[K2], acc1[K1], acc3[3] = {0, 0, 0}, accb = 0.0f, accb12 = 0.0f;
#pragma unroll
  for (int k = 0; k < K2; ++k) acc2[k] = 0.0f;
#pragma unroll
  for (int k = 0; k < K1; ++k) acc1[k] = 0.0f;
  double loss = 0.0;
  int64_t step = 0;
  if (MODE == 1) step = *a.step;

  const int64_t n_tiles = (a.n + kFitTile - 1) / kFitTile;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t s = tile * kFitTile + tid;
    const bool valid = s < a.n;
    int ix = 0, iy = 0, j = 0;
    float h1[H];
    float dy0 = 0.f, dy1 = 0.f, dy2 = 0.f;
    // ---- phase A: forward of this thread's sample ----
    if (valid) {
      if (MODE == 0) {
        ix = a.samples[3 * s];
        iy = a.samples[3 * s + 1];
        j = a.samples[3 * s + 2];
      } else {
        draw_sample(a.seed, step, s, a.lm_w, a.lm_h, a.t_count, ix, iy, j);
      }
      float x[CIN];
      fit_gather<CS, CT>(a, ix, iy, j, x);
#pragma unroll
      for (int i = 0; i < CIN; ++i) sX[tid * LX + i] = x[i];
#pragma unroll
      for (int o = 0; o < H; ++o) h1[o] = sB1[o];
#pragma unroll
      for (int i = 0; i < CIN; ++i) {
#pragma unroll
        for (int o = 0; o < H; ++o) h1[o] = fmaf(x[i], sW1[i * H + o], h1[o]);
      }
#pragma unroll
      for (int o = 0; o < H; ++o) {
        h1[o] = fmaxf(h1[o], 0.0f);
        sH1[tid * LH + o] = h1[o];
      }
      float y0 = sB3[0], y1 = sB3[1], y2 = sB3[2];
#pragma unroll 4
      for (int o = 0; o < H; ++o) {
        float z = sB2[o];
#pragma unroll
        for (int i = 0; i < H; ++i) z = fmaf(h1[i], sW2t[o * H + i], z);
        const float h = fmaxf(z, 0.0f);
        sH2[tid * LH + o] = h;
        y0 = fmaf(h, sW3[o * 4 + 0], y0);
        y1 = fmaf(h, sW3[o * 4 + 1], y1);
        y2 = fmaf(h, sW3[o * 4 + 2], y2);
      }
      if (MODE == 0) {
        dy0 = a.grad_rgb[3 * s];
        dy1 = a.grad_rgb[3 * s + 1];
        dy2 = a.grad_rgb[3 * s + 2];
      } else {
        const __half* tg = a.targets + (((int64_t)j * a.lm_h + iy) * a.lm_w + ix) * 3;
        const float d0 = y0 - __half2float(tg[0]), d1 = y1 - __half2float(tg[1]), d2 = y2 - __half2float(tg[2]);
        loss += (double)d0 * d0 + (double)d1 * d1 + (double)d2 * d2;
        const float sc = 2.0f / (3.0f * (float)a.n);
        dy0 = sc * d0;
        dy1 = sc * d1;
        dy2 = sc * d2;
      }
    } else {
#pragma unroll
      for (int i = 0; i < CIN; ++i) sX[tid * LX + i] = 0.0f;
#pragma unroll
      for (int o = 0; o < H; ++o) {
        sH1[tid * LH + o] = 0.0f;
        sH2[tid * LH + o] = 0.0f;
      }
    }
    sDY[tid * 4 + 0] = dy0;
    sDY[tid * 4 + 1] = dy1;
    sDY[tid * 4 + 2] = dy2;
    sDY[tid * 4 + 3] = 0.0f;
    __syncthreads();
    // ---- phase B: dW3 += H2^T dY, db3 += colsum dY ----
    if (tid < H) {
      for (int r = 0; r < kFitTile; ++r) {
        const float h = sH2[r * LH + tid];
        acc3[0] = fmaf(h, sDY[r * 4 + 0], acc3[0]);
        acc3[1] = fmaf(h, sDY[r * 4 + 1], acc3[1]);
        acc3[2] = fmaf(h, sDY[r * 4 + 2], acc3[2]);
      }
    } else if (tid >= kFitThreads - 3) {
      const int c = tid - (kFitThreads - 3);
      for (int r = 0; r < kFitTile; ++r) accb += sDY[r * 4 + c];
    }
    __syncthreads();
    // ---- phase C: per-sample backward through layers 2, 1 and the gather ----
    if (valid) {
      float gz2[H];
#pragma unroll
      for (int o = 0; o < H; ++o) {
        const float h = sH2[tid * LH + o];
        const float g = sW3[o * 4] * dy0 + sW3[o * 4 + 1] * dy1 + sW3[o * 4 + 2] * dy2;
        gz2[o] = h > 0.0f ? g : 0.0f;
        sH2[tid * LH + o] = gz2[o];
      }
      float gz1[H];
#pragma unroll 4
      for (int i = 0; i < H; ++i) {
        const float4* row = reinterpret_cast<const float4*>(sW2 + i * H);
        float g = 0.0f;
#pragma unroll
        for (int o4 = 0; o4 < H / 4; ++o4) {
          const float4 w = row[o4];
          g = fmaf(w.x, gz2[4 * o4], g);
          g = fmaf(w.y, gz2[4 * o4 + 1], g);
          g = fmaf(w.z, gz2[4 * o4 + 2], g);
          g = fmaf(w.w, gz2[4 * o4 + 3], g);
        }
        gz1[i] = sH1[tid * LH + i] > 0.0f ? g : 0.0f;
        sG1[tid * LH + i] = gz1[i];
      }
      float gx[CIN];
#pragma unroll
      for (int k = 0; k < CIN; ++k) {
        const float4* row = reinterpret_cast<const float4*>(sW1 + k * H);
        float g = 0.0f;
#pragma unroll
        for (int o4 = 0; o4 < H / 4; ++o4) {
          const float4 w = row[o4];
          g = fmaf(w.x, gz1[4 * o4], g);
          g = fmaf(w.y, gz1[4 * o4 + 1], g);
          g = fmaf(w.z, gz1[4 * o4 + 2], g);
          g = fmaf(w.w, gz1[4 * o4 + 3], g);
        }
        gx[k] = g;
      }
#pragma unroll
      for (int c = 0; c < CT; ++c) atomicAdd(&sGK[j * CT + c], gx[CS + c]);
      TapInfo t[4];
      float fx, fy;
      fit_taps(a, ix, iy, t, fx, fy);
#pragma unroll
      for (int c = 0; c < CS; ++c) {
        float gea[4], geb[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float dea, deb, dw;
          const int64_t bc = t[q].blk + c;
          sim_value(a, bc, t[q].p, dea, deb, dw);
          const float gf = t[q].wt * gx[c];
          gea[q] = dea * gf;
          geb[q] = deb * gf;
          atomicAdd(&a.g_w[bc * 16 + t[q].p], dw * gf);
        }
        // merge the endpoint gradients of taps in the same block
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          bool first = true;
#pragma unroll
          for (int r = 0; r < q; ++r) first = first && (t[r].blk != t[q].blk);
          if (!first) continue;
          float sa = gea[q], sb = geb[q];
#pragma unroll
          for (int r = q + 1; r < 4; ++r) {
            if (t[r].blk == t[q].blk) {
              sa += gea[r];
              sb += geb[r];
            }
          }
          atomicAdd(&a.g_ea[t[q].blk + c], sa);
          atomicAdd(&a.g_eb[t[q].blk + c], sb);
        }
      }
    } else {
#pragma unroll
      for (int o = 0; o < H; ++o) {
        sH2[tid * LH + o] = 0.0f;
        sG1[tid * LH + o] = 0.0f;
      }
    }
    __syncthreads();
    // ---- phase D: dW2 += H1^T dZ2, dW1 += X^T dZ1, db1, db2 ----
    {
      const int o = tid % H, i0 = tid / H;
      for (int r = 0; r < kFitTile; ++r) {
        const float g2 = sH2[r * LH + o];
        const float g1 = sG1[r * LH + o];
#pragma unroll
        for (int k = 0; k < K2; ++k) acc2[k] = fmaf(sH1[r * LH + i0 + RPT * k], g2, acc2[k]);
#pragma unroll
        for (int k = 0; k < K1; ++k) acc1[k] = fmaf(sX[r * LX + i0 + RPT * k], g1, acc1[k]);
        if (i0 == 0) accb12 += g2;        // db2 = colsum dZ2
        else if (i0 == 1) accb12 += g1;   // db1 = colsum dZ1
      }
    }
    __syncthreads();
  }
  // ---- flush per-CTA accumulators ----
  {
    const int o = tid % H, i0 = tid / H;
#pragma unroll
    for (int k = 0; k < K2; ++k) atomicAdd(&a.g_w2[(i0 + RPT * k) * H + o], acc2[k]);
#pragma unroll
    for (int k = 0; k < K1; ++k) atomicAdd(&a.g_w1[(i0 + RPT * k) * H + o], acc1[k]);
  }
  if (tid < H) {
    atomicAdd(&a.g_w3[tid * 3 + 0], acc3[0]);
    atomicAdd(&a.g_w3[tid * 3 + 1], acc3[1]);
    atomicAdd(&a.g_w3[tid * 3 + 2], acc3[2]);
  } else if (tid >= kFitThreads - 3) {
    atomicAdd(&a.g_b3[tid - (kFitThreads - 3)], accb);
  }
  {
    const int o = tid % H, i0 = tid / H;
    if (i0 == 0) atomicAdd(&a.g_b2[o], accb12);
    else if (i0 == 1) atomicAdd(&a.g_b1[o], accb12);
  }
  __syncthreads();
  for (int i = tid; i < a.t_count * CT; i += kFitThreads) atomicAdd(&a.g_temporal[i], sGK[i]);
  if (MODE == 1) {
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

static cudaError_t launch_fit_backward(const FitArgs& a, int mode, cudaStream_t s) {
  const int64_t tiles = (a.n + kFitTile - 1) / kFitTile;
  const int64_t cap = num_sms();
  const int grid = (int)(tiles < cap ? (tiles > 0 ? tiles : 1) : cap);
#define X(A, B, C)                                                                                   \
  if (a.cs == A && a.ct == B && a.hidden == C) {                                                     \
    const size_t smem = fit_smem_bytes<A, B, C>(a.t_count);                                          \
    auto kern = mode == 0 ? k_fit_backward<A, B, C, 0> : k_fit_backward<A, B, C, 1>;                  \
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    if (e != cudaSuccess) return e;                                                                  \
    kern<<<grid, kFitThreads, smem, s>>>(a);                                                         \
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

ndgi_status ndgi_fit_forward(const ndgi_fit_params* params, const int32_t* samples, int64_t n, int32_t relaxed,
                             float* rgb, void* stream) {
  ndgi_status st = check_fit(params, "ndgi_fit_forward");
  if (st != NDGI_OK) return st;
  if (n < 0) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_fit_forward: n < 0");
  if (n == 0) return NDGI_OK;
  if (!samples || !rgb) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_fit_forward: samples or rgb is NULL");
  FitArgs a = make_args(params);
  a.relaxed = relaxed != 0;
  a.n = n;
  a.samples = samples;
  return cuda_status(launch_fit_forward(a, rgb, (cudaStream_t)stream), "ndgi_fit_forward");
}

ndgi_status ndgi_fit_backward(const ndgi_fit_params* params, const int32_t* samples, int64_t n, int32_t relaxed,
                              const float* grad_rgb, const ndgi_fit_grads* grads, void* stream) {
  ndgi_status st = check_fit(params, "ndgi_fit_backward");
  if (st != NDGI_OK) return st;
  if (n < 0) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_fit_backward: n < 0");
  if (n == 0) return NDGI_OK;
  if (!samples || !grad_rgb || !grads)
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_fit_backward: samples, grad_rgb or grads is NULL");
  if (!grads->ea || !grads->eb || !grads->w || !grads->w1 || !grads->b1 || !grads->w2 || !grads->b2 || !grads->w3 ||
      !grads->b3 || (params->ct > 0 && !grads->temporal))
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_fit_backward: a gradient pointer is NULL");
  FitArgs a = make_args(params);
  a.relaxed = relaxed != 0;
  a.n = n;
  a.samples = samples;
  a.grad_rgb = grad_rgb;
  a.g_ea = grads->ea; a.g_eb = grads->eb; a.g_w = grads->w; a.g_temporal = grads->temporal;
  a.g_w1 = grads->w1; a.g_b1 = grads->b1; a.g_w2 = grads->w2; a.g_b2 = grads->b2; a.g_w3 = grads->w3;
  a.g_b3 = grads->b3;
  return cuda_status(launch_fit_backward(a, 0, (cudaStream_t)stream), "ndgi_fit_backward");
}

size_t ndgi_encode_fit_workspace_size(const ndgi_fit_params* params, const ndgi_fit_config* cfg) {
  (void)cfg;
  if (!params) return 0;
  int64_t n[10];
  fit_sizes(params, n);
  int64_t tot = 0;
  for (int k = 0; k < 10; ++k) tot += n[k];
  return 256 + 3 * round256((size_t)tot * sizeof(float));
}

ndgi_status ndgi_encode_fit(const ndgi_fit_params* params, const uint16_t* targets, const ndgi_fit_config* cfg,
                            int32_t step_offset, void* ws, size_t ws_bytes, double* loss_log, void* stream) {
  ndgi_status st = check_fit(params, "ndgi_encode_fit");
  if (st != NDGI_OK) return st;
  if (!cfg || !targets || !ws) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_encode_fit: NULL argument");
  if (cfg->steps < 0 || cfg->batch <= 0 || cfg->freeze_steps < 0 || cfg->loss_every < 0 || step_offset < 0)
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_encode_fit: bad config");
  if (!(cfg->lr > 0.0f) || !(cfg->beta1 >= 0.0f && cfg->beta1 < 1.0f) || !(cfg->beta2 >= 0.0f && cfg->beta2 < 1.0f))
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_encode_fit: bad optimiser settings");
  const size_t need = ndgi_encode_fit_workspace_size(params, cfg);
  if (ws_bytes < need || ((uintptr_t)ws % 256))
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_encode_fit: ws must be 256-byte aligned with >= %zu bytes", need);
  if (cfg->steps == 0) return NDGI_OK;
  cudaStream_t s = (cudaStream_t)stream;
  int64_t n[10];
  fit_sizes(params, n);
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
      k_fit_step_end<<<1, 1, 0, cs_>>>(d_step, d_local, d_loss, loss_log, cfg->loss_every, cfg->batch);
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

}  // extern "C"
