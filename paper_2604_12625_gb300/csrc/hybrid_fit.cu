// Fit of the hybrid decoder (Sec. 3.4's BC simulation, Eq. 6-7, applied to
// the decoder of Sec. 3.3): F_uv and every F3D t-slice are trained as BC
// endpoints (ea, eb) per block and channel plus a weight per texel, read
// through the straight-through quantisers of the simple fit (A = q255(ea),
// B = q255(eb), k = q7(w), value P35/8925; the backward treats them as the
// identity with quantised chain-rule factors); F_ut and F_vt are continuous
// values; the MLP is the hybrid decoder's (GELU hidden layers).  Everything is
// FP32 on the CUDA cores:
//   - k_hfit_forward: one thread per query;
//   - k_hfit_backward: tiles of 128 samples, one thread per sample for the
//     forward and the backward of its activations (kept in shared memory),
//     then the whole CTA forms the tile's weight gradients as sums over the
//     samples (each thread owning a fixed set of entries, accumulated over the
//     tiles in registers and added to global memory once at the end); the
//     feature-map gradients are scattered with atomics.
// MODE 1 draws the samples on the device (the simple fit's counter-based
// generator) and takes the MSE against keyframe targets interpolated at t.
#include <cuda_fp16.h>

#include <climits>

#include "bc4.cuh"
#include "bc7.cuh"
#include "ndgi_internal.h"
#include "sampler.cuh"

namespace ndgi {

struct HFitArgs {
  int lm_w, lm_h, uv_w, uv_h, vol_w, vol_h, vol_t, ut_w, ut_t, vt_h, vt_t, hidden, address_mode;
  const float* p[14];   // uv_ea, uv_eb, uv_wt, vol_ea, vol_eb, vol_wt, ut, vt, w1, b1, w2, b2, w3, b3
  float* g[14];         // gradients, same order
  int relaxed;
  int shared_w;            // Eq. 7's weight per texel shared by the four channels (BC7 simulation)
  float noise_alpha;       // mode 1: training-time quantisation noise on the 12 sampled map inputs
  int64_t n;
  const float* uvt;        // mode 0: queries [n][3]
  const float* grad_rgb;   // mode 0: dL/drgb [n][3]
  const __half* targets;   // mode 1: keyframe targets [t_count][lm_h][lm_w][3]
  int t_count;
  const float* key_t;      // keyframe times of the targets or null (j / t_count)
  uint64_t seed;
  const int64_t* step;
  double* loss_acc;
  int64_t ms[14];          // batched fit: elements of each tensor per model (model m at m * ms[k])
  int64_t tgt_stride;      // batched fit: target elements per model
};

// Batched fit: CTA row m trains model m of the stacked tensors, with samples
// (and noise) drawn from seed + m.
__device__ __forceinline__ void hfit_select_model(HFitArgs& a) {
  const int64_t m = blockIdx.y;
  if (m == 0) return;
#pragma unroll
  for (int k = 0; k < 14; ++k) {
    a.p[k] += m * a.ms[k];
    a.g[k] += m * a.ms[k];
  }
  a.targets += m * a.tgt_stride;
  a.seed += (uint64_t)m;
}
enum { kUvEa, kUvEb, kUvWt, kVolEa, kVolEb, kVolWt, kUt, kVt, kW1, kB1, kW2, kB2, kW3, kB3 };

// Straight-through value of texel p of BC entry e (block * 4 + channel) and its factors.
// Index of texel p's weight for BC entry e: per channel, or per block with shared weights.
__device__ __forceinline__ int64_t hfit_widx(int shared, int64_t e, int p) { return (shared ? e >> 2 : e) * 16 + p; }

__device__ __forceinline__ float hfit_sim(const float* ea, const float* eb, const float* wt, int64_t e, int p,
                                          int relaxed, int shared, float& dea, float& deb, float& dw) {
  const float a = __ldg(ea + e), b = __ldg(eb + e), w = __ldg(wt + hfit_widx(shared, e, p));
  if (relaxed) {
    dea = 1.0f - w;
    deb = w;
    dw = b - a;
    return (1.0f - w) * a + w * b;
  }
  if (shared) {   // BC7 mode 6: mode-6 endpoints and the 4-bit weight of index q15(w)
    const int64_t b4 = e & ~(int64_t)3;
    int qa[4], qb[4], EA[4], EB[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      qa[c] = quant(__ldg(ea + b4 + c), 255.0f);
      qb[c] = quant(__ldg(eb + b4 + c), 255.0f);
    }
    bc7_mode6_endpoint(qa, EA);
    bc7_mode6_endpoint(qb, EB);
    const int ch = (int)(e - b4);
    int A = EA[0], B = EB[0];
#pragma unroll
    for (int c = 1; c < 4; ++c)
      if (ch == c) {
        A = EA[c];
        B = EB[c];
      }
    const int W = bc7_weight(quant(w, 15.0f), 4);
    dea = 1.0f - (float)W / 64.0f;
    deb = (float)W / 64.0f;
    dw = (float)B / 255.0f - (float)A / 255.0f;
    return (float)(((64 - W) * A + W * B + 32) >> 6) * (1.0f / 255.0f);
  }
  const int A = quant(a, 255.0f), B = quant(b, 255.0f), k = quant(w, 7.0f);
  dea = 1.0f - (float)k / 7.0f;
  deb = (float)k / 7.0f;
  dw = (float)B / 255.0f - (float)A / 255.0f;
  return p35_value(5 * ((7 - k) * A + k * B));
}

// Visits the taps of one query: f(k, map, entry, texel, weight) for each
// feature input k < 12 (map 0 F3D, 1 F_uv: entry = block * 4 + channel; 2 F_ut,
// 3 F_vt: entry = value index), in a fixed order.
template <typename F>
__device__ __forceinline__ void hfit_for_each_tap(const HFitArgs& a, float u, float v, float t, F&& f) {
  const int mode = a.address_mode;
  int x0, x1, y0, y1, z0, z1;
  float fx, fy, fz;
  axis_setup(u, a.vol_w, mode, x0, x1, fx);
  axis_setup(v, a.vol_h, mode, y0, y1, fy);
  axis_setup(t, a.vol_t, 0, z0, z1, fz);
  {
    const int tx[4] = {x0, x1, x0, x1}, ty[4] = {y0, y0, y1, y1};
    const float wb[4] = {(1 - fx) * (1 - fy), fx * (1 - fy), (1 - fx) * fy, fx * fy};
    const int64_t bws = a.vol_w / 4, nbs = (int64_t)(a.vol_h / 4) * bws;
    for (int zz = 0; zz < 2; ++zz)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t blk = (zz ? z1 : z0) * nbs + (int64_t)(ty[q] >> 2) * bws + (tx[q] >> 2);
        const int p = ((ty[q] & 3) << 2) | (tx[q] & 3);
        const float w = (zz ? fz : 1.0f - fz) * wb[q];
#pragma unroll
        for (int c = 0; c < 4; ++c) f(c, 0, blk * 4 + c, p, w);
      }
  }
  axis_setup(u, a.uv_w, mode, x0, x1, fx);
  axis_setup(v, a.uv_h, mode, y0, y1, fy);
  {
    const int ux[4] = {x0, x1, x0, x1}, uy[4] = {y0, y0, y1, y1};
    const float wu[4] = {(1 - fx) * (1 - fy), fx * (1 - fy), (1 - fx) * fy, fx * fy};
    const int64_t bwu = a.uv_w / 4;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t blk = (int64_t)(uy[q] >> 2) * bwu + (ux[q] >> 2);
      const int p = ((uy[q] & 3) << 2) | (ux[q] & 3);
#pragma unroll
      for (int c = 0; c < 4; ++c) f(4 + c, 1, blk * 4 + c, p, wu[q]);
    }
  }
#pragma unroll
  for (int pl = 0; pl < 2; ++pl) {
    const int nx = pl ? a.vt_h : a.ut_w, nt = pl ? a.vt_t : a.ut_t;
    axis_setup(pl ? v : u, nx, mode, x0, x1, fx);
    axis_setup(t, nt, 0, y0, y1, fy);
    const int px[4] = {x0, x1, x0, x1}, py[4] = {y0, y0, y1, y1};
    const float wp[4] = {(1 - fx) * (1 - fy), fx * (1 - fy), (1 - fx) * fy, fx * fy};
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int c = 0; c < 2; ++c) f(8 + 2 * pl + c, 2 + pl, ((int64_t)py[q] * nx + px[q]) * 2 + c, 0, wp[q]);
  }
}

__device__ __forceinline__ float hfit_value(const HFitArgs& a, int map, int64_t e, int p, float& d0, float& d1,
                                            float& d2) {
  if (map == 0) return hfit_sim(a.p[kVolEa], a.p[kVolEb], a.p[kVolWt], e, p, a.relaxed, a.shared_w, d0, d1, d2);
  if (map == 1) return hfit_sim(a.p[kUvEa], a.p[kUvEb], a.p[kUvWt], e, p, a.relaxed, a.shared_w, d0, d1, d2);
  d0 = 1.0f;
  d1 = d2 = 0.0f;
  return __ldg(a.p[map == 2 ? kUt : kVt] + e);
}

// The decoder input x[16] of a query; with q >= 0 only the inputs k with
// k % 4 == q (the others are left 0).
__device__ __forceinline__ void hfit_inputs(const HFitArgs& a, float u, float v, float t, float (&x)[16], int q = -1) {
#pragma unroll
  for (int k = 0; k < 12; ++k) x[k] = 0.0f;
  hfit_for_each_tap(a, u, v, t, [&](int k, int map, int64_t e, int p, float w) {
    if (q >= 0 && (k & 3) != q) return;
    float d0, d1, d2;
    x[k] = fmaf(w, hfit_value(a, map, e, p, d0, d1, d2), x[k]);
  });
  sincospif(t, &x[12], &x[13]);
  sincospif(2.0f * t, &x[14], &x[15]);
}

// Scatters dL/dx[k] (k < 12) to the feature-map parameters of the query's taps
// (with q >= 0 only the inputs k with k % 4 == q).
__device__ __forceinline__ void hfit_scatter(const HFitArgs& a, float u, float v, float t, const float (&gx)[16],
                                             int q = -1) {
  hfit_for_each_tap(a, u, v, t, [&](int k, int map, int64_t e, int p, float w) {
    if (q >= 0 && (k & 3) != q) return;
    float d0, d1, d2;
    hfit_value(a, map, e, p, d0, d1, d2);
    const float g = w * gx[k];
    if (g == 0.0f) return;
    if (map == 0) {
      atomicAdd(a.g[kVolEa] + e, d0 * g);
      atomicAdd(a.g[kVolEb] + e, d1 * g);
      atomicAdd(a.g[kVolWt] + hfit_widx(a.shared_w, e, p), d2 * g);
    } else if (map == 1) {
      atomicAdd(a.g[kUvEa] + e, d0 * g);
      atomicAdd(a.g[kUvEb] + e, d1 * g);
      atomicAdd(a.g[kUvWt] + hfit_widx(a.shared_w, e, p), d2 * g);
    } else {
      atomicAdd(a.g[map == 2 ? kUt : kVt] + e, g);
    }
  });
}

__device__ __forceinline__ float gelu32(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
// d GELU / dz = Phi(z) + z phi(z)
__device__ __forceinline__ float gelu32_grad(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.3989422804014327f * __expf(-0.5f * z * z);
}

// ---------------------------------------------------------------------------
// Forward: one thread per query (MLP weights read through the read-only path).
// ---------------------------------------------------------------------------
template <int H>
__global__ void __launch_bounds__(128) k_hfit_forward(HFitArgs a, float* __restrict__ rgb) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < a.n; s += (int64_t)gridDim.x * blockDim.x) {
    const float u = a.uvt[3 * s], v = a.uvt[3 * s + 1], t = a.uvt[3 * s + 2];
    float x[16];
    hfit_inputs(a, u, v, t, x);
    float h1[H], y[3];
#pragma unroll 4
    for (int o = 0; o < H; ++o) {
      float z = __ldg(a.p[kB1] + o);
#pragma unroll
      for (int k = 0; k < 16; ++k) z = fmaf(x[k], __ldg(a.p[kW1] + k * H + o), z);
      h1[o] = gelu32(z);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) y[c] = __ldg(a.p[kB3] + c);
    for (int o = 0; o < H; ++o) {
      float z = __ldg(a.p[kB2] + o);
#pragma unroll
      for (int i = 0; i < H; ++i) z = fmaf(h1[i], __ldg(a.p[kW2] + i * H + o), z);
      const float h2 = gelu32(z);
#pragma unroll
      for (int c = 0; c < 3; ++c) y[c] = fmaf(h2, __ldg(a.p[kW3] + o * 3 + c), y[c]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) rgb[3 * s + c] = y[c];
  }
}

// ---------------------------------------------------------------------------
// Backward: tiles of kHfTile samples, kHfQ = 4 threads per sample.  Thread
// (r, q) of sample r owns hidden units q H/4 .. (q+1) H/4 - 1 of both layers
// and the feature inputs k with k % 4 == q (their BC simulation, noise and
// gradient scatter).  A sample's four threads are adjacent lanes of one warp:
// the per-sample rows in shared memory are exchanged with __syncwarp between
// the layers.  Then the whole CTA forms the tile's weight gradients as sums
// over the samples, each thread owning fixed entries in registers across
// tiles, added to global memory once at the end.
// ---------------------------------------------------------------------------
constexpr int kHfTile = 128;
constexpr int kHfQ = 4;
constexpr int kHfThreads = kHfTile * kHfQ;

// Shared memory: the MLP (forward and backward), then per-sample rows padded
// to H + 4 floats (whole float4s; the 8 samples of a warp hit 8 distinct
// banks): inputs, h1, z1 -> dz1, z2 -> dz2, h2, dL/drgb.
template <int H>
struct HFitSmem {
  static constexpr int R = H + 4;
  static constexpr int HQ = H / kHfQ;
  static constexpr int HS = H + 4 * kHfQ;   // skewed weight row: each quarter's HQ columns + 4 padding floats
  __host__ __device__ static constexpr int skew(int o) { return o + 4 * (o / HQ); }
  static constexpr int kW1 = 0;                     // [16][HS]  W1, skewed columns
  static constexpr int kB1 = kW1 + 16 * HS;
  static constexpr int kW2 = kB1 + H;               // [H][HS]   W2 (row = input), skewed columns
  static constexpr int kW2t = kW2 + H * HS;         // [H][HS]   W2^T (row = output), skewed columns
  static constexpr int kB2 = kW2t + H * HS;
  static constexpr int kW3 = kB2 + H, kB3 = kW3 + 3 * H;
  static constexpr int kX = kB3 + 4;                    // [tile][17]
  static constexpr int kH1 = kX + kHfTile * 17;
  static constexpr int kZ1 = kH1 + kHfTile * R;
  static constexpr int kZ2 = kZ1 + kHfTile * R;
  static constexpr int kH2 = kZ2 + kHfTile * R;
  static constexpr int kDY = kH2 + kHfTile * R;          // [tile][4]
  static constexpr int kFloats = kDY + kHfTile * 4;
};

template <int H, int MODE>
__global__ void __launch_bounds__(kHfThreads, 1) k_hfit_backward(HFitArgs a_in) {
  using S = HFitSmem<H>;
  HFitArgs a = a_in;
  if (MODE == 1) hfit_select_model(a);
  constexpr int R = S::R, HQ = H / kHfQ;
  constexpr bool kBlocked = H == 64;   // dW2 as 2 x 4 register blocks per thread (512 threads x 8 = 64 x 64)
  static_assert(!kBlocked || (S::kZ2 % 4 == 0 && S::R % 4 == 0), "float4-aligned dZ2 rows");
  constexpr int E2 = (H * H + kHfThreads - 1) / kHfThreads, E1 = (16 * H + kHfThreads - 1) / kHfThreads;
  constexpr int E3 = (3 * H + 3 + kHfThreads - 1) / kHfThreads;   // dW3 entries, then db3
  extern __shared__ float sm[];
  const int tid = threadIdx.x;
  constexpr int HS = S::HS;
  for (int i = tid; i < 16 * H; i += kHfThreads) sm[S::kW1 + (i / H) * HS + S::skew(i % H)] = a.p[kW1][i];
  for (int i = tid; i < H * H; i += kHfThreads) {
    const int ri = i / H, co = i % H;   // W2[ri][co]: input ri, output co
    const float w = a.p[kW2][i];
    sm[S::kW2 + ri * HS + S::skew(co)] = w;
    sm[S::kW2t + co * HS + S::skew(ri)] = w;
  }
  for (int i = tid; i < 3 * H; i += kHfThreads) sm[S::kW3 + i] = a.p[kW3][i];
  for (int i = tid; i < H; i += kHfThreads) {
    sm[S::kB1 + i] = a.p[kB1][i];
    sm[S::kB2 + i] = a.p[kB2][i];
  }
  if (tid < 3) sm[S::kB3 + tid] = a.p[kB3][tid];
  __syncthreads();
  const float* sW1 = sm + S::kW1;
  const float* sW2 = sm + S::kW2;
  const float* sW2t = sm + S::kW2t;
  const float* sW3 = sm + S::kW3;
  const int r = tid / kHfQ, q = tid % kHfQ, o0 = q * HQ, c0 = S::skew(o0);
  static_assert(HQ % 4 == 0, "float4 blocks of a quarter's units");
  float* xr = sm + S::kX + r * 17;
  float* h1 = sm + S::kH1 + r * R;
  float* z1 = sm + S::kZ1 + r * R;
  float* z2 = sm + S::kZ2 + r * R;
  float* h2 = sm + S::kH2 + r * R;
  float* dyr = sm + S::kDY + r * 4;
  float acc2[E2], acc1[E1], acc3[E3], accb1 = 0.0f, accb2 = 0.0f;
#pragma unroll
  for (int j = 0; j < E3; ++j) acc3[j] = 0.0f;
#pragma unroll
  for (int j = 0; j < E2; ++j) acc2[j] = 0.0f;
#pragma unroll
  for (int j = 0; j < E1; ++j) acc1[j] = 0.0f;
  double loss = 0.0;
  int64_t step = 0;
  if (MODE == 1) step = *a.step;
  const int64_t tiles = (a.n + kHfTile - 1) / kHfTile;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t s = tile * kHfTile + r;
    const bool valid = s < a.n;   // uniform over the sample's four threads
    float u = 0.5f, v = 0.5f, t = 0.0f;
    int ix = 0, iy = 0;
    if (valid) {
      if (MODE == 0) {
        u = a.uvt[3 * s];
        v = a.uvt[3 * s + 1];
        t = a.uvt[3 * s + 2];
      } else {
        draw_sample(a.seed, step, s, a.lm_w, a.lm_h, ix, iy, t);
        u = ((float)ix + 0.5f) / (float)a.lm_w;
        v = ((float)iy + 0.5f) / (float)a.lm_h;
      }
    }
    // ---- this thread's inputs k = q, q + 4, q + 8 (and gamma component 12 + q) ----
    {
      float x[16];
      hfit_inputs(a, u, v, t, x, q);
      if (MODE == 1 && valid && a.noise_alpha > 0.0f) {   // V' = V + U(-1/2, 1/2) alpha
        const uint64_t g = 0x9E3779B97F4A7C15ull;
        const uint64_t b = (a.seed ^ 0x6E6F697365ull) + 12ull * (((uint64_t)step << 32) + (uint64_t)s) * g;
#pragma unroll
        for (int k = 0; k < 12; ++k)
          if ((k & 3) == q) {
            const uint64_t z = splitmix64(b + (uint64_t)k * g);
            x[k] += a.noise_alpha * ((float)(uint32_t)(z >> 40) * 0x1p-24f - 0.5f);
          }
      }
#pragma unroll
      for (int k = 0; k < 16; ++k)
        if ((k & 3) == q) xr[k] = x[k];
    }
    __syncwarp();
    // ---- layer 1 and layer 2 for this thread's units; the output's partial sums ----
    {
      float acc[HQ];
#pragma unroll
      for (int u1 = 0; u1 < HQ; ++u1) acc[u1] = sm[S::kB1 + o0 + u1];
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const float xv = xr[k];
#pragma unroll
        for (int u4 = 0; u4 < HQ / 4; ++u4) {
          const float4 w = *reinterpret_cast<const float4*>(sW1 + k * HS + c0 + 4 * u4);
          acc[4 * u4] = fmaf(xv, w.x, acc[4 * u4]);
          acc[4 * u4 + 1] = fmaf(xv, w.y, acc[4 * u4 + 1]);
          acc[4 * u4 + 2] = fmaf(xv, w.z, acc[4 * u4 + 2]);
          acc[4 * u4 + 3] = fmaf(xv, w.w, acc[4 * u4 + 3]);
        }
      }
#pragma unroll
      for (int u1 = 0; u1 < HQ; ++u1) {
        z1[o0 + u1] = acc[u1];
        h1[o0 + u1] = gelu32(acc[u1]);
      }
    }
    __syncwarp();
    float y[3] = {0.0f, 0.0f, 0.0f};
    {
      float acc[HQ];
#pragma unroll
      for (int u1 = 0; u1 < HQ; ++u1) acc[u1] = sm[S::kB2 + o0 + u1];
#pragma unroll 4
      for (int i = 0; i < H; ++i) {
        const float hv = h1[i];
#pragma unroll
        for (int u4 = 0; u4 < HQ / 4; ++u4) {
          const float4 w = *reinterpret_cast<const float4*>(sW2 + i * HS + c0 + 4 * u4);
          acc[4 * u4] = fmaf(hv, w.x, acc[4 * u4]);
          acc[4 * u4 + 1] = fmaf(hv, w.y, acc[4 * u4 + 1]);
          acc[4 * u4 + 2] = fmaf(hv, w.z, acc[4 * u4 + 2]);
          acc[4 * u4 + 3] = fmaf(hv, w.w, acc[4 * u4 + 3]);
        }
      }
#pragma unroll
      for (int u1 = 0; u1 < HQ; ++u1) {
        const int o = o0 + u1;
        z2[o] = acc[u1];
        const float hh = gelu32(acc[u1]);
        h2[o] = hh;
#pragma unroll
        for (int c = 0; c < 3; ++c) y[c] = fmaf(hh, sW3[o * 3 + c], y[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {   // the four quarters' partial outputs
      y[c] += __shfl_xor_sync(0xffffffffu, y[c], 1);
      y[c] += __shfl_xor_sync(0xffffffffu, y[c], 2);
      y[c] += sm[S::kB3 + c];
    }
    float dy[3] = {0.0f, 0.0f, 0.0f};
    if (valid) {
      if (MODE == 0) {
#pragma unroll
        for (int c = 0; c < 3; ++c) dy[c] = a.grad_rgb[3 * s + c];
      } else {
        int j0, j1;
        float al;
        temporal_setup_k(t, a.t_count, a.key_t, j0, j1, al);
        const int64_t plane = (int64_t)a.lm_h * a.lm_w * 3, px = ((int64_t)iy * a.lm_w + ix) * 3;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float tg = (1.0f - al) * __half2float(a.targets[j0 * plane + px + c]) +
                           al * __half2float(a.targets[j1 * plane + px + c]);
          const float d = y[c] - tg;
          if (q == 0) loss += (double)d * d;
          dy[c] = 2.0f * d / (3.0f * (float)a.n);
        }
      }
    }
    if (q == 0) {
#pragma unroll
      for (int c = 0; c < 3; ++c) dyr[c] = dy[c];
    }
    // ---- backward of the activations: dz2 and dz1 for this thread's units ----
    for (int u1 = 0; u1 < HQ; ++u1) {
      const int o = o0 + u1;
      const float dh = sW3[o * 3] * dy[0] + sW3[o * 3 + 1] * dy[1] + sW3[o * 3 + 2] * dy[2];
      z2[o] = dh * gelu32_grad(z2[o]);   // z2 -> dz2
    }
    __syncwarp();
    {
      float acc[HQ];   // dh1 for this thread's units i: sum over o of W2[i][o] dz2[o]
#pragma unroll
      for (int u1 = 0; u1 < HQ; ++u1) acc[u1] = 0.0f;
#pragma unroll 4
      for (int o = 0; o < H; ++o) {
        const float gz = z2[o];
#pragma unroll
        for (int u4 = 0; u4 < HQ / 4; ++u4) {
          const float4 w = *reinterpret_cast<const float4*>(sW2t + o * HS + c0 + 4 * u4);
          acc[4 * u4] = fmaf(gz, w.x, acc[4 * u4]);
          acc[4 * u4 + 1] = fmaf(gz, w.y, acc[4 * u4 + 1]);
          acc[4 * u4 + 2] = fmaf(gz, w.z, acc[4 * u4 + 2]);
          acc[4 * u4 + 3] = fmaf(gz, w.w, acc[4 * u4 + 3]);
        }
      }
#pragma unroll
      for (int u1 = 0; u1 < HQ; ++u1) z1[o0 + u1] = acc[u1] * gelu32_grad(z1[o0 + u1]);   // z1 -> dz1
    }
    __syncwarp();
    {
      float gx[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        float g = 0.0f;
        if ((k & 3) == q && k < 12)
          for (int o = 0; o < H; ++o) g = fmaf(sW1[k * HS + S::skew(o)], z1[o], g);
        gx[k] = g;
      }
      if (valid) hfit_scatter(a, u, v, t, gx, q);
    }
    __syncthreads();
    // ---- the tile's weight gradients: sums over its samples ----
    if constexpr (kBlocked) {   // thread (ib, ob): dW2[2 ib .. 2 ib + 1][4 ob .. 4 ob + 3]
      const int i0 = 2 * (tid >> 4), ob = 4 * (tid & 15);
      float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll 4
      for (int rr = 0; rr < kHfTile; ++rr) {
        const float ha = sm[S::kH1 + rr * R + i0], hb = sm[S::kH1 + rr * R + i0 + 1];
        const float4 z = *reinterpret_cast<const float4*>(sm + S::kZ2 + rr * R + ob);
        acc[0] = fmaf(ha, z.x, acc[0]);
        acc[1] = fmaf(ha, z.y, acc[1]);
        acc[2] = fmaf(ha, z.z, acc[2]);
        acc[3] = fmaf(ha, z.w, acc[3]);
        acc[4] = fmaf(hb, z.x, acc[4]);
        acc[5] = fmaf(hb, z.y, acc[5]);
        acc[6] = fmaf(hb, z.z, acc[6]);
        acc[7] = fmaf(hb, z.w, acc[7]);
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) acc2[j] += acc[j];
    } else {
#pragma unroll
      for (int j = 0; j < E2; ++j) {
        const int e = tid + kHfThreads * j;
        if (e < H * H) {
          const int i = e / H, o = e % H;
          float acc = 0.0f;
          for (int rr = 0; rr < kHfTile; ++rr) acc = fmaf(sm[S::kH1 + rr * R + i], sm[S::kZ2 + rr * R + o], acc);
          acc2[j] += acc;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < E1; ++j) {
      const int e = tid + kHfThreads * j;
      if (e < 16 * H) {
        const int k = e / H, o = e % H;
        float acc = 0.0f;
        for (int rr = 0; rr < kHfTile; ++rr) acc = fmaf(sm[S::kX + rr * 17 + k], sm[S::kZ1 + rr * R + o], acc);
        acc1[j] += acc;
      }
    }
    if (tid < H) {
      float b1 = 0.0f, b2 = 0.0f;
      for (int rr = 0; rr < kHfTile; ++rr) {
        b1 += sm[S::kZ1 + rr * R + tid];
        b2 += sm[S::kZ2 + rr * R + tid];
      }
      accb1 += b1;
      accb2 += b2;
    }
#pragma unroll
    for (int j = 0; j < E3; ++j) {
      const int e = tid + kHfThreads * j;
      float g = 0.0f;
      if (e < 3 * H) {
        const int o = e / 3, c = e % 3;
        for (int rr = 0; rr < kHfTile; ++rr) g = fmaf(sm[S::kH2 + rr * R + o], sm[S::kDY + rr * 4 + c], g);
      } else if (e < 3 * H + 3) {
        for (int rr = 0; rr < kHfTile; ++rr) g += sm[S::kDY + rr * 4 + (e - 3 * H)];
      }
      acc3[j] += g;
    }
    __syncthreads();   // the rows are rewritten by the next tile
  }
  if constexpr (kBlocked) {
    const int i0 = 2 * (tid >> 4), ob = 4 * (tid & 15);
#pragma unroll
    for (int j = 0; j < 8; ++j) atomicAdd(a.g[kW2] + (i0 + j / 4) * H + ob + (j % 4), acc2[j]);
  } else {
#pragma unroll
    for (int j = 0; j < E2; ++j) {
      const int e = tid + kHfThreads * j;
      if (e < H * H) atomicAdd(a.g[kW2] + e, acc2[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < E1; ++j) {
    const int e = tid + kHfThreads * j;
    if (e < 16 * H) atomicAdd(a.g[kW1] + e, acc1[j]);
  }
  if (tid < H) {
    atomicAdd(a.g[kB1] + tid, accb1);
    atomicAdd(a.g[kB2] + tid, accb2);
  }
#pragma unroll
  for (int j = 0; j < E3; ++j) {
    const int e = tid + kHfThreads * j;
    if (e < 3 * H) atomicAdd(a.g[kW3] + e, acc3[j]);
    else if (e < 3 * H + 3) atomicAdd(a.g[kB3] + (e - 3 * H), acc3[j]);
  }
  if (MODE == 1) {
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
    if ((tid & 31) == 0) atomicAdd(a.loss_acc, loss);
  }
}

// ---------------------------------------------------------------------------
// Adam over the fourteen tensors (Kingma & Ba; bias-corrected).  The feature
// maps (the BC endpoints and weights of F_uv and F3D, and F_ut / F_vt, tensors
// 0..7) are projected onto [0, 1] and frozen for the last steps of a run (the
// paper's final stage fine-tunes the MLP alone).
// ---------------------------------------------------------------------------
struct HAdam {
  float* p[14];
  int64_t off[15];
  const float* g;
  float *m, *v;
  const int64_t* step;    // global steps taken
  const int64_t* local;   // steps taken in this call
  int64_t freeze_from;
  float lr, beta1, beta2, eps;
};

__global__ void k_hfit_adam(HAdam t) {
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
  const int64_t n = t.off[14];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int k = 0;
#pragma unroll
    for (int q = 1; q < 14; ++q) k += (i >= t.off[q]);
    if (freeze && k < 8) continue;
    const float g = t.g[i];
    const float m = t.beta1 * t.m[i] + (1.0f - t.beta1) * g;
    const float v = t.beta2 * t.v[i] + (1.0f - t.beta2) * g * g;
    t.m[i] = m;
    t.v[i] = v;
    float* pp = t.p[k] + (i - t.off[k]);
    float q = *pp - t.lr * (m / c1) / (sqrtf(v / c2) + t.eps);
    if (k < 8) q = fminf(fmaxf(q, 0.0f), 1.0f);
    *pp = q;
  }
}

__global__ void k_hfit_step_end(int64_t* step, int64_t* local, const double* loss_acc, double* loss_log, int every,
                                int64_t batch) {
  const int64_t l = *local;   // batch: samples of the step over all models
  if (loss_log && every > 0 && l % every == 0) loss_log[l / every] = *loss_acc / (3.0 * (double)batch);
  *local = l + 1;
  *step = *step + 1;
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
#define NDGI_HFIT_HIDDEN(X) X(16) X(32) X(64)

static bool hfit_hidden_ok(int h) {
#define X(H) if (h == H) return true;
  NDGI_HFIT_HIDDEN(X)
#undef X
  return false;
}

static cudaError_t launch_hfit_forward(const HFitArgs& a, float* rgb, cudaStream_t s) {
  const int grid = (int)std::min<int64_t>((a.n + 127) / 128, (int64_t)num_sms() * 16);
#define X(H)                                                        \
  if (a.hidden == H) {                                              \
    k_hfit_forward<H><<<grid > 0 ? grid : 1, 128, 0, s>>>(a, rgb);  \
    return cudaGetLastError();                                      \
  }
  NDGI_HFIT_HIDDEN(X)
#undef X
  return cudaErrorInvalidValue;
}

static cudaError_t launch_hfit_backward(const HFitArgs& a, int mode, cudaStream_t s, int n_models = 1) {
  const int64_t tiles = (a.n + kHfTile - 1) / kHfTile, sms = num_sms();
  // CTAs per model (one CTA per SM): the count with the fewest waves x tiles per CTA
  int64_t per_model = 1, best = INT64_MAX;
  for (int64_t c = 1; c <= std::min<int64_t>(tiles, std::max<int64_t>(1, 2 * sms / n_models + 1)); ++c) {
    const int64_t cost = ((c * n_models + sms - 1) / sms) * ((tiles + c - 1) / c);
    if (cost < best) {
      best = cost;
      per_model = c;
    }
  }
  const dim3 grid((unsigned)per_model, (unsigned)n_models);
#define X(H)                                                                                          \
  if (a.hidden == H) {                                                                                \
    const size_t smem = sizeof(float) * HFitSmem<H>::kFloats;                                         \
    auto kern = mode == 0 ? k_hfit_backward<H, 0> : k_hfit_backward<H, 1>;                             \
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    if (e != cudaSuccess) return e;                                                                   \
    kern<<<grid, kHfThreads, smem, s>>>(a);                                                              \
    return cudaGetLastError();                                                                        \
  }
  NDGI_HFIT_HIDDEN(X)
#undef X
  return cudaErrorInvalidValue;
}

// Element counts of the fourteen tensors.
static void hfit_sizes(const ndgi_hybrid_fit_params* p, int64_t (&n)[14]) {
  const int64_t ub = (int64_t)(p->uv_h / 4) * (p->uv_w / 4) * 4, vb = (int64_t)p->vol_t * (p->vol_h / 4) * (p->vol_w / 4) * 4;
  const int64_t H = p->hidden;
  const int64_t wpb = p->shared_w ? 4 : 16;   // weights per BC entry (block x channel)
  n[kUvEa] = ub; n[kUvEb] = ub; n[kUvWt] = ub * wpb;
  n[kVolEa] = vb; n[kVolEb] = vb; n[kVolWt] = vb * wpb;
  n[kUt] = (int64_t)p->ut_t * p->ut_w * 2; n[kVt] = (int64_t)p->vt_t * p->vt_h * 2;
  n[kW1] = 16 * H; n[kB1] = H; n[kW2] = H * H; n[kB2] = H; n[kW3] = 3 * H; n[kB3] = 3;
}

static ndgi_status check_hfit(const ndgi_hybrid_fit_params* p, const char* who) {
  if (!p) return set_error(NDGI_ERR_INVALID_ARG, "%s: params is NULL", who);
  if (p->lm_w <= 0 || p->lm_h <= 0 || p->uv_w <= 0 || p->uv_h <= 0 || p->uv_w % 4 || p->uv_h % 4 ||
      p->vol_w <= 0 || p->vol_h <= 0 || p->vol_w % 4 || p->vol_h % 4 || p->vol_t <= 0 || p->ut_w <= 0 ||
      p->ut_t <= 0 || p->vt_h <= 0 || p->vt_t <= 0)
    return set_error(NDGI_ERR_INVALID_ARG, "%s: bad sizes", who);
  if (!hfit_hidden_ok(p->hidden))
    return set_error(NDGI_ERR_UNSUPPORTED, "%s: hidden width %d not built (16, 32, 64)", who, p->hidden);
  if (p->address_mode != 0 && p->address_mode != 1)
    return set_error(NDGI_ERR_INVALID_ARG, "%s: address_mode must be 0 or 1", who);
  float* const q[14] = {p->uv_ea, p->uv_eb, p->uv_wt, p->vol_ea, p->vol_eb, p->vol_wt, p->ut,
                        p->vt,    p->w1,    p->b1,    p->w2,     p->b2,     p->w3,     p->b3};
  for (int k = 0; k < 14; ++k)
    if (!q[k]) return set_error(NDGI_ERR_INVALID_ARG, "%s: a parameter pointer is NULL", who);
  return NDGI_OK;
}

static HFitArgs make_hfit_args(const ndgi_hybrid_fit_params* p) {
  HFitArgs a{};
  a.lm_w = p->lm_w; a.lm_h = p->lm_h; a.uv_w = p->uv_w; a.uv_h = p->uv_h; a.vol_w = p->vol_w; a.vol_h = p->vol_h;
  a.vol_t = p->vol_t; a.ut_w = p->ut_w; a.ut_t = p->ut_t; a.vt_h = p->vt_h; a.vt_t = p->vt_t; a.hidden = p->hidden;
  a.address_mode = p->address_mode;
  a.shared_w = p->shared_w != 0;
  float* const q[14] = {p->uv_ea, p->uv_eb, p->uv_wt, p->vol_ea, p->vol_eb, p->vol_wt, p->ut,
                        p->vt,    p->w1,    p->b1,    p->w2,     p->b2,     p->w3,     p->b3};
  for (int k = 0; k < 14; ++k) a.p[k] = q[k];
  return a;
}

static size_t round256h(size_t b) { return (b + 255) / 256 * 256; }

static size_t hfit_ws_bytes(const ndgi_hybrid_fit_params* params, int32_t n_models) {
  if (!params || n_models < 1) return 0;
  int64_t n[14];
  hfit_sizes(params, n);
  int64_t tot = 0;
  for (int k = 0; k < 14; ++k) tot += n[k];
  return 256 + 3 * round256h((size_t)tot * n_models * sizeof(float));
}

static ndgi_status hybrid_encode_fit(const ndgi_hybrid_fit_params* params, int32_t n_models, const uint16_t* targets,
                                     int32_t t_count, const float* key_t, const ndgi_fit_config* cfg,
                                     int32_t step_offset, void* ws, size_t ws_bytes, double* loss_log, void* stream,
                                     const char* who) {
  ndgi_status st = check_hfit(params, who);
  if (st != NDGI_OK) return st;
  if (n_models < 1 || n_models > 65535)   // one CTA row (grid y) per model
    return set_error(NDGI_ERR_INVALID_ARG, "%s: n_models must be in 1..65535", who);
  if (!cfg || !targets || !ws || t_count <= 0) return set_error(NDGI_ERR_INVALID_ARG, "%s: bad argument", who);
  if ((uintptr_t)targets % 2 || (uintptr_t)loss_log % 8)
    return set_error(NDGI_ERR_INVALID_ARG, "%s: targets must be 2-byte and loss_log 8-byte aligned", who);
  if (cfg->steps < 0 || cfg->batch <= 0 || cfg->freeze_steps < 0 || cfg->loss_every < 0 || step_offset < 0)
    return set_error(NDGI_ERR_INVALID_ARG, "%s: bad config", who);
  if (!(cfg->lr > 0.0f) || !(cfg->beta1 >= 0.0f && cfg->beta1 < 1.0f) || !(cfg->beta2 >= 0.0f && cfg->beta2 < 1.0f))
    return set_error(NDGI_ERR_INVALID_ARG, "%s: bad optimiser settings", who);
  if (!(cfg->noise_alpha >= 0.0f && cfg->noise_alpha <= 1.0f))
    return set_error(NDGI_ERR_INVALID_ARG, "%s: noise_alpha must be in [0, 1]", who);
  const size_t need = hfit_ws_bytes(params, n_models);
  if (ws_bytes < need || ((uintptr_t)ws % 256))
    return set_error(NDGI_ERR_INVALID_ARG, "%s: ws must be 256-byte aligned with >= %zu bytes", who, need);
  if (cfg->steps == 0) return NDGI_OK;
  cudaStream_t s = (cudaStream_t)stream;
  int64_t n[14];
  hfit_sizes(params, n);
  HFitArgs a = make_hfit_args(params);
  HAdam t{};
  int64_t tot = 0;
  for (int k = 0; k < 14; ++k) {
    a.ms[k] = n[k];
    t.p[k] = const_cast<float*>(a.p[k]);
    t.off[k] = tot;
    tot += n[k] * n_models;   // each tensor holds the n_models models one after another
  }
  a.tgt_stride = (int64_t)t_count * params->lm_h * params->lm_w * 3;
  t.off[14] = tot;
  unsigned char* base = static_cast<unsigned char*>(ws);
  int64_t* d_step = reinterpret_cast<int64_t*>(base);
  int64_t* d_local = d_step + 1;
  double* d_loss = reinterpret_cast<double*>(base + 16);
  const size_t tb = round256h((size_t)tot * sizeof(float));
  float* g = reinterpret_cast<float*>(base + 256);
  float* m = reinterpret_cast<float*>(base + 256 + tb);
  float* v = reinterpret_cast<float*>(base + 256 + 2 * tb);
  const int64_t init[2] = {step_offset, 0};
  cudaError_t e = cudaMemcpyAsync(d_step, init, sizeof(init), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // `init` lives on this stack frame
  if (e == cudaSuccess && step_offset == 0) e = cudaMemsetAsync(m, 0, 2 * tb, s);
  if (e != cudaSuccess) return cuda_status(e, who);
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
  for (int k = 0; k < 14; ++k) a.g[k] = g + t.off[k];
  a.relaxed = cfg->relaxed != 0;
  a.noise_alpha = cfg->noise_alpha;
  a.n = cfg->batch;
  a.targets = reinterpret_cast<const __half*>(targets);
  a.t_count = t_count;
  a.key_t = key_t;
  a.seed = cfg->seed;
  a.step = d_step;
  a.loss_acc = d_loss;
  // one step captured as a graph (zero grads and loss, backward, Adam, counters) and replayed
  cudaStream_t cs = nullptr;
  e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_status(e, who);
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  cudaError_t le = cudaSuccess;
  if (e == cudaSuccess) {
    le = cudaMemsetAsync(g, 0, (size_t)tot * sizeof(float), cs);
    if (le == cudaSuccess) le = cudaMemsetAsync(d_loss, 0, sizeof(double), cs);
    if (le == cudaSuccess) le = launch_hfit_backward(a, 1, cs, n_models);
    if (le == cudaSuccess) {
      const int64_t blocks = std::min<int64_t>((tot + 255) / 256, (int64_t)num_sms() * 8);
      k_hfit_adam<<<(int)std::max<int64_t>(blocks, 1), 256, 0, cs>>>(t);
      le = cudaGetLastError();
    }
    if (le == cudaSuccess) {
      k_hfit_step_end<<<1, 1, 0, cs>>>(d_step, d_local, d_loss, loss_log, cfg->loss_every,
                                       (int64_t)cfg->batch * n_models);
      le = cudaGetLastError();
    }
    e = cudaStreamEndCapture(cs, &graph);
  }
  if (le != cudaSuccess) e = le;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  for (int i = 0; e == cudaSuccess && i < cfg->steps; ++i) e = cudaGraphLaunch(exec, s);
  if (exec) cudaGraphExecDestroy(exec);
  cudaStreamDestroy(cs);
  return cuda_status(e, who);
}


}  // namespace ndgi

using namespace ndgi;

extern "C" {

ndgi_status ndgi_hybrid_fit_forward(const ndgi_hybrid_fit_params* params, const float* uvt, int64_t n,
                                    int32_t relaxed, float* rgb, void* stream) {
  ndgi_status st = check_hfit(params, "ndgi_hybrid_fit_forward");
  if (st != NDGI_OK) return st;
  if (n < 0) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_hybrid_fit_forward: n < 0");
  if (n == 0) return NDGI_OK;
  if (!uvt || !rgb) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_hybrid_fit_forward: uvt or rgb is NULL");
  HFitArgs a = make_hfit_args(params);
  a.relaxed = relaxed != 0;
  a.n = n;
  a.uvt = uvt;
  return cuda_status(launch_hfit_forward(a, rgb, (cudaStream_t)stream), "ndgi_hybrid_fit_forward");
}

ndgi_status ndgi_hybrid_fit_backward(const ndgi_hybrid_fit_params* params, const float* uvt, int64_t n,
                                     int32_t relaxed, const float* grad_rgb, const ndgi_hybrid_fit_grads* grads,
                                     void* stream) {
  ndgi_status st = check_hfit(params, "ndgi_hybrid_fit_backward");
  if (st != NDGI_OK) return st;
  if (n < 0) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_hybrid_fit_backward: n < 0");
  if (n == 0) return NDGI_OK;
  if (!uvt || !grad_rgb || !grads) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_hybrid_fit_backward: NULL argument");
  HFitArgs a = make_hfit_args(params);
  for (int k = 0; k < 14; ++k) {
    a.g[k] = grads->g[k];
    if (!a.g[k]) return set_error(NDGI_ERR_INVALID_ARG, "ndgi_hybrid_fit_backward: a gradient pointer is NULL");
  }
  a.relaxed = relaxed != 0;
  a.n = n;
  a.uvt = uvt;
  a.grad_rgb = grad_rgb;
  return cuda_status(launch_hfit_backward(a, 0, (cudaStream_t)stream), "ndgi_hybrid_fit_backward");
}

size_t ndgi_hybrid_encode_fit_workspace_size(const ndgi_hybrid_fit_params* params, const ndgi_fit_config* cfg) {
  (void)cfg;
  return hfit_ws_bytes(params, 1);
}

size_t ndgi_hybrid_encode_fit_batch_workspace_size(const ndgi_hybrid_fit_params* params, int32_t n_models,
                                                   const ndgi_fit_config* cfg) {
  (void)cfg;
  return hfit_ws_bytes(params, n_models);
}

ndgi_status ndgi_hybrid_encode_fit(const ndgi_hybrid_fit_params* params, const uint16_t* targets, int32_t t_count,
                                   const float* key_t, const ndgi_fit_config* cfg, int32_t step_offset, void* ws,
                                   size_t ws_bytes, double* loss_log, void* stream) {
  return hybrid_encode_fit(params, 1, targets, t_count, key_t, cfg, step_offset, ws, ws_bytes, loss_log, stream,
                           "ndgi_hybrid_encode_fit");
}

ndgi_status ndgi_hybrid_encode_fit_batch(const ndgi_hybrid_fit_params* params, int32_t n_models,
                                         const uint16_t* targets, int32_t t_count, const float* key_t,
                                         const ndgi_fit_config* cfg, int32_t step_offset, void* ws, size_t ws_bytes,
                                         double* loss_log, void* stream) {
  return hybrid_encode_fit(params, n_models, targets, t_count, key_t, cfg, step_offset, ws, ws_bytes, loss_log,
                           stream, "ndgi_hybrid_encode_fit_batch");
}

}  // extern "C"
