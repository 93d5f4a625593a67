// Tiled, mask-aware quality metrics of decoded lightmaps (supplement S4.2):
// each map is cut into tile x tile tiles; per tile, over the texels whose mask
// is non-zero, the reference's range L = max - min (all channels) sets the
// PSNR peak and Wang et al.'s SSIM constants C1 = (0.01 L)^2, C2 = (0.03 L)^2;
// SSIM uses an 11 x 11 Gaussian window (sigma 1.5) lying inside the tile and
// is averaged over the valid centres and the channels.  One CTA per tile: a
// first pass reduces the range and the squared error, a second the SSIM map.
// Window statistics run in FP32 on values shifted by the tile's minimum (the
// covariances are shift-invariant, so only the means are shifted back); the
// sums over the tile are FP64.
#include <cmath>

#include "ndgi_internal.h"

namespace ndgi {

constexpr int kMetR = 5;           // window radius
constexpr int kMetThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < kMetThreads / 32; ++i) s += sh[i];
  return s;
}

__device__ __forceinline__ float block_min(float v, float* sh) {
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  float s = sh[0];
  for (int i = 1; i < kMetThreads / 32; ++i) s = fminf(s, sh[i]);
  return s;
}

__global__ void __launch_bounds__(kMetThreads) k_tile_metrics(const float* __restrict__ pred,
                                                              const float* __restrict__ ref,
                                                              const uint8_t* __restrict__ mask, int h, int w, int c,
                                                              int tile, int ty_n, int tx_n, double* __restrict__ psnr,
                                                              double* __restrict__ ssim) {
  __shared__ float gw[2 * kMetR + 1];
  __shared__ double shd[kMetThreads / 32];
  __shared__ float shf[kMetThreads / 32];
  const int tid = threadIdx.x;
  const int64_t b = blockIdx.x;
  const int per_map = ty_n * tx_n;
  const int mi = (int)(b / per_map), rem = (int)(b % per_map), ty = rem / tx_n, tx = rem % tx_n;
  if (tid == 0) {
    float s = 0.0f;
    for (int i = 0; i <= 2 * kMetR; ++i) {
      const float d = (float)(i - kMetR);
      gw[i] = expf(-d * d / 4.5f);
      s += gw[i];
    }
    for (int i = 0; i <= 2 * kMetR; ++i) gw[i] /= s;
  }
  const int y0 = ty * tile, x0 = tx * tile, y1 = min(y0 + tile, h), x1 = min(x0 + tile, w);
  const int th = y1 - y0, tw = x1 - x0;
  const size_t base = (size_t)mi * h * w;
  const float* P = pred + base * c;
  const float* Q = ref + base * c;
  const uint8_t* M = mask ? mask + base : nullptr;
  // ---- pass 1: range, squared error, valid count ----
  float lo = INFINITY, nhi = INFINITY;
  double se = 0.0, cnt = 0.0;
  for (int i = tid; i < th * tw; i += kMetThreads) {
    const int y = y0 + i / tw, x = x0 + i % tw;
    if (M && !M[(size_t)y * w + x]) continue;
    cnt += 1.0;
    for (int k = 0; k < c; ++k) {
      const size_t e = ((size_t)y * w + x) * c + k;
      const float q = Q[e];
      const double d = (double)P[e] - (double)q;
      lo = fminf(lo, q);
      nhi = fminf(nhi, -q);
      se += d * d;
    }
  }
  lo = block_min(lo, shf);
  const float hi = -block_min(nhi, shf);
  se = block_sum(se, shd);
  cnt = block_sum(cnt, shd);
  const size_t o = (size_t)b;
  if (cnt == 0.0) {
    if (tid == 0) {
      psnr[o] = nan("");
      ssim[o] = nan("");
    }
    return;   // uniform over the CTA
  }
  const double L = (double)hi - (double)lo, mse = se / (cnt * c);
  if (tid == 0) psnr[o] = mse > 0.0 ? 10.0 * log10(L * L / mse) : INFINITY;
  // ---- pass 2: SSIM over valid centres whose window lies inside the tile ----
  const float C1 = (float)((0.01 * L) * (0.01 * L)), C2 = (float)((0.03 * L) * (0.03 * L));
  const int ch = th - 2 * kMetR, cw = tw - 2 * kMetR;
  double acc = 0.0, ns = 0.0;
  if (ch > 0 && cw > 0) {
    for (int i = tid; i < ch * cw; i += kMetThreads) {
      const int y = y0 + kMetR + i / cw, x = x0 + kMetR + i % cw;
      if (M && !M[(size_t)y * w + x]) continue;
      ns += 1.0;
      for (int k = 0; k < c; ++k) {
        float mx = 0.0f, my = 0.0f, sxx = 0.0f, syy = 0.0f, sxy = 0.0f;
        for (int dy = -kMetR; dy <= kMetR; ++dy) {
          const float wy = gw[dy + kMetR];
          const size_t row = ((size_t)(y + dy) * w + x) * c + k;
          for (int dx = -kMetR; dx <= kMetR; ++dx) {
            const float wt = wy * gw[dx + kMetR];
            const float a = __ldg(P + row + (int64_t)dx * c) - lo, q = __ldg(Q + row + (int64_t)dx * c) - lo;
            mx = fmaf(wt, a, mx);
            my = fmaf(wt, q, my);
            sxx = fmaf(wt * a, a, sxx);
            syy = fmaf(wt * q, q, syy);
            sxy = fmaf(wt * a, q, sxy);
          }
        }
        const float vx = sxx - mx * mx, vy = syy - my * my, cxy = sxy - mx * my;
        const float ux = mx + lo, uy = my + lo;
        acc += ((2.0f * ux * uy + C1) * (2.0f * cxy + C2)) / ((ux * ux + uy * uy + C1) * (vx + vy + C2));
      }
    }
  }
  acc = block_sum(acc, shd);
  ns = block_sum(ns, shd);
  if (tid == 0) ssim[o] = ns > 0.0 ? acc / (ns * c) : nan("");
}

}  // namespace ndgi

extern "C" ndgi_status ndgi_tile_metrics(const float* pred, const float* ref, const uint8_t* mask, int32_t n_maps,
                                         int32_t h, int32_t w, int32_t channels, int32_t tile, double* psnr,
                                         double* ssim, void* stream) {
  using ndgi::set_error;
  if (!pred || !ref || !psnr || !ssim)
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_tile_metrics: NULL argument");
  if ((uintptr_t)pred % 4 || (uintptr_t)ref % 4 || (uintptr_t)psnr % 8 || (uintptr_t)ssim % 8)
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_tile_metrics: pred/ref must be 4-byte and psnr/ssim 8-byte aligned");
  if (n_maps <= 0 || h <= 0 || w <= 0 || channels < 1 || channels > 4 || tile < 1)
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_tile_metrics: bad sizes");
  const int64_t ty_n = (h + tile - 1) / tile, tx_n = (w + tile - 1) / tile;
  if ((int64_t)n_maps * ty_n * tx_n > ((int64_t)1 << 31) - 1 || (int64_t)h * w > ((int64_t)1 << 31) - 1)
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_tile_metrics: too many tiles");
  ndgi::k_tile_metrics<<<(unsigned)(n_maps * ty_n * tx_n), ndgi::kMetThreads, 0, (cudaStream_t)stream>>>(
      pred, ref, mask, h, w, channels, tile, (int)ty_n, (int)tx_n, psnr, ssim);
  return ndgi::cuda_status(cudaGetLastError(), "ndgi_tile_metrics");
}
