// Tensor-core decode: the MLP of the decoder on tcgen05 (FP16 or BF16
// operands, FP32 accumulation in tensor memory).
//
// A CTA of 128 threads owns one 128-row MMA tile at a time: thread r gathers
// the features of query (or page texel) r in FP32 exactly as the CUDA-core
// decode does, rounds them to FP16/BF16 and writes row r of the A tile in
// shared memory.  One thread then issues the layer-1 MMAs
//   D1[128 x H] = [x, 1, 0...] [128 x K1]  *  [W1; b1; 0]^T       (bias folded into K padding)
// and commits them to an mbarrier; every thread reads its row of D1 from
// tensor memory, applies ReLU, rounds and writes row r of the next A tile;
// layer 2 (D2 = H1 W2, bias added in FP32 in the epilogue) and the output
// layer (N padded from 3 to 16) follow the same pattern.  Several CTAs are
// resident per SM, so the gathers and epilogues of one CTA overlap the MMAs
// of the others.  Every mbarrier wait is bounded; a timeout is latched in a
// device error word that ndgi_check reports, and the CTA unwinds and frees
// its tensor memory.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ndgi_internal.h"
#include "bc4.cuh"
#include "gather.cuh"
#include "tc_decode.h"
#include "umma.cuh"

namespace ndgi {

// Device error word of the tensor-core kernels (bit 0: an mbarrier wait timed out).
static __device__ int g_tc_error;

constexpr int kTcThreads = 128;
constexpr int kTcMinSmem = 48 * 1024;   // caps residency at 4 CTAs/SM, so 4 x TMEM allocation <= 512 columns

template <int CS, int CT, int H>
struct TcLayout {
  static constexpr int CIN = CS + CT;
  static constexpr int K1 = ((CIN + 1 + 15) / 16) * 16;   // inputs + ones column, padded to the MMA K step
  static constexpr int N3 = 16;                           // output layer N (3 used)
  static constexpr uint32_t kB1 = 0;                      // [H][K1]
  static constexpr uint32_t kB2 = kB1 + H * K1 * 2;       // [H][H]
  static constexpr uint32_t kB3 = kB2 + H * H * 2;        // [16][H]
  static constexpr uint32_t kBias2 = kB3 + N3 * H * 2;    // H floats
  static constexpr uint32_t kBias3 = kBias2 + H * 4;      // 4 floats
  static constexpr uint32_t kWsBytes = kBias3 + 16;
  static constexpr uint32_t kA1 = (kWsBytes + 127) / 128 * 128;
  static constexpr uint32_t kA2 = kA1 + 128 * K1 * 2;
  static constexpr uint32_t kUsed = kA2 + 128 * H * 2;
  static constexpr uint32_t kSmem = kUsed > (uint32_t)kTcMinSmem ? kUsed : (uint32_t)kTcMinSmem;
  static constexpr uint32_t kTmemCols = 2 * H <= 32 ? 32 : (2 * H <= 64 ? 64 : (2 * H <= 128 ? 128 : 256));
  static_assert(H % 16 == 0 && H <= 128, "hidden width must be a multiple of 16, at most 128");
  static_assert(kWsBytes % 16 == 0, "weight image must be 16-byte granular");
};

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

// Two floats -> packed pair (first value in the low half).
template <bool BF16>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
  return (uint32_t)to_bits<BF16>(a) | ((uint32_t)to_bits<BF16>(b) << 16);
}

// ---------------------------------------------------------------------------
// Weight image: the shared-memory operand tiles, built once per model.
// ---------------------------------------------------------------------------
template <int CS, int CT, int H, bool BF16>
__global__ void k_tc_prepare(DevModel m, unsigned char* __restrict__ ws) {
  using L = TcLayout<CS, CT, H>;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
  for (int i = tid; i < H * L::K1; i += nt) {      // B1[n][k] = W1[k][n], row CIN = b1
    const int n = i / L::K1, k = i % L::K1;
    const float v = k < L::CIN ? m.w1[k * H + n] : (k == L::CIN ? m.b1[n] : 0.0f);
    *reinterpret_cast<uint16_t*>(ws + L::kB1 + kmajor_offset(n, k, L::K1)) = to_bits<BF16>(v);
  }
  for (int i = tid; i < H * H; i += nt) {          // B2[n][k] = W2[k][n]
    const int n = i / H, k = i % H;
    *reinterpret_cast<uint16_t*>(ws + L::kB2 + kmajor_offset(n, k, H)) = to_bits<BF16>(m.w2[k * H + n]);
  }
  for (int i = tid; i < L::N3 * H; i += nt) {      // B3[n][k] = W3[k][n], rows 3..15 zero
    const int n = i / H, k = i % H;
    const float v = n < 3 ? m.w3[k * 3 + n] : 0.0f;
    *reinterpret_cast<uint16_t*>(ws + L::kB3 + kmajor_offset(n, k, H)) = to_bits<BF16>(v);
  }
  for (int i = tid; i < H; i += nt) reinterpret_cast<float*>(ws + L::kBias2)[i] = round_stored<BF16>(m.b2[i]);
  if (tid < 4) reinterpret_cast<float*>(ws + L::kBias3)[tid] = tid < 3 ? round_stored<BF16>(m.b3[tid]) : 0.0f;
}

// ---------------------------------------------------------------------------
// Shared pieces of the tile pipeline
// ---------------------------------------------------------------------------
template <int CS, int CT, int H, bool BF16>
struct TcTile {
  using L = TcLayout<CS, CT, H>;

  // Row `row` of the layer-1 A tile from the FP32 features (ones column for the bias).
  static __device__ __forceinline__ void write_a1(unsigned char* sm, int row, const float (&x)[L::CIN]) {
#pragma unroll
    for (int c = 0; c < L::K1 / 8; ++c) {
      float v[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int k = 8 * c + e;
        v[e] = k < L::CIN ? x[k < L::CIN ? k : 0] : (k == L::CIN ? 1.0f : 0.0f);
      }
      uint4 p;
      p.x = pack2<BF16>(v[0], v[1]);
      p.y = pack2<BF16>(v[2], v[3]);
      p.z = pack2<BF16>(v[4], v[5]);
      p.w = pack2<BF16>(v[6], v[7]);
      *reinterpret_cast<uint4*>(sm + L::kA1 + kmajor_offset(row, 8 * c, L::K1)) = p;
    }
  }

  // Issue one layer's MMAs (single thread) and commit to the barrier.
  static __device__ __forceinline__ void mma_layer(uint32_t d_tmem, uint32_t a_smem, uint32_t b_smem, int K, int N,
                                                   uint64_t* bar) {
    tc_fence_after();
    const uint32_t sbo = (uint32_t)K * 16u;
    const uint32_t id = idesc_f16(128, N, BF16);
    for (int ks = 0; ks < K / 16; ++ks)
      umma_f16(d_tmem, sdesc(a_smem + 256u * ks, 128u, sbo), sdesc(b_smem + 256u * ks, 128u, sbo), id, ks > 0);
    umma_commit(bar);
  }

  // Epilogue of a hidden layer: this thread's row of D (H columns) -> ReLU(D + bias) -> A2 row.
  static __device__ __forceinline__ void hidden_epilogue(unsigned char* sm, uint32_t taddr, int row,
                                                         const float* bias) {
#pragma unroll
    for (int c = 0; c < H / 16; ++c) {
      uint32_t r[16];
      tmem_ld16(taddr + 16u * c, r);
      tmem_ld_wait();
      float v[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const float b = bias ? bias[16 * c + e] : 0.0f;
        v[e] = fmaxf(__uint_as_float(r[e]) + b, 0.0f);
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint4 p;
        p.x = pack2<BF16>(v[8 * h + 0], v[8 * h + 1]);
        p.y = pack2<BF16>(v[8 * h + 2], v[8 * h + 3]);
        p.z = pack2<BF16>(v[8 * h + 4], v[8 * h + 5]);
        p.w = pack2<BF16>(v[8 * h + 6], v[8 * h + 7]);
        *reinterpret_cast<uint4*>(sm + L::kA2 + kmajor_offset(row, 16 * c + 8 * h, H)) = p;
      }
    }
  }

  // Runs layers 1-3 on the A1 tile already in shared memory; y = this thread's RGB.
  // Returns false if a barrier wait timed out (uniform across the CTA).
  static __device__ __forceinline__ bool mlp(unsigned char* sm, uint32_t tmem, uint64_t* bar, uint32_t& phase,
                                             int tid, float& y0, float& y1, float& y2) {
    const uint32_t lane = (uint32_t)((tid >> 5) * 32) << 16;
    const uint32_t base = smem_addr(sm);
    const float* bias2 = reinterpret_cast<const float*>(sm + L::kBias2);
    const float* bias3 = reinterpret_cast<const float*>(sm + L::kBias3);
    // layer 1
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) mma_layer(tmem, base + L::kA1, base + L::kB1, L::K1, H, bar);
    bool ok = mbar_wait(bar, phase);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) return false;
    tc_fence_after();
    hidden_epilogue(sm, tmem + lane, tid, nullptr);
    // layer 2
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) mma_layer(tmem + H, base + L::kA2, base + L::kB2, H, H, bar);
    ok = mbar_wait(bar, phase);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) return false;
    tc_fence_after();
    hidden_epilogue(sm, tmem + H + lane, tid, bias2);
    // output layer (N = 16, columns 0..2 used), into the columns of D1
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) mma_layer(tmem, base + L::kA2, base + L::kB3, H, L::N3, bar);
    ok = mbar_wait(bar, phase);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) return false;
    tc_fence_after();
    uint32_t r[16];
    tmem_ld16(tmem + lane, r);
    tmem_ld_wait();
    y0 = __uint_as_float(r[0]) + bias3[0];
    y1 = __uint_as_float(r[1]) + bias3[1];
    y2 = __uint_as_float(r[2]) + bias3[2];
    tc_fence_before();
    return true;
  }

  // CTA start: weight image -> smem, TMEM allocation, barrier init.
  static __device__ __forceinline__ uint32_t setup(unsigned char* sm, const unsigned char* ws, uint64_t* bar,
                                                   uint32_t* slot, int tid) {
    for (uint32_t i = tid * 16; i < L::kWsBytes; i += kTcThreads * 16)
      *reinterpret_cast<uint4*>(sm + i) = *reinterpret_cast<const uint4*>(ws + i);
    if ((tid >> 5) == 0) {
      tmem_alloc(slot, L::kTmemCols);
      tmem_relinquish();
    }
    if (tid == 0) {
      mbar_init(bar, 1);
      mbar_fence_init();
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return *slot;
  }

  // CTA end: after a timeout, wait (bounded) for the MMAs still in flight; free TMEM.
  static __device__ __forceinline__ void teardown(uint32_t tmem, uint64_t* bar, uint32_t phase, bool failed,
                                                  int tid) {
    if (failed) {
      if (tid == 0) atomicOr(&g_tc_error, 1);
      mbar_wait(bar, phase);
    }
    tc_fence_before();
    __syncthreads();
    if ((tid >> 5) == 0) {
      tc_fence_after();
      tmem_dealloc(tmem, L::kTmemCols);
    }
  }
};

// ---------------------------------------------------------------------------
// Random-access points
// ---------------------------------------------------------------------------
template <int CS, int CT, int H, bool BF16>
__global__ void __launch_bounds__(kTcThreads, 4) k_points_tc(DevModel m, const unsigned char* __restrict__ ws,
                                                             const float* __restrict__ uvt, int64_t n,
                                                             float* __restrict__ rgb) {
  using T = TcTile<CS, CT, H, BF16>;
  using L = TcLayout<CS, CT, H>;
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ uint64_t bar;
  __shared__ uint32_t slot;
  const int tid = threadIdx.x;
  const uint32_t tmem = T::setup(sm, ws, &bar, &slot, tid);
  uint32_t phase = 0;
  bool failed = false;
  const int64_t tiles = (n + 127) / 128;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t q = tile * 128 + tid;
    float x[L::CIN];
    if (q < n) {
      gather_f32<CS, CT>(m, uvt[3 * q], uvt[3 * q + 1], uvt[3 * q + 2], x, nullptr);
    } else {
#pragma unroll
      for (int k = 0; k < L::CIN; ++k) x[k] = 0.0f;
    }
    T::write_a1(sm, tid, x);
    float y0, y1, y2;
    if (!T::mlp(sm, tmem, &bar, phase, tid, y0, y1, y2)) {
      failed = true;
      break;
    }
    if (q < n) {
      rgb[3 * q] = y0;
      rgb[3 * q + 1] = y1;
      rgb[3 * q + 2] = y2;
    }
  }
  T::teardown(tmem, &bar, phase, failed, tid);
}

// ---------------------------------------------------------------------------
// Batched pages: persistent CTAs pull work items (request, group of tiles)
// from an atomic counter; a tile is tile_w x (128 / tile_w) texels of the page.
// ---------------------------------------------------------------------------
template <int CS, int CT, int H, bool BF16>
__global__ void __launch_bounds__(kTcThreads, 4) k_pages_tc(PagesCtx c, const ndgi_page_req* __restrict__ reqs,
                                                            const int32_t* __restrict__ n_dev, int tile_w,
                                                            int tiles_per_item) {
  using T = TcTile<CS, CT, H, BF16>;
  using L = TcLayout<CS, CT, H>;
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ uint64_t bar;
  __shared__ uint32_t slot;
  __shared__ int s_item;
  const int tid = threadIdx.x;
  int n = *n_dev;
  if (n > c.max_reqs || n < 0) {   // reject the whole frame: the request buffer may be shorter
    if (blockIdx.x == 0 && tid == 0) atomicOr(c.error_word, 1);
    n = 0;
  }
  const int tile_h = 128 / tile_w;
  const int items_per_req = (128 / tiles_per_item);     // 128 tiles cover the largest (128 x 128) page
  const int64_t items = (int64_t)n * items_per_req;
  // the first model's weights; reloaded when a work item's model differs
  const uint32_t tmem = T::setup(sm, static_cast<const unsigned char*>(c.ws[0]), &bar, &slot, tid);
  int loaded = 0;
  uint32_t phase = 0;
  bool failed = false;
  for (;;) {
    if (tid == 0) s_item = (int)atomicAdd(c.work_counter, 1u);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if ((int64_t)item >= items) break;
    const ndgi_page_req r = reqs[item / items_per_req];
    const bool valid = r.model >= 0 && r.model < c.n_models && r.w >= 1 && r.w <= 128 && r.h >= 1 && r.h <= 128;
    const int first_tile = (item % items_per_req) * tiles_per_item;
    if (!valid) {
      if (first_tile == 0 && tid == 0) atomicOr(c.error_word, 2);
      continue;
    }
    const DevModel& m = c.models[r.model];
    const bool inside = r.x0 >= 0 && r.y0 >= 0 && (int64_t)r.x0 + r.w <= m.lm_w && (int64_t)r.y0 + r.h <= m.lm_h &&
                        r.dst_x >= 0 && r.dst_y >= 0 && (int64_t)r.dst_x + r.w <= c.phys_w &&
                        (int64_t)r.dst_y + r.h <= c.phys_h;
    if (!inside) {
      if (first_tile == 0 && tid == 0) atomicOr(c.error_word, 4);
      continue;
    }
    const int tiles_x = (r.w + tile_w - 1) / tile_w, tiles_y = (r.h + tile_h - 1) / tile_h;
    const int tiles = tiles_x * tiles_y;
    if (first_tile >= tiles) continue;
    if (r.model != loaded) {        // block-uniform: swap in this model's weight image
      const unsigned char* w = static_cast<const unsigned char*>(c.ws[r.model]);
      for (uint32_t i = tid * 16; i < L::kWsBytes; i += kTcThreads * 16)
        *reinterpret_cast<uint4*>(sm + i) = *reinterpret_cast<const uint4*>(w + i);
      loaded = r.model;            // the next MLP's fence + barrier publishes it to the tensor core
    }
    const int last_tile = min(first_tile + tiles_per_item, tiles);
    for (int t = first_tile; t < last_tile; ++t) {
      const int i = (t % tiles_x) * tile_w + tid % tile_w;
      const int j = (t / tiles_x) * tile_h + tid / tile_w;
      const bool in = i < r.w && j < r.h;
      float x[L::CIN];
      if (in) {
        const float u = ((float)(r.x0 + i) + 0.5f) / (float)m.lm_w;
        const float v = ((float)(r.y0 + j) + 0.5f) / (float)m.lm_h;
        gather_f32<CS, CT>(m, u, v, r.t, x, nullptr);
      } else {
#pragma unroll
        for (int k = 0; k < L::CIN; ++k) x[k] = 0.0f;
      }
      T::write_a1(sm, tid, x);
      float y0, y1, y2;
      if (!T::mlp(sm, tmem, &bar, phase, tid, y0, y1, y2)) {
        failed = true;
        break;
      }
      if (in) {
        const int64_t o = (int64_t)(r.dst_y + j) * c.phys_w + (r.dst_x + i);
        if (c.out_format == NDGI_RGBA32F) {
          reinterpret_cast<float4*>(c.phys)[o] = make_float4(y0, y1, y2, 1.0f);
        } else {
          uint2 p;
          p.x = pack2<false>(y0, y1);
          p.y = pack2<false>(y2, 1.0f);
          reinterpret_cast<uint2*>(c.phys)[o] = p;
        }
      }
    }
    if (failed) break;
  }
  T::teardown(tmem, &bar, phase, failed, tid);
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

size_t tc_workspace_bytes(int cs, int ct, int hidden) {
#define X(A, B, C) if (cs == A && ct == B && hidden == C) return TcLayout<A, B, C>::kWsBytes;
  NDGI_TC_SHAPES(X)
#undef X
  return 0;
}

cudaError_t launch_tc_prepare(const DevModel& m, bool bf16, void* ws, cudaStream_t s) {
#define X(A, B, C)                                                                                       \
  if (m.cs == A && m.ct == B && m.hidden == C) {                                                         \
    if (bf16) k_tc_prepare<A, B, C, true><<<8, 256, 0, s>>>(m, static_cast<unsigned char*>(ws));        \
    else k_tc_prepare<A, B, C, false><<<8, 256, 0, s>>>(m, static_cast<unsigned char*>(ws));            \
    return cudaGetLastError();                                                                           \
  }
  NDGI_TC_SHAPES(X)
#undef X
  return cudaErrorInvalidValue;
}

template <typename K>
static cudaError_t set_smem(K kern, uint32_t bytes) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t launch_tc_points(const DevModel& m, bool bf16, const void* ws, const float* uvt, int64_t n, float* rgb,
                             cudaStream_t s) {
  const int64_t tiles = (n + 127) / 128;
  const int64_t cap = (int64_t)num_sms() * 4;
  const int grid = (int)(tiles < cap ? tiles : cap);
#define X(A, B, C)                                                                                    \
  if (m.cs == A && m.ct == B && m.hidden == C) {                                                      \
    using L = TcLayout<A, B, C>;                                                                      \
    auto kern = bf16 ? k_points_tc<A, B, C, true> : k_points_tc<A, B, C, false>;                       \
    cudaError_t e = set_smem(kern, L::kSmem);                                                         \
    if (e != cudaSuccess) return e;                                                                   \
    kern<<<grid, kTcThreads, L::kSmem, s>>>(m, static_cast<const unsigned char*>(ws), uvt, n, rgb);   \
    return cudaGetLastError();                                                                        \
  }
  NDGI_TC_SHAPES(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t launch_tc_pages(const PagesCtx& c, bool bf16, int cs, int ct, int hidden, const TcPagesShape& shape,
                            const ndgi_page_req* reqs, const int32_t* n_dev, cudaStream_t s) {
  const int grid = num_sms() * shape.ctas_per_sm;
#define X(A, B, C)                                                                                         \
  if (cs == A && ct == B && hidden == C) {                                                                 \
    using L = TcLayout<A, B, C>;                                                                           \
    auto kern = bf16 ? k_pages_tc<A, B, C, true> : k_pages_tc<A, B, C, false>;                              \
    cudaError_t e = set_smem(kern, L::kSmem);                                                              \
    if (e != cudaSuccess) return e;                                                                        \
    kern<<<grid, kTcThreads, L::kSmem, s>>>(c, reqs, n_dev, shape.tile_w, shape.tiles_per_item);           \
    return cudaGetLastError();                                                                             \
  }
  NDGI_TC_SHAPES(X)
#undef X
  return cudaErrorInvalidValue;
}

TcPagesShape tc_default_pages_shape() { return TcPagesShape{4, 16, 16}; }

std::vector<TcPagesShape> tc_pages_candidates(int) {
  std::vector<TcPagesShape> v;
  for (int cps : {2, 3, 4})
    for (int tw : {128, 32, 16})
      for (int tpi : {4, 16, 128}) v.push_back(TcPagesShape{cps, tw, tpi});
  return v;
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
