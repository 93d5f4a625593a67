// Tensor-core random-access point decode (Sec. 3.1, Eq. 3): one thread per
// query gathers its features, a lane of 128 threads runs the MLP of its
// 128-query tile on tcgen05 (tc_engine.cuh).  Also the gather-only kernels
// used to validate the tensor-core gathers.
//
// Two gathers.  Direct: every query decodes the BC4 palette entries of its
// four taps (16 planes x 4 taps = 64 palette decodes) from the texel-sliced
// planes.  Through a decoded-texel cache: when a call has many queries per
// feature texel, it first decodes every BC4 texel of the map once into an FP16
// texel cache in the workspace ([feat_h][feat_w][cs], at most 64 MiB so it
// stays in L2), then each query blends its four cached taps in half2
// arithmetic, as the page decode blends its decoded feature rows.  The cache is
// rebuilt by every call (it is part of the decode, not of ndgi_prepare).
#include "tc_engine.cuh"

namespace ndgi {

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

// Builds the decoded-texel cache: texel (x, y), plane c -> FP16 of
// fl32(P35) * fl32(1/8925), the same value and the same FP16 rounding as the
// page decode's feature ring.  One thread per texel; consecutive threads
// write consecutive 2*CS-byte entries.
template <int CS>
__global__ void __launch_bounds__(256) k_feature_cache(int feat_w, int feat_h, int bw, const uint8_t* __restrict__ sl,
                                                       unsigned char* __restrict__ cache) {
  using SL = Sliced<CS>;
  static_assert(CS % 4 == 0, "cache entries are whole 8-byte words");
  __shared__ uint2 luts[16];
  init_p35_lut_sliced(luts, threadIdx.x);
  __syncthreads();
  const int64_t ntex = (int64_t)feat_w * feat_h;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ntex; i += (int64_t)gridDim.x * blockDim.x) {
    const int y = (int)(i / feat_w), x = (int)(i - (int64_t)y * feat_w);
    const uint8_t* base = sl + ((size_t)(y >> 2) * bw + (x >> 2)) * SL::BLOCK;
    const int p = ((y & 3) << 2) | (x & 3);
    uint32_t ew[SL::EP / 4];
#pragma unroll
    for (int k = 0; k < SL::EP / 16; ++k) {
      const uint4 e = __ldg(reinterpret_cast<const uint4*>(base) + k);
      ew[4 * k] = e.x;
      ew[4 * k + 1] = e.y;
      ew[4 * k + 2] = e.z;
      ew[4 * k + 3] = e.w;
    }
    const uint2 ix = __ldg(reinterpret_cast<const uint2*>(base + SL::EP) + p);
    uint32_t h[CS / 2];
#pragma unroll
    for (int j = 0; j < CS / 2; ++j) {
      const uint2 el = luts[nibble_at(ix, 2 * j)], eh = luts[nibble_at(ix, 2 * j + 1)];
      const float f0 = __fmul_rn(__uint_as_float(__dp2a_lo(el.x, ew[j], el.y)) - 8388608.0f, kInv8925);
      const float f1 = __fmul_rn(__uint_as_float(__dp2a_hi(eh.x, ew[j], eh.y)) - 8388608.0f, kInv8925);
      h[j] = pack2<false>(f0, f1);
    }
    unsigned char* dst = cache + (size_t)i * (CS * 2);
#pragma unroll
    for (int j = 0; j + 4 <= CS / 2; j += 4)
      *reinterpret_cast<uint4*>(dst + 4 * j) = make_uint4(h[j], h[j + 1], h[j + 2], h[j + 3]);
    if constexpr ((CS / 2) % 4 == 2)
      *reinterpret_cast<uint2*>(dst + 4 * (CS / 2 - 2)) = make_uint2(h[CS / 2 - 2], h[CS / 2 - 1]);
  }
}

// The spatial features of one query from the decoded-texel cache: the same
// taps and fractions as the direct gather (axis_setup), blended in half2 as
// the page decode does (weights rounded to FP16, products and sums rounded
// once each): sw[j] holds planes 2j, 2j+1.
template <int CS>
__device__ __forceinline__ void gather_cache_spatial(const DevModel& m, const unsigned char* __restrict__ cache,
                                                     float u, float v, uint32_t (&sw)[CS / 2]) {
  int x0, x1, y0, y1;
  float fx, fy;
  axis_setup(u, m.feat_w, m.address_mode, x0, x1, fx);
  axis_setup(v, m.feat_h, m.address_mode, y0, y1, fy);
  const __half2 wx1 = __float2half2_rn(fx), wx0 = __float2half2_rn(1.0f - fx);
  const __half2 wy1 = __float2half2_rn(fy), wy0 = __float2half2_rn(1.0f - fy);
  const __half2 w00 = __hmul2(wx0, wy0), w10 = __hmul2(wx1, wy0), w01 = __hmul2(wx0, wy1), w11 = __hmul2(wx1, wy1);
  constexpr size_t kTex = CS * 2;   // bytes per cached texel
  const unsigned char* r0 = cache + (size_t)y0 * m.feat_w * kTex;
  const unsigned char* r1 = cache + (size_t)y1 * m.feat_w * kTex;
  const unsigned char* tp[4] = {r0 + x0 * kTex, r0 + x1 * kTex, r1 + x0 * kTex, r1 + x1 * kTex};
  constexpr int NV = CS / 8 > 0 ? CS / 8 : 1;   // 16-byte loads per tap (CS = 4: one 8-byte load)
  uint32_t tw[4][CS / 2];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if constexpr (CS >= 8) {
#pragma unroll
      for (int g = 0; g < NV; ++g) {
        const uint4 a = __ldg(reinterpret_cast<const uint4*>(tp[q]) + g);
        tw[q][4 * g] = a.x;
        tw[q][4 * g + 1] = a.y;
        tw[q][4 * g + 2] = a.z;
        tw[q][4 * g + 3] = a.w;
      }
    } else {
      const uint2 a = __ldg(reinterpret_cast<const uint2*>(tp[q]));
      tw[q][0] = a.x;
      tw[q][1] = a.y;
    }
  }
#pragma unroll
  for (int j = 0; j < CS / 2; ++j) {
    __half2 r = __hmul2(w00, *reinterpret_cast<const __half2*>(&tw[0][j]));
    r = __hfma2(w10, *reinterpret_cast<const __half2*>(&tw[1][j]), r);
    r = __hfma2(w01, *reinterpret_cast<const __half2*>(&tw[2][j]), r);
    r = __hfma2(w11, *reinterpret_cast<const __half2*>(&tw[3][j]), r);
    sw[j] = *reinterpret_cast<const uint32_t*>(&r);
  }
}

// The temporal feature (linear interpolation of the two keyframe rows around
// t, in FP32) exactly as the direct gather computes it.
template <int CT>
__device__ __forceinline__ void gather_temporal(const DevModel& m, float t, float (&xt)[CT]) {
  int j0, j1;
  float a;
  temporal_setup_k(t, m.t_count, m.key_t, j0, j1, a);
  const float ga = 1.0f - a;
  const bool vec = (reinterpret_cast<uintptr_t>(m.temporal) & 15u) == 0u;
  if (CT % 8 == 0 && m.temporal_f16 && vec) {
    const uint4* q0 = reinterpret_cast<const uint4*>(static_cast<const __half*>(m.temporal) + (size_t)j0 * CT);
    const uint4* q1 = reinterpret_cast<const uint4*>(static_cast<const __half*>(m.temporal) + (size_t)j1 * CT);
#pragma unroll
    for (int g = 0; g < (CT % 8 == 0 ? CT / 8 : 0); ++g) {
      const uint4 k0 = __ldg(q0 + g), k1 = __ldg(q1 + g);
      const uint32_t w0[4] = {k0.x, k0.y, k0.z, k0.w}, w1[4] = {k1.x, k1.y, k1.z, k1.w};
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const float2 f0 = __half22float2(*reinterpret_cast<const __half2*>(&w0[h]));
        const float2 f1 = __half22float2(*reinterpret_cast<const __half2*>(&w1[h]));
        xt[8 * g + 2 * h] = ga * f0.x + a * f1.x;
        xt[8 * g + 2 * h + 1] = ga * f0.y + a * f1.y;
      }
    }
  } else {
#pragma unroll
    for (int c = 0; c < CT; ++c) {
      const float k0 = load_temporal(m.temporal, m.temporal_f16, j0 * CT + c);
      const float k1 = load_temporal(m.temporal, m.temporal_f16, j1 * CT + c);
      xt[c] = ga * k0 + a * k1;
    }
  }
}

// Layer-1 words of one query on the cache path: the blended spatial half2
// words (converted for BF16), then the temporal features, the ones column
// for b1 and zeros.
template <int CS, int CT, int K1, bool BF16>
__device__ __forceinline__ void pack_a1_cache(const uint32_t (&sw)[CS / 2], const float (&xt)[CT],
                                              uint32_t (&w)[K1 / 2]) {
  constexpr int CIN = CS + CT;
#pragma unroll
  for (int j = 0; j < CS / 2; ++j) {
    if constexpr (BF16) {
      const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&sw[j]));
      w[j] = pack2<true>(f.x, f.y);
    } else {
      w[j] = sw[j];
    }
  }
#pragma unroll
  for (int j = CS / 2; j < K1 / 2; ++j) {
    float v[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int k = 2 * j + e;
      v[e] = k < CIN ? xt[k < CIN ? k - CS : 0] : (k == CIN ? 1.0f : 0.0f);
    }
    w[j] = pack2<BF16>(v[0], v[1]);
  }
}

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

// CACHE: gather through the decoded-texel cache `cache` (built by
// k_feature_cache earlier on the stream) instead of the direct gather.
template <int CS, int CT, int H, bool BF16, int NWG, int SL, bool CACHE>
__global__ void __launch_bounds__(kLaneThreads* NWG, 1) k_points_tc(DevModel m, const unsigned char* __restrict__ ws,
                                                                    const float* __restrict__ uvt, int64_t n,
                                                                    float* __restrict__ rgb, int* err,
                                                                    const unsigned char* __restrict__ cache) {
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
  if (*reinterpret_cast<const int*>(ws + L::kDbgOff) & kDbgInjectTimeout) inject_timeout(e);
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
    uint32_t w[L::K1P / 2];
    if constexpr (CACHE) {
      uint32_t sw[CS / 2];
      float xt[CT];
      if (q < n) {
        gather_cache_spatial<CS>(m, cache, qu, qv, sw);
        gather_temporal<CT>(m, qt, xt);
      } else {
#pragma unroll
        for (int k = 0; k < CS / 2; ++k) sw[k] = 0u;
#pragma unroll
        for (int k = 0; k < CT; ++k) xt[k] = 0.0f;
      }
      pack_a1_cache<CS, CT, L::K1P, BF16>(sw, xt, w);
    } else {
      float x[L::CIN];
      if (q < n) {
        gather_sliced<CS, CT>(m, sliced, qu, qv, qt, x, lut);
      } else {
#pragma unroll
        for (int k = 0; k < L::CIN; ++k) x[k] = 0.0f;
      }
      pack_a1<L::CIN, L::K1P, BF16>(x, w);
    }
    e.write_a1(0, w);
  };
  int64_t tile = lane_id;
  bool started = false;
  if (tile < tiles) {
    produce(tile);
    started = e.layer1(0);   // false only when an injected wait has run out
    timed_out = !started;
  }
  if (started) {
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
  cta_teardown<SL * NWG, E::kSlotCols>(tbase, e, inflight, timed_out, tid, err);
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

// Points: 4 lanes x 1 slot per CTA, one CTA per SM (4 tiles in flight: the
// tensor memory holds 4 slots of 128 columns).
constexpr int kPointsLanes = 4, kPointsSlots = 1;

// ---------------------------------------------------------------------------
// Warp-specialised point decode through the decoded-texel cache.  Each of the
// CTA's kWsLanes lanes (one tensor-memory slot) has two warpgroups:
//   producer  gathers each tile's queries from the cache (half2 blend) and the
//             temporal line into its layer-1 rows: it loads and blends tile k
//             first, then waits for the slot's previous layer 1 to complete,
//             writes the rows and arrives, so the gather's L2 latency overlaps
//             the consumer's MMA chain;
//   consumer  runs [layer 3 of the previous tile + layer 1] -> RGB out,
//             ReLU -> [layer 2] -> ReLU -> A3 and stores the results.
// No lane's issuing thread sits in the CTA's warp 0 (the warp that allocates
// the tensor memory).  With lane 0's issuer there, lane 0's last tile came out
// wrong at hidden width 32 (only there: not at 16 or 64, not with 32-column
// epilogues, not with the issuer in any other warp); the cause was not found,
// and the tests cover every built shape and tile count.
// Both warpgroups walk the same tiles (lane_id, lane_id + lanes, ...).  The
// barrier protocol and the abort handling are those of the warp-specialised
// page decode.
// ---------------------------------------------------------------------------
template <int CS, int CT, int H, bool BF16>
__global__ void __launch_bounds__(2 * kLaneThreads * kWsLanes, 1)
    k_points_ws(DevModel m, const unsigned char* __restrict__ ws, const float* __restrict__ uvt, int64_t n,
                float* __restrict__ rgb, int* err, const unsigned char* __restrict__ cache) {
  constexpr int NL = kWsLanes;
  using L = TcLayout<CS, CT, H>;
  using S = PointsSmem<CS, CT, H>;
  constexpr int P = BF16 ? kBF16 : kF16;
  using E = Engine<H, P, L::K1P, 1>;
  static_assert(NL * E::kSlotCols <= 512, "one slot per lane");
  if constexpr (!E::kMerge) {
    return;   // not launched for this shape (see ws_points_built)
  } else {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ uint64_t bar1[NL], bar2[NL];   // per lane: layer-1 (+ layer-3) and layer-2 completion
  __shared__ uint32_t slot;
  __shared__ int s_abort;
  __shared__ float s_b3[3];
  const int tid = threadIdx.x, wg = tid >> 7, lane = wg & (NL - 1), t = tid & (kLaneThreads - 1);
  const bool producer = wg >= NL;
  // named barriers: 1 + lane ready (256), 5 + lane consumer (128)
  const int bar_ready = 1 + lane, bar_cons = 1 + NL + lane;
  copy16(sm + S::kW, ws, L::kShared, tid, 2 * kLaneThreads * NL);
  copy16(sm + S::kB1, ws + L::kB1P, H * L::K1P * 2, tid, 2 * kLaneThreads * NL);
  if (tid < 3) s_b3[tid] = stored_b3<BF16>(ws + L::kB3, tid, H, L::K2);
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
  e.b3 = s_b3;
  e.lane_off = (uint32_t)(((t >> 5) * 32) << 16);
  e.tmem[0] = tbase + (uint32_t)(lane * E::kSlotCols);
  e.bar[0] = &bar1[lane];
  e.phase[0] = 0;
  e.db1 = sdesc(base + S::kB1, 128u, L::K1P * 2 * 8u);
  e.db2 = sdesc(base + S::kW + L::kB2, 128u, E::K2 * 2 * 8u);
  e.db3 = sdesc(base + S::kW + L::kB3, 128u, E::K2 * 2 * 8u);
  const bool issuer = !producer && t == e.it;
  if (tid == 0 && (*reinterpret_cast<const int*>(ws + L::kDbgOff) & kDbgInjectTimeout)) {
    // injected timeout: a short wait on a phase nothing completes, then the real abort path
    bool done = false;
    for (uint32_t i = 0; i < kInjectSpin && !done; ++i) done = mbar_try_wait_for(&bar1[0], 0u, kInjectHintNs) != 0;
    if (!done) *abort = 1;
  }
  __syncthreads();
  uint32_t ph1 = 0, ph2 = 0;   // parity of the next bar1 / bar2 phase this thread waits for
  bool out1 = false, out2 = false;   // issuer: a commit whose completion it has not seen
  const int64_t tiles = (n + 127) / 128;
  const int64_t lanes = (int64_t)gridDim.x * NL, lane_id = (int64_t)blockIdx.x * NL + lane;
  const int64_t my_tiles = lane_id < tiles ? (tiles - lane_id + lanes - 1) / lanes : 0;
  if (my_tiles > 0) {   // uniform over the lane's two warpgroups
    if (producer) {
      // ---- producer: each tile's layer-1 rows ----
      for (int64_t k = 0; k < my_tiles; ++k) {
        const int64_t q = (lane_id + k * lanes) * 128 + t;
        uint32_t sw[CS / 2];
        float xt[CT];
        if (q < n) {
          const float qu = __ldcs(uvt + 3 * q), qv = __ldcs(uvt + 3 * q + 1), qt = __ldcs(uvt + 3 * q + 2);
          gather_cache_spatial<CS>(m, cache, qu, qv, sw);
          gather_temporal<CT>(m, qt, xt);
        } else {
#pragma unroll
          for (int j = 0; j < CS / 2; ++j) sw[j] = 0u;
#pragma unroll
          for (int j = 0; j < CT; ++j) xt[j] = 0.0f;
        }
        uint32_t w[L::K1P / 2];
        pack_a1_cache<CS, CT, L::K1P, BF16>(sw, xt, w);
        // the slot's layer-1 columns are free once the previous tile's layer 1 has completed
        if (k > 0) ws_wait(&bar1[lane], ph1, abort);
        e.write_a1(0, w);
        tmem_st_wait();
        tc_fence_before();
        // Normally the producer cannot get ahead (it waited for this slot's previous
        // layer 1), so arriving is enough; once the CTA has aborted its waits return
        // at once, and it must sync instead so that it never arrives twice before
        // the consumer's sync of the same barrier generation.
        if (*abort) named_sync(bar_ready, 2 * kLaneThreads);
        else named_arrive(bar_ready, 2 * kLaneThreads);
      }
    } else {
      // ---- consumer: the MMA chain, the epilogues and the stores ----
      auto put = [&](int64_t q, float y0, float y1, float y2) {
        if (q < n) {
          __stcs(rgb + 3 * q, y0);
          __stcs(rgb + 3 * q + 1, y1);
          __stcs(rgb + 3 * q + 2, y2);
        }
      };
      int64_t prev_q = 0;
      for (int64_t k = 0; k < my_tiles; ++k) {
        // this lane's layer-3 rows (previous tile) and the producer's layer-1 rows are written
        tmem_st_wait();
        tc_fence_before();
        named_sync(bar_ready, 2 * kLaneThreads);
        if (issuer && !*abort) {
          tc_fence_after();
          if (k > 0) e.template mma<E::K3 / E::KS, 16>(0, E::kD3Col, E::kACol, e.db3);
          e.template mma<L::K1P / E::KS, H>(0, 0u, E::kA1Col, e.db1);
          umma_commit(&bar1[lane]);
          out1 = true;
        }
        if (ws_wait(&bar1[lane], ph1, abort) && issuer) out1 = false;
        if (k > 0) {   // the previous tile's RGB leaves tensor memory before the layer-2 rows overwrite it
          float y0, y1, y2;
          e.output(0, y0, y1, y2);
          put(prev_q, y0, y1, y2);
        }
        e.template epilogue16<true>(0);
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
        e.template epilogue16<false>(0);
        prev_q = (lane_id + k * lanes) * 128 + t;
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
      put(prev_q, y0, y1, y2);
    }
  }
  // teardown: an issuer that gave up waiting waits (bounded) for its MMAs
  // before the tensor memory is freed
  if (issuer) {
    if (out1 && !mbar_wait(&bar1[lane], ph1)) atomicOr(err, kErrTimeout);
    if (out2 && !mbar_wait(&bar2[lane], ph2)) atomicOr(err, kErrTimeout);
  }
  if (tid == 0 && *abort) atomicOr(err, kErrTimeout);
  tc_fence_before();
  __syncthreads();
  if ((tid >> 5) == 0) {
    tc_fence_after();
    tmem_dealloc(tbase, tmem_alloc_cols(NL * E::kSlotCols));
  }
  }
}

bool tc_points_cache_path(const DevModel& m, int64_t n, int mode) {
  if (mode == kPointsDirect || points_cache_bytes(m.cs, m.feat_w, m.feat_h) == 0) return false;
  if (mode == kPointsBuild || mode == kPointsReuse) return true;
  return 2 * n >= (int64_t)m.feat_w * m.feat_h;
}

// The warp-specialised point kernel needs the merged slot layout (layer 3
// issued with the next tile's layer 1) in a quarter of the tensor memory.
template <int CS, int CT, int H>
constexpr bool ws_points_built() {
  return kPointsLanes == kWsLanes && Engine<H, kF16, TcLayout<CS, CT, H>::K1P, 1>::kMerge;
}

template <int CS, int CT, int H>
static cudaError_t build_cache(const DevModel& m, const void* ws, cudaStream_t s) {
  const unsigned char* w = static_cast<const unsigned char*>(ws);
  unsigned char* cache = const_cast<unsigned char*>(w) + points_cache_offset<CS, CT, H>(m.feat_w, m.feat_h);
  const int64_t ntex = (int64_t)m.feat_w * m.feat_h;
  const int grid = (int)std::min<int64_t>((ntex + 255) / 256, (int64_t)num_sms() * 8);
  k_feature_cache<CS><<<grid > 0 ? grid : 1, 256, 0, s>>>(m.feat_w, m.feat_h, m.bw, w + TcLayout<CS, CT, H>::kSliceOff,
                                                          cache);
  return cudaGetLastError();
}

bool tc_points_ws_built(int cs, int ct, int hidden) {
#define X(A, B, C) if (cs == A && ct == B && hidden == C) return ws_points_built<A, B, C>();
  NDGI_TC_SHAPES(X)
#undef X
  return false;
}

cudaError_t launch_tc_points(const DevModel& m, bool bf16, const void* ws, const float* uvt, int64_t n, float* rgb,
                             cudaStream_t s, int mode) {
  const int64_t tiles = (n + 127) / 128;
  const int64_t need = (tiles + kPointsLanes * kPointsSlots - 1) / (kPointsLanes * kPointsSlots);
  const int64_t cap = num_sms();
  const int grid = (int)(need < cap ? need : cap);
  const bool cached = tc_points_cache_path(m, n, mode);
#define X(A, B, C)                                                                                              \
  if (m.cs == A && m.ct == B && m.hidden == C) {                                                                \
    using S = PointsSmem<A, B, C>;                                                                              \
    if (cached && mode != kPointsReuse) {                                                                       \
      cudaError_t eb = build_cache<A, B, C>(m, ws, s);                                                          \
      if (eb != cudaSuccess) return eb;                                                                         \
    }                                                                                                           \
    const uint32_t smem = tc_smem(S::kBytes);                                                                   \
    unsigned char* w = static_cast<unsigned char*>(const_cast<void*>(ws));                                      \
    int* err = reinterpret_cast<int*>(w + TcLayout<A, B, C>::kErrOff);                                          \
    const unsigned char* cache = cached ? w + points_cache_offset<A, B, C>(m.feat_w, m.feat_h) : nullptr;       \
    if (cached && ws_points_built<A, B, C>()) {                                                                 \
      auto kern = bf16 ? k_points_ws<A, B, C, true> : k_points_ws<A, B, C, false>;                              \
      cudaError_t e = set_smem(kern, smem);                                                                     \
      if (e != cudaSuccess) return e;                                                                           \
      kern<<<grid, 2 * kLaneThreads * kWsLanes, smem, s>>>(m, w, uvt, n, rgb, err, cache);                     \
      return cudaGetLastError();                                                                                \
    }                                                                                                           \
    auto kern = cached ? (bf16 ? k_points_tc<A, B, C, true, kPointsLanes, kPointsSlots, true>                   \
                               : k_points_tc<A, B, C, false, kPointsLanes, kPointsSlots, true>)                 \
                       : (bf16 ? k_points_tc<A, B, C, true, kPointsLanes, kPointsSlots, false>                  \
                               : k_points_tc<A, B, C, false, kPointsLanes, kPointsSlots, false>);               \
    cudaError_t e = set_smem(kern, smem);                                                                       \
    if (e != cudaSuccess) return e;                                                                             \
    kern<<<grid, kLaneThreads * kPointsLanes, smem, s>>>(m, w, uvt, n, rgb, err, cache);                       \
    return cudaGetLastError();                                                                                  \
  }
  NDGI_TC_SHAPES(X)
#undef X
  return cudaErrorInvalidValue;
}

// The cache path's features alone, for validation: x [n][cs+ct] FP32 of the
// FP16 blend and the FP32 temporal feature.
template <int CS, int CT>
__global__ void __launch_bounds__(128) k_debug_features_cache(DevModel m, const unsigned char* __restrict__ cache,
                                                              const float* __restrict__ uvt, int64_t n,
                                                              float* __restrict__ xo) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t sw[CS / 2];
    float xt[CT];
    gather_cache_spatial<CS>(m, cache, uvt[3 * i], uvt[3 * i + 1], sw);
    gather_temporal<CT>(m, uvt[3 * i + 2], xt);
#pragma unroll
    for (int j = 0; j < CS / 2; ++j) {
      const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&sw[j]));
      xo[i * (CS + CT) + 2 * j] = f.x;
      xo[i * (CS + CT) + 2 * j + 1] = f.y;
    }
#pragma unroll
    for (int c = 0; c < CT; ++c) xo[i * (CS + CT) + CS + c] = xt[c];
  }
}

cudaError_t launch_debug_features_cache(const DevModel& m, const void* ws, const float* uvt, int64_t n, float* x,
                                        cudaStream_t s) {
  if (points_cache_bytes(m.cs, m.feat_w, m.feat_h) == 0) return cudaErrorInvalidValue;
  const int64_t blocks = (n + 127) / 128;
  const int grid = (int)std::min<int64_t>(blocks > 0 ? blocks : 1, (int64_t)num_sms() * 16);
#define X(A, B, C)                                                                                              \
  if (m.cs == A && m.ct == B && m.hidden == C) {                                                                \
    cudaError_t e = build_cache<A, B, C>(m, ws, s);                                                             \
    if (e != cudaSuccess) return e;                                                                             \
    k_debug_features_cache<A, B><<<grid, 128, 0, s>>>(                                                          \
        m, static_cast<const unsigned char*>(ws) + points_cache_offset<A, B, C>(m.feat_w, m.feat_h), uvt, n, x); \
    return cudaGetLastError();                                                                                  \
  }
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

}  // namespace ndgi
