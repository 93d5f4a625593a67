// BC7 compression of the 8-bit quantised feature maps (Sec. 3.4: after
// training, F_uv and every F3D slice are quantised to 8 bits and compressed
// with BC7 using several modes) and BC7 decode.
//
// Encoder (k_bc7_encode): one thread per 4x4 block, every candidate of a
// fixed list tried in order, the first with the smallest squared error kept:
//   mode 6; mode 5 with rotation 0..3; mode 4 with rotation 0..3 and index
//   selector 0..1; mode 7 with partitions 0..63; for blocks whose alpha is
//   255 everywhere also modes 3, 1, 2 (partitions 0..63) and 0 (0..15).
// Per candidate, subset and endpoint group (colour and alpha separately in
// modes 4 and 5), the endpoints are the corners of the subset's per-channel
// bounding box on the diagonal along the data (a channel runs from maximum to
// minimum when its integer covariance with the widest channel is negative),
// each coded by its nearest code (a 256-entry table per
// code width and p-bit, built per CTA by exhaustive search, lowest code on
// ties; a p-bit per endpoint or per subset picks the smaller summed squared
// error, 0 on ties); each texel takes its nearest palette entry (lowest index
// on ties).  Everything is integer arithmetic, so the blocks are exact.  The
// winning candidate is re-run to emit its bits, with the anchor fix-up
// (swap a group's endpoints and mirror its indices when an anchor index has
// its top bit set, which leaves the decoded texels unchanged).
#include "ndgi_internal.h"
#include "bc4.cuh"
#include "bc7.cuh"

namespace ndgi {

// Code tables: 4 widths without p-bit (5..8 bits) and 8 with one (4..7 bits, p = 0, 1).
constexpr int kQTables = 12;
__device__ __forceinline__ int qtab_nop(int n) { return n - 5; }
__device__ __forceinline__ int qtab_p(int n, int p) { return 4 + 2 * (n - 4) + p; }

__device__ void build_qtables(uint16_t* qt) {
  for (int i = threadIdx.x; i < kQTables * 256; i += blockDim.x) {
    const int k = i >> 8, v = i & 255;
    int n, p;
    if (k < 4) {
      n = k + 5;
      p = -1;
    } else {
      n = (k - 4) / 2 + 4;
      p = (k - 4) & 1;
    }
    int best = 0, be = 1 << 30, bx = 0;
    for (int q = 0; q < (1 << n); ++q) {
      const int x = p < 0 ? bc7_expand(q, n) : bc7_expand((q << 1) | p, n + 1);
      const int e = abs(x - v);
      if (e < be) {
        be = e;
        best = q;
        bx = x;
      }
    }
    qt[i] = (uint16_t)(best | (bx << 8));
  }
}

__device__ __forceinline__ int chan(uint32_t v, int c) { return (int)((v >> (8 * c)) & 0xffu); }

__device__ __forceinline__ void put_bits(uint64_t& lo, uint64_t& hi, int& pos, int n, uint32_t v) {
  if (n == 0) return;
  const uint64_t x = (uint64_t)v & ((1ull << n) - 1ull);
  if (pos >= 64) {
    hi |= x << (pos - 64);
  } else {
    lo |= x << pos;
    if (pos + n > 64) hi |= x >> (64 - pos);
  }
  pos += n;
}

// Squared error of one candidate; with EMIT also its block.
template <bool EMIT>
__device__ int bc7_try(const uint32_t (&x0)[16], int mode, int part, int rot, int isb, const uint16_t* qt,
                       uint4* out) {
  const Bc7Mode M = bc7_mode(mode);
  uint32_t x[16];
#pragma unroll
  for (int p = 0; p < 16; ++p) {
    uint32_t v = x0[p];
    if (rot) {
      const uint32_t a = (v >> 24) & 0xffu, o = (v >> (8 * (rot - 1))) & 0xffu;
      v = (v & ~(0xffu << 24) & ~(0xffu << (8 * (rot - 1)))) | (o << 24) | (a << (8 * (rot - 1)));
    }
    x[p] = v;
  }
  const bool split = mode == 4 || mode == 5;
  const int ngroups = split ? 2 : 1;
  const int nch = M.ab ? 4 : 3;
  uint32_t sub = 0;   // subset of texel p at bits 2p..2p+1
  if (M.ns == 2) {
    const uint32_t m = __ldg(&kBc7Part2[part]);
#pragma unroll
    for (int p = 0; p < 16; ++p) sub |= ((m >> p) & 1u) << (2 * p);
  } else if (M.ns == 3) {
    sub = __ldg(&kBc7Part3[part]);
  }
  int err = 0;
  int code[3][2][4];
  int pbit[3][2];
  uint8_t idx[2][16];
  for (int g = 0; g < ngroups; ++g) {
    const int c0 = split ? (g ? 3 : 0) : 0, c1 = split ? (g ? 4 : 3) : nch;
    const int n = split ? (g ? M.ab : M.cb) : M.cb;
    const int ib = split ? (mode == 4 ? ((g ? !isb : isb) ? 3 : 2) : 2) : M.ib;
    for (int s = 0; s < M.ns; ++s) {
      int lo[4] = {255, 255, 255, 255}, hi[4] = {0, 0, 0, 0};
      for (int p = 0; p < 16; ++p) {
        if ((int)((sub >> (2 * p)) & 3u) != s) continue;
        for (int c = c0; c < c1; ++c) {
          const int v = chan(x[p], c);
          lo[c] = min(lo[c], v);
          hi[c] = max(hi[c], v);
        }
      }
      // the box diagonal along the data: channel r of largest range runs low to high, another channel high to
      // low when its integer covariance with r is negative
      int r = c0;
      for (int c = c0; c < c1; ++c)
        if (hi[c] - lo[c] > hi[r] - lo[r]) r = c;
      int cnt = 0, sr = 0, sc[4] = {0, 0, 0, 0}, scr[4] = {0, 0, 0, 0};
      for (int p = 0; p < 16; ++p) {
        if ((int)((sub >> (2 * p)) & 3u) != s) continue;
        const int vr = chan(x[p], r);
        ++cnt;
        sr += vr;
        for (int c = c0; c < c1; ++c) {
          const int v = chan(x[p], c);
          sc[c] += v;
          scr[c] += v * vr;
        }
      }
      for (int c = c0; c < c1; ++c)
        if (c != r && cnt * scr[c] - sc[c] * sr < 0) {
          const int t = lo[c];
          lo[c] = hi[c];
          hi[c] = t;
        }
      int val[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
      if (M.epb || M.spb) {
        int pe[2] = {0, 0};
        int cost[2][2] = {{0, 0}, {0, 0}};   // [endpoint][p]
        for (int e = 0; e < 2; ++e)
          for (int p = 0; p < 2; ++p)
            for (int c = c0; c < c1; ++c) {
              const int v = e ? hi[c] : lo[c];
              const int d = (int)(qt[qtab_p(n, p) * 256 + v] >> 8) - v;
              cost[e][p] += d * d;
            }
        if (M.epb) {
          pe[0] = cost[0][1] < cost[0][0];
          pe[1] = cost[1][1] < cost[1][0];
        } else {
          pe[0] = pe[1] = (cost[0][1] + cost[1][1]) < (cost[0][0] + cost[1][0]);
        }
        for (int e = 0; e < 2; ++e) {
          pbit[s][e] = pe[e];
          for (int c = c0; c < c1; ++c) {
            const uint16_t t = qt[qtab_p(n, pe[e]) * 256 + (e ? hi[c] : lo[c])];
            code[s][e][c] = t & 0xff;
            val[e][c] = t >> 8;
          }
        }
      } else {
        for (int e = 0; e < 2; ++e)
          for (int c = c0; c < c1; ++c) {
            const uint16_t t = qt[qtab_nop(n) * 256 + (e ? hi[c] : lo[c])];
            code[s][e][c] = t & 0xff;
            val[e][c] = t >> 8;
          }
      }
      for (int p = 0; p < 16; ++p) {
        if ((int)((sub >> (2 * p)) & 3u) != s) continue;
        int best = 1 << 30, bi = 0;
        for (int i = 0; i < (1 << ib); ++i) {
          const int w = bc7_weight(i, ib);
          int e2 = 0;
          for (int c = c0; c < c1; ++c) {
            const int d = (((64 - w) * val[0][c] + w * val[1][c] + 32) >> 6) - chan(x[p], c);
            e2 += d * d;
          }
          if (e2 < best) {
            best = e2;
            bi = i;
          }
        }
        err += best;
        if (EMIT) idx[g][p] = (uint8_t)bi;
      }
      if (EMIT) {
        int a = 0;
        if (!split && s > 0) {
          const uint32_t an = __ldg(&kBc7Anchors[part]);
          a = M.ns == 2 ? (int)(an & 0xffu) : (int)((an >> (s == 1 ? 8 : 16)) & 0xffu);
        }
        if (idx[g][a] >> (ib - 1)) {
          for (int c = c0; c < c1; ++c) {
            const int t = code[s][0][c];
            code[s][0][c] = code[s][1][c];
            code[s][1][c] = t;
          }
          if (!split) {
            const int t = pbit[s][0];
            pbit[s][0] = pbit[s][1];
            pbit[s][1] = t;
          }
          for (int p = 0; p < 16; ++p)
            if ((int)((sub >> (2 * p)) & 3u) == s) idx[g][p] = (uint8_t)((1 << ib) - 1 - idx[g][p]);
        }
      }
    }
  }
  if (nch == 3)
    for (int p = 0; p < 16; ++p) {
      const int d = 255 - chan(x[p], 3);
      err += d * d;
    }
  if (EMIT) {
    uint64_t lo = 0, hi = 0;
    int pos = 0;
    put_bits(lo, hi, pos, mode + 1, 1u << mode);
    put_bits(lo, hi, pos, M.pb, (uint32_t)part);
    put_bits(lo, hi, pos, M.rb, (uint32_t)rot);
    put_bits(lo, hi, pos, M.isb, (uint32_t)isb);
    for (int c = 0; c < nch; ++c)
      for (int s = 0; s < M.ns; ++s)
        for (int e = 0; e < 2; ++e) put_bits(lo, hi, pos, c < 3 ? M.cb : M.ab, (uint32_t)code[s][e][c]);
    if (M.epb)
      for (int s = 0; s < M.ns; ++s)
        for (int e = 0; e < 2; ++e) put_bits(lo, hi, pos, 1, (uint32_t)pbit[s][e]);
    if (M.spb)
      for (int s = 0; s < M.ns; ++s) put_bits(lo, hi, pos, 1, (uint32_t)pbit[s][0]);
    uint32_t an = M.ns > 1 ? __ldg(&kBc7Anchors[part]) : 0u;
    const int a1 = M.ns == 2 ? (int)(an & 0xffu) : M.ns == 3 ? (int)((an >> 8) & 0xffu) : 16;
    const int a2 = M.ns == 3 ? (int)((an >> 16) & 0xffu) : 16;
    const int gp = (mode == 4 && isb) ? 1 : 0;
    for (int p = 0; p < 16; ++p) {
      const bool anchor = p == 0 || p == a1 || p == a2;
      put_bits(lo, hi, pos, M.ib - (anchor ? 1 : 0), idx[gp][p]);
    }
    if (M.ib2)
      for (int p = 0; p < 16; ++p) put_bits(lo, hi, pos, M.ib2 - (p == 0), idx[1 - gp][p]);
    *out = make_uint4((uint32_t)lo, (uint32_t)(lo >> 32), (uint32_t)hi, (uint32_t)(hi >> 32));
  }
  return err;
}

__global__ void __launch_bounds__(128) k_bc7_encode(const uint4* __restrict__ rgba, int bw, int64_t n_blocks,
                                                    uint4* __restrict__ out, unsigned long long* __restrict__ err) {
  __shared__ uint16_t qt[kQTables * 256];
  build_qtables(qt);
  __syncthreads();
  const int w4 = bw;   // uint4 (4 texels) per image row = bw
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n_blocks;
       b += (int64_t)gridDim.x * blockDim.x) {
    const int64_t by = b / bw, bx = b % bw;
    uint32_t x[16];
    bool opaque = true;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const uint4 v = __ldg(rgba + (4 * by + r) * w4 + bx);
      x[4 * r] = v.x;
      x[4 * r + 1] = v.y;
      x[4 * r + 2] = v.z;
      x[4 * r + 3] = v.w;
    }
#pragma unroll
    for (int p = 0; p < 16; ++p) opaque &= (x[p] >> 24) == 255u;
    int best = 1 << 30, bm = 6, bp = 0, br = 0, bi = 0;
    auto consider = [&](int mode, int part, int rot, int isb) {
      const int e = bc7_try<false>(x, mode, part, rot, isb, qt, nullptr);
      if (e < best) {
        best = e;
        bm = mode;
        bp = part;
        br = rot;
        bi = isb;
      }
    };
    consider(6, 0, 0, 0);
    for (int r = 0; r < 4; ++r) consider(5, 0, r, 0);
    for (int r = 0; r < 4; ++r)
      for (int i = 0; i < 2; ++i) consider(4, 0, r, i);
    for (int q = 0; q < 64; ++q) consider(7, q, 0, 0);
    if (opaque) {
      for (int q = 0; q < 64; ++q) consider(3, q, 0, 0);
      for (int q = 0; q < 64; ++q) consider(1, q, 0, 0);
      for (int q = 0; q < 64; ++q) consider(2, q, 0, 0);
      for (int q = 0; q < 16; ++q) consider(0, q, 0, 0);
    }
    uint4 blk;
    bc7_try<true>(x, bm, bp, br, bi, qt, &blk);
    out[b] = blk;
    if (err) atomicAdd(err, (unsigned long long)best);
  }
}

__global__ void k_bc7_decode(const uint4* __restrict__ blocks, int bw, int64_t n_blocks, uint4* __restrict__ rgba) {
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n_blocks;
       b += (int64_t)gridDim.x * blockDim.x) {
    uint32_t px[16];
    bc7_block(__ldg(blocks + b), px);
    const int64_t by = b / bw, bx = b % bw;
#pragma unroll
    for (int r = 0; r < 4; ++r)
      rgba[(4 * by + r) * bw + bx] = make_uint4(px[4 * r], px[4 * r + 1], px[4 * r + 2], px[4 * r + 3]);
  }
}

// 8-bit quantisation of four BC4 planes: round(255 P35 / 8925) = round(P35 / 35) per channel (no ties).
__global__ void k_bc4x4_to_rgba8(const uint4* __restrict__ bc4, int bw, int64_t n_blocks, uint4* __restrict__ rgba) {
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n_blocks;
       b += (int64_t)gridDim.x * blockDim.x) {
    const uint4 a = __ldg(bc4 + 2 * b), c = __ldg(bc4 + 2 * b + 1);
    const uint32_t lo[4] = {a.x, a.z, c.x, c.z}, hi[4] = {a.y, a.w, c.y, c.w};
    const int64_t by = b / bw, bx = b % bw;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      uint32_t o[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int p = 4 * r + q;
        uint32_t v = 0;
#pragma unroll
        for (int ch = 0; ch < 4; ++ch) {
          const uint64_t blk = (uint64_t)lo[ch] | ((uint64_t)hi[ch] << 32);
          const int r0 = (int)(blk & 255u), r1 = (int)((blk >> 8) & 255u);
          const int k = (int)((blk >> (16 + 3 * p)) & 7u);
          int p35;
          if (k == 0) p35 = 35 * r0;
          else if (k == 1) p35 = 35 * r1;
          else if (r0 > r1) p35 = 5 * ((8 - k) * r0 + (k - 1) * r1);
          else if (k == 6) p35 = 0;
          else if (k == 7) p35 = 8925;
          else p35 = 7 * ((6 - k) * r0 + (k - 1) * r1);
          v |= (uint32_t)((p35 + 17) / 35) << (8 * ch);
        }
        o[q] = v;
      }
      rgba[(4 * by + r) * bw + bx] = make_uint4(o[0], o[1], o[2], o[3]);
    }
  }
}

// 8-bit export of a shared-weight BC simulation (Eq. 7 with one weight per
// texel): texel value ((64 - W) A + W B + 32) >> 6 per channel with A, B the
// mode-6 endpoints of ea, eb and W the 4-bit BC7 weight of index q15(w).  One
// thread per block.
__device__ __forceinline__ int mode6_endpoint(const float* __restrict__ e, int (&E)[4]) {
  int q[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) q[c] = quant(__ldg(e + c), 255.0f);
  return bc7_mode6_endpoint(q, E);
}

__global__ void k_bc_sim7_to_rgba8(const float* __restrict__ ea, const float* __restrict__ eb,
                                   const float* __restrict__ w, int bw, int64_t n_blocks, uint4* __restrict__ rgba) {
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n_blocks;
       b += (int64_t)gridDim.x * blockDim.x) {
    int A[4], B[4];
    mode6_endpoint(ea + 4 * b, A);
    mode6_endpoint(eb + 4 * b, B);
    const int64_t by = b / bw, bx = b % bw;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      uint32_t o[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int W = bc7_weight(quant(__ldg(w + 16 * b + 4 * r + q), 15.0f), 4);
        uint32_t v = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c) v |= (uint32_t)(((64 - W) * A[c] + W * B[c] + 32) >> 6) << (8 * c);
        o[q] = v;
      }
      rgba[(4 * by + r) * bw + bx] = make_uint4(o[0], o[1], o[2], o[3]);
    }
  }
}

// Exact mode-6 blocks of a shared-weight BC simulation: the mode-6 endpoint
// codes and p-bits, indices q15(w); where texel 0's index is 8 or more the
// endpoints swap and every index k becomes 15 - k (symmetric weights).
__global__ void k_bc7_pack_sim(const float* __restrict__ ea, const float* __restrict__ eb,
                               const float* __restrict__ w, int64_t n_blocks, uint4* __restrict__ out) {
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n_blocks;
       b += (int64_t)gridDim.x * blockDim.x) {
    int A[4], B[4], k[16];
    int pa = mode6_endpoint(ea + 4 * b, A), pb = mode6_endpoint(eb + 4 * b, B);
#pragma unroll
    for (int p = 0; p < 16; ++p) k[p] = quant(__ldg(w + 16 * b + p), 15.0f);
    if (k[0] >= 8) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int t = A[c];
        A[c] = B[c];
        B[c] = t;
      }
      const int t = pa;
      pa = pb;
      pb = t;
#pragma unroll
      for (int p = 0; p < 16; ++p) k[p] = 15 - k[p];
    }
    uint64_t lo = 0, hi = 0;
    int pos = 0;
    put_bits(lo, hi, pos, 7, 1u << 6);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      put_bits(lo, hi, pos, 7, (uint32_t)(A[c] >> 1));
      put_bits(lo, hi, pos, 7, (uint32_t)(B[c] >> 1));
    }
    put_bits(lo, hi, pos, 1, (uint32_t)pa);
    put_bits(lo, hi, pos, 1, (uint32_t)pb);
#pragma unroll
    for (int p = 0; p < 16; ++p) put_bits(lo, hi, pos, p == 0 ? 3 : 4, (uint32_t)k[p]);
    out[b] = make_uint4((uint32_t)lo, (uint32_t)(lo >> 32), (uint32_t)hi, (uint32_t)(hi >> 32));
  }
}

// Fixed-function reference: the texture unit's own BC7 decode, point-sampled at texel centres.
__global__ void k_bc7_tex_fetch(cudaTextureObject_t tex, int w, int h, uint32_t* __restrict__ rgba) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)w * h) return;
  const int x = (int)(i % w), y = (int)(i / w);
  const float4 v = tex2D<float4>(tex, (float)x + 0.5f, (float)y + 0.5f);
  const uint32_t r = (uint32_t)__float2int_rn(v.x * 255.0f), g = (uint32_t)__float2int_rn(v.y * 255.0f);
  const uint32_t b = (uint32_t)__float2int_rn(v.z * 255.0f), a = (uint32_t)__float2int_rn(v.w * 255.0f);
  rgba[i] = r | (g << 8) | (b << 16) | (a << 24);
}

static int grid_for(int64_t n, int threads, int per_sm) {
  int64_t g = (n + threads - 1) / threads;
  const int64_t cap = (int64_t)num_sms() * per_sm;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

static ndgi_status check_image(const void* a, const void* b, int32_t w, int32_t h, const char* who) {
  if (!a || !b) return set_error(NDGI_ERR_INVALID_ARG, "%s: NULL buffer", who);
  if (w <= 0 || h <= 0 || w % 4 || h % 4)
    return set_error(NDGI_ERR_INVALID_ARG, "%s: w and h must be positive multiples of 4 (got %d x %d)", who, w, h);
  if ((uintptr_t)a % 16 || (uintptr_t)b % 16) return set_error(NDGI_ERR_INVALID_ARG, "%s: buffers must be 16-byte aligned", who);
  return NDGI_OK;
}

}  // namespace ndgi

using namespace ndgi;

extern "C" {

ndgi_status ndgi_bc7_encode(const uint8_t* rgba, int32_t w, int32_t h, uint8_t* blocks, uint64_t* sq_err,
                            void* stream) {
  ndgi_status st = check_image(rgba, blocks, w, h, "ndgi_bc7_encode");
  if (st != NDGI_OK) return st;
  if ((uintptr_t)sq_err % 8)   // the 64-bit atomic accumulation needs an 8-byte aligned word
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_bc7_encode: sq_err must be 8-byte aligned");
  const int bw = w / 4;
  const int64_t n = (int64_t)bw * (h / 4);
  k_bc7_encode<<<grid_for(n, 128, 8), 128, 0, (cudaStream_t)stream>>>(
      reinterpret_cast<const uint4*>(rgba), bw, n, reinterpret_cast<uint4*>(blocks),
      reinterpret_cast<unsigned long long*>(sq_err));
  return cuda_status(cudaGetLastError(), "ndgi_bc7_encode");
}

ndgi_status ndgi_bc7_decode(const uint8_t* blocks, int32_t w, int32_t h, uint8_t* rgba, void* stream) {
  ndgi_status st = check_image(blocks, rgba, w, h, "ndgi_bc7_decode");
  if (st != NDGI_OK) return st;
  const int bw = w / 4;
  const int64_t n = (int64_t)bw * (h / 4);
  k_bc7_decode<<<grid_for(n, 256, 16), 256, 0, (cudaStream_t)stream>>>(reinterpret_cast<const uint4*>(blocks), bw, n,
                                                                         reinterpret_cast<uint4*>(rgba));
  return cuda_status(cudaGetLastError(), "ndgi_bc7_decode");
}

ndgi_status ndgi_bc4x4_to_rgba8(const uint8_t* bc4, int32_t w, int32_t h, uint8_t* rgba, void* stream) {
  ndgi_status st = check_image(bc4, rgba, w, h, "ndgi_bc4x4_to_rgba8");
  if (st != NDGI_OK) return st;
  const int bw = w / 4;
  const int64_t n = (int64_t)bw * (h / 4);
  k_bc4x4_to_rgba8<<<grid_for(n, 256, 16), 256, 0, (cudaStream_t)stream>>>(reinterpret_cast<const uint4*>(bc4), bw,
                                                                             n, reinterpret_cast<uint4*>(rgba));
  return cuda_status(cudaGetLastError(), "ndgi_bc4x4_to_rgba8");
}

ndgi_status ndgi_bc_sim7_to_rgba8(const float* ea, const float* eb, const float* w, int32_t width, int32_t height,
                                  uint8_t* rgba, void* stream) {
  ndgi_status st = check_image(ea, rgba, width, height, "ndgi_bc_sim7_to_rgba8");
  if (st != NDGI_OK) return st;
  if (!eb || !w || (uintptr_t)eb % 16 || (uintptr_t)w % 16)
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_bc_sim7_to_rgba8: eb and w must be non-NULL and 16-byte aligned");
  const int bw = width / 4;
  const int64_t n = (int64_t)bw * (height / 4);
  k_bc_sim7_to_rgba8<<<grid_for(n, 256, 16), 256, 0, (cudaStream_t)stream>>>(ea, eb, w, bw, n,
                                                                              reinterpret_cast<uint4*>(rgba));
  return cuda_status(cudaGetLastError(), "ndgi_bc_sim7_to_rgba8");
}

ndgi_status ndgi_bc7_pack_sim(const float* ea, const float* eb, const float* w, int64_t n_blocks, uint8_t* blocks,
                              void* stream) {
  if (!ea || !eb || !w || !blocks || n_blocks < 0)
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_bc7_pack_sim: NULL buffer or n_blocks < 0");
  if ((uintptr_t)ea % 16 || (uintptr_t)eb % 16 || (uintptr_t)w % 16 || (uintptr_t)blocks % 16)
    return set_error(NDGI_ERR_INVALID_ARG, "ndgi_bc7_pack_sim: buffers must be 16-byte aligned");
  if (n_blocks == 0) return NDGI_OK;
  k_bc7_pack_sim<<<grid_for(n_blocks, 256, 16), 256, 0, (cudaStream_t)stream>>>(ea, eb, w, n_blocks,
                                                                                 reinterpret_cast<uint4*>(blocks));
  return cuda_status(cudaGetLastError(), "ndgi_bc7_pack_sim");
}

ndgi_status ndgi_debug_bc7_hw_decode(const uint8_t* blocks, int32_t w, int32_t h, uint8_t* rgba, void* stream) {
  ndgi_status st = check_image(blocks, rgba, w, h, "ndgi_debug_bc7_hw_decode");
  if (st != NDGI_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int bw = w / 4, bh = h / 4;
  // the blocks as a CUDA array of 32-bit x 4 elements, viewed as BC7 texels
  cudaChannelFormatDesc fmt = cudaCreateChannelDesc(32, 32, 32, 32, cudaChannelFormatKindUnsigned);
  cudaArray_t arr = nullptr;
  cudaError_t e = cudaMallocArray(&arr, &fmt, (size_t)bw, (size_t)bh);
  if (e != cudaSuccess) return cuda_status(e, "ndgi_debug_bc7_hw_decode: array");
  e = cudaMemcpy2DToArrayAsync(arr, 0, 0, blocks, (size_t)bw * 16, (size_t)bw * 16, (size_t)bh,
                               cudaMemcpyDeviceToDevice, s);
  cudaTextureObject_t tex = 0;
  if (e == cudaSuccess) {
    cudaResourceDesc res{};
    res.resType = cudaResourceTypeArray;
    res.res.array.array = arr;
    cudaTextureDesc td{};
    td.addressMode[0] = td.addressMode[1] = cudaAddressModeClamp;
    td.filterMode = cudaFilterModePoint;
    td.readMode = cudaReadModeElementType;
    td.normalizedCoords = 0;
    cudaResourceViewDesc view{};
    view.format = cudaResViewFormatUnsignedBlockCompressed7;
    view.width = (size_t)w;
    view.height = (size_t)h;
    e = cudaCreateTextureObject(&tex, &res, &td, &view);
  }
  if (e == cudaSuccess) {
    const int64_t n = (int64_t)w * h;
    k_bc7_tex_fetch<<<(int)((n + 255) / 256), 256, 0, s>>>(tex, w, h, reinterpret_cast<uint32_t*>(rgba));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (tex) cudaDestroyTextureObject(tex);
  cudaFreeArray(arr);
  return cuda_status(e, "ndgi_debug_bc7_hw_decode");
}

}  // extern "C"
